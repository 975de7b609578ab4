"""The Poisson-likelihood fit on the GPU (``fit_spots_poisson``) against the oracle's: every
spot's convergence class, and on the statistically determined spots the centre to 1e-3 px,
widths and amplitudes to 1e-4 relative; noise-free spots recovered to FP32 precision; the
amplitudes at every fitted point solve the score equations of the likelihood."""
import numpy as np
import pytest
import torch

from paper_2106_02045_gb300 import fitspots, synth
from tests.parity import determined

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
CONV = (1, 2, 3, 4)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _run(b):
    g = b.to(DEV)
    out = fitspots.fit_poisson(g.images, g.offsets, g.dims, g.init, g.model)
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("name,n", [("iso15", 3000), ("ell32", 1500), ("mixed", 3000)])
def test_poisson_matches_oracle(name, n):
    import oracle
    b = synth.make_workload(name, n)
    d = b.numpy()
    img = synth.as_numpy_images(b)
    ref = oracle.fit_spots_poisson(img, d["offsets"], d["dims"], d["init"], d["model"])
    out = _run(b)
    imp = oracle.fit_spots(img, d["offsets"], d["dims"], d["init"], d["model"])
    det = determined(b, imp) & np.isin(ref["state"], CONV)
    agree = np.isin(out["state"], CONV) == np.isin(ref["state"], CONV)
    p, r = out["params"][det], ref["params"][det]
    rel = lambda u, v: np.abs(u - v) / np.maximum(np.abs(v), 1e-30)
    ok = ((np.abs(p[:, :2] - r[:, :2]) <= 1e-3).all(1) & (rel(p[:, 2:], r[:, 2:]) <= 1e-4).all(1)
          & (rel(out["alpha"][det], ref["alpha"][det]) <= 1e-4)
          & (rel(out["beta"][det], ref["beta"][det]) <= 1e-4))
    dev = rel(out["chi2"][det], ref["chi2"][det])
    print(f"{name}: class agreement {agree.mean():.4f} ({agree[det].mean():.4f} determined), "
          f"bar {ok.mean():.4f} of {det.sum()}, deviance rel. diff. median {np.median(dev):.2e}")
    assert det.sum() >= n // 5
    # the class disagreements outside the determined set are fits that wander to the limit()
    # box or to negative amplitudes, where FP32 and FP64 paths part (2.4 % of ell32 measured)
    assert agree.mean() >= 0.97 and agree[det].mean() >= 0.999
    assert ok.mean() >= 0.999
    assert np.median(dev) < 1e-4


def test_poisson_noise_free_and_score_equations():
    """Noise-free spots of every ROI shape class: the fit returns the generating parameters
    to FP32 precision. The returned amplitudes solve the score equations (FP64 check on the
    host at the returned shape parameters)."""
    import oracle
    rng = np.random.default_rng(77)
    spots, dims, init, truth, model = [], [], [], [], []
    for _ in range(400):
        W, H = int(rng.integers(5, 33)), int(rng.integers(5, 33))
        m = int(rng.integers(0, 2))
        cap = min(W, H) / 4
        p = np.array([(W - 1) / 2 + rng.uniform(-1, 1), (H - 1) / 2 + rng.uniform(-1, 1),
                      rng.uniform(0.9, max(1.0, min(2.5, cap))),
                      rng.uniform(0.9, max(1.0, min(2.5, cap)))])
        if m == 0:
            p[3] = p[2]
        amp, bg = rng.uniform(200, 5000), rng.uniform(5, 300)
        x, y = np.arange(W)[None, :], np.arange(H)[:, None]
        f = np.exp(-0.5 * ((x - p[0]) / p[2]) ** 2 - 0.5 * ((y - p[1]) / p[3]) ** 2)
        spots.append((amp * f + bg).astype(np.float32).ravel())
        dims.append((W, H))
        q = p + np.array([rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5), 0, 0])
        q[2] *= rng.uniform(0.85, 1.2)
        q[3] = q[2] if m == 0 else q[3] * rng.uniform(0.85, 1.2)
        init.append(q)
        truth.append((p, amp, bg))
        model.append(m)
    offs = np.cumsum([0] + [s.size for s in spots[:-1]]).astype(np.int64)
    img = np.concatenate(spots)
    t = lambda a, dt: torch.as_tensor(np.asarray(a), dtype=dt, device=DEV)
    out = fitspots.fit_poisson(t(img, torch.float32), t(offs, torch.int64),
                               t(dims, torch.int32), t(init, torch.float32), t(model, torch.uint8),
                               max_iter=60, min_delta=0.0, min_step=1e-6)
    out = {k: v.cpu().numpy() for k, v in out.items()}
    for s, (p, amp, bg) in enumerate(truth):
        assert np.isin(out["state"][s], CONV), (s, out["state"][s])
        assert np.max(np.abs(out["params"][s] - p)) < 2e-3, (s, out["params"][s], p)
        assert abs(out["alpha"][s] - amp) < 2e-3 * amp and abs(out["beta"][s] - bg) < 2e-3 * amp
        W, H = dims[s]
        g = img[offs[s]:offs[s] + W * H].astype(np.float64)
        pp = out["params"][s].astype(np.float64)
        x, y = np.arange(W)[None, :], np.arange(H)[:, None]
        f = np.exp(-0.5 * ((x - pp[0]) / pp[2]) ** 2 - 0.5 * ((y - pp[1]) / pp[3]) ** 2).ravel()
        a, b = oracle.poisson_amplitudes(f, g)
        assert abs(out["alpha"][s] - a) < 2e-5 * a and abs(out["beta"][s] - b) < 2e-5 * a
