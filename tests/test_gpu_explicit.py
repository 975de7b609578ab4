"""The explicit-amplitude LM on the GPU (``fit_spots_explicit``) against the FP64 oracle's
explicit LM, and the paper's claim: with the same start values, damping schedule and stop
tests, the implicit-amplitude fit needs fewer iterations and stops on its budget less often
(camera-like 32x32 spots). Evaluated points are not compared: the implicit kernel reuses an
accepted trial's sums as the next gradient point, the explicit one evaluates it again."""
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


def _explicit_gpu(b):
    g = b.to(DEV)
    out = fitspots.fit_explicit(g.images, g.offsets, g.dims, g.init, g.model)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("name,n", [("iso15", 2000), ("ell32", 2000), ("mixed", 3000)])
def test_explicit_matches_oracle(name, n):
    import oracle
    b = synth.make_workload(name, n)
    d = b.numpy()
    img = synth.as_numpy_images(b)
    ref = oracle.fit_spots_explicit(img, d["offsets"], d["dims"], d["init"], d["model"])
    out = _explicit_gpu(b)
    # determined spots of the (common) minimum, selected with the implicit oracle fit
    imp = oracle.fit_spots(img, d["offsets"], d["dims"], d["init"], d["model"])
    det = determined(b, imp) & np.isin(ref["state"], CONV)
    agree = np.isin(out["state"], CONV) == np.isin(ref["state"], CONV)
    same_class = agree.mean()
    p, r = out["params"][det], ref["params"][det]
    rel = lambda u, v: np.abs(u - v) / np.maximum(np.abs(v), 1e-30)
    ok = ((np.abs(p[:, :2] - r[:, :2]) <= 1e-3).all(1) & (rel(p[:, 2:], r[:, 2:]) <= 1e-4).all(1)
          & (rel(out["alpha"][det], ref["alpha"][det]) <= 1e-4)
          & (rel(out["beta"][det], ref["beta"][det]) <= 1e-4))
    print(f"{name}: class agreement {same_class:.4f}, bar {ok.mean():.4f} of {det.sum()} "
          f"determined; iterations GPU {out['iters'].mean():.2f} oracle {ref['iters'].mean():.2f}")
    assert det.sum() >= n // 5
    # all spots: the explicit method ends on its iteration budget for ~12 % of the ell32
    # spots, where one iteration more or less flips the class; determined spots: stricter
    assert same_class >= 0.97
    assert agree[det].mean() >= 0.995
    assert ok.mean() >= 0.99


def test_implicit_needs_fewer_iterations_than_explicit():
    b = synth.make_workload("ell32", 20000, device=DEV)
    imp = fitspots.fit_batch(b)
    exp = fitspots.fit_explicit(b.images, b.offsets, b.dims, b.init, b.model)
    torch.cuda.synchronize()
    ci = torch.isin(imp["state"], torch.tensor(CONV, device=DEV))
    ce = torch.isin(exp["state"], torch.tensor(CONV, device=DEV))
    both = ci & ce
    it_i = imp["iters"][both].float().mean().item()
    it_e = exp["iters"][both].float().mean().item()
    ev_i = imp["evals"][both].float().mean().item()
    ev_e = exp["evals"][both].float().mean().item()
    cap_i = (imp["state"] == 0).float().mean().item()
    cap_e = (exp["state"] == 0).float().mean().item()
    print(f"ell32: iterations implicit {it_i:.2f} explicit {it_e:.2f}; evaluations "
          f"{ev_i:.2f} / {ev_e:.2f}; at the iteration budget {cap_i:.3f} / {cap_e:.3f}")
    assert it_e > 1.1 * it_i and cap_e > 1.5 * cap_i
