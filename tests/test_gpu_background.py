"""Local background pre-subtraction on the GPU (``fit_spots_subtract_background``) against
the oracle's: plane coefficients and subtracted pixels on uint16 and float32 ROIs of every
shape class, invalid ROIs, in-place use, a sample of the full 1,000,000-spot tilted batch,
and the fit of the subtracted spots against the oracle's fit of its own subtraction."""
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


def _coords(W, H):
    x, y = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
    return (x - (W - 1) / 2).ravel(), (y - (H - 1) / 2).ravel()


def _check(img, offs, dims, out, plane, ref_out, ref_plane, exact_sums):
    """Coefficients: uint16 sums are exact, then converted to FP32 and divided (4 ulp);
    float32 sums carry FP32 lane rounding, bounded by 1e-6 of the ring's |dx g| sum over
    sum dx^2. Pixels: the FP32 subtraction, 4 ulp of |g| + |tilt term| plus the slope error
    times the distance from the centre."""
    worst = 0.0
    for k in range(len(offs)):
        W, H = dims[k]
        g = img[offs[k]:offs[k] + W * H].astype(np.float64)
        xc, yc = _coords(W, H)
        rp = ref_plane[k]
        if exact_sums:
            tol_c = 4.8e-7 * np.abs(rp) + 1e-30
        else:
            tol_c = 1e-6 * np.abs(g).max() * np.array([1.0, 2.0 / W, 2.0 / H]) + 1e-30
        assert np.all(np.abs(plane[k] - rp) <= tol_c), (k, plane[k], rp)
        tilt = np.abs(rp[1] * xc) + np.abs(rp[2] * yc)
        tol_p = (4.8e-7 * (np.abs(g) + tilt) + np.abs(plane[k][1] - rp[1]) * np.abs(xc)
                 + np.abs(plane[k][2] - rp[2]) * np.abs(yc) + 1e-6)
        got = out[offs[k]:offs[k] + W * H]
        ref = ref_out[offs[k]:offs[k] + W * H]
        d = np.abs(got - ref)
        assert np.all(d <= tol_p), (k, d.max())
        worst = max(worst, float((d / tol_p).max()))
    return worst


@pytest.mark.parametrize("name,n,border", [("tilted", 3000, 1), ("tilted", 1000, 3),
                                           ("mixed", 3000, 1), ("ell32", 1000, 2),
                                           ("elongated", 2000, 1)])
def test_background_matches_oracle(name, n, border):
    import oracle
    b = synth.make_workload(name, n)
    d = b.numpy()
    img = synth.as_numpy_images(b)
    ref_out, ref_plane = oracle.subtract_background(img, d["offsets"], d["dims"], border=border)
    g = b.to(DEV)
    out, plane = fitspots.subtract_background(g.images, g.offsets, g.dims, border=border)
    worst = _check(img, d["offsets"], d["dims"], out.cpu().numpy(), plane.cpu().numpy(),
                   ref_out, ref_plane, exact_sums=img.dtype == np.uint16)
    print(f"{name} border {border}: worst pixel difference / tolerance {worst:.3f}")


def test_invalid_rois_and_in_place():
    """Invalid ROIs get NaN coefficients and leave their pixels alone; float32 images can
    be processed in place."""
    import oracle
    b = synth.make_workload("mixed", 200)
    d = b.numpy()
    img = synth.as_numpy_images(b).copy()
    dims = d["dims"].copy()
    offs = d["offsets"].copy()
    dims[3] = (2, 9)
    dims[7] = (400, 3)                       # 1200 pixels
    offs[11] = img.size - 5                  # past the end of the buffer
    ref_out, ref_plane = oracle.subtract_background(img, offs, dims)
    t = lambda a, dt: torch.as_tensor(a, dtype=dt, device=DEV)
    images = t(img, torch.float32)
    sentinel = torch.full_like(images, -12345.0)
    out, plane = fitspots.subtract_background(images, t(offs, torch.int64), t(dims, torch.int32),
                                              out=sentinel)
    out, plane = out.cpu().numpy(), plane.cpu().numpy()
    bad = [3, 7, 11]
    assert np.isnan(plane[bad]).all() and np.isnan(ref_plane[bad]).all()
    good = np.setdiff1d(np.arange(200), bad)
    assert np.isfinite(plane[good]).all()
    W, H = d["dims"][3]
    assert (out[d["offsets"][3]:d["offsets"][3] + 2 * 9] == -12345.0).all()
    _check(img, offs[good], dims[good], out, plane[good], ref_out, ref_plane[good], False)
    # in place
    fitspots.subtract_background(images, t(offs, torch.int64), t(dims, torch.int32), out=images)
    inplace = images.cpu().numpy()
    for k in good:
        W, H = dims[k]
        sl = slice(offs[k], offs[k] + W * H)
        assert np.array_equal(inplace[sl], out[sl])


def test_full_size_tilted_sampled():
    """The full tilted batch (1,000,000 spots of 21 x 21 uint16) in one launch; 2,000
    sampled ROIs checked against the oracle one by one."""
    import oracle
    b = synth.make_workload("tilted", device=DEV)
    out, plane = fitspots.subtract_background(b.images, b.offsets, b.dims)
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    idx = np.sort(rng.choice(b.n, 2000, replace=False))
    sub = b.subset(torch.as_tensor(idx, device=DEV))
    simg = synth.as_numpy_images(sub)
    sd = sub.numpy()
    ref_out, ref_plane = oracle.subtract_background(simg, sd["offsets"], sd["dims"])
    N = 21 * 21
    src = torch.as_tensor(idx, device=DEV)[:, None] * N + torch.arange(N, device=DEV)[None, :]
    got = out[src.reshape(-1)].cpu().numpy()
    got_full = np.zeros(simg.size, np.float32)
    for j in range(idx.size):
        got_full[sd["offsets"][j]:sd["offsets"][j] + N] = got[j * N:(j + 1) * N]
    _check(simg, sd["offsets"], sd["dims"], got_full, plane[torch.as_tensor(idx, device=DEV)]
           .cpu().numpy(), ref_out, ref_plane, exact_sums=True)


def test_fit_after_subtraction_matches_oracle():
    """GPU subtraction then GPU fit, against the oracle's subtraction then the oracle's fit:
    the convergence class of every spot, and the accuracy bar on the determined spots."""
    import oracle
    b = synth.make_workload("tilted", 3000)
    d = b.numpy()
    img = synth.as_numpy_images(b)
    ref_img, _ = oracle.subtract_background(img, d["offsets"], d["dims"])
    ref = oracle.fit_spots(ref_img, d["offsets"], d["dims"], d["init"], d["model"])
    g = b.to(DEV)
    sub, _ = fitspots.subtract_background(g.images, g.offsets, g.dims)
    out = fitspots.fit(sub, g.offsets, g.dims, g.init, g.model)
    out = {k: v.cpu().numpy() for k, v in out.items()}
    ob = synth.SpotBatch(torch.as_tensor(ref_img.astype(np.float32)), b.offsets, b.dims,
                         b.model, b.init, b.truth, "tilted-subtracted")
    det = determined(ob, ref)
    agree = np.isin(out["state"], CONV) == np.isin(ref["state"], CONV)
    p, r = out["params"][det], ref["params"][det]
    rel = lambda u, v: np.abs(u - v) / np.maximum(np.abs(v), 1e-30)
    ok = ((np.abs(p[:, :2] - r[:, :2]) <= 1e-3).all(1) & (rel(p[:, 2:], r[:, 2:]) <= 1e-4).all(1)
          & (rel(out["alpha"][det], ref["alpha"][det]) <= 1e-4)
          & (rel(out["beta"][det], ref["beta"][det]) <= 1e-4))
    print(f"tilted, subtracted: class agreement {agree.mean():.4f}, bar {ok.mean():.4f} "
          f"of {det.sum()}")
    assert det.sum() >= 2500
    assert agree.mean() >= 0.999 and ok.mean() >= 0.995
