"""Pins of the oracle's local-background pre-subtraction (least-squares plane on each ROI's
border ring, its tilt subtracted): exact recovery of a plane, agreement with a generic
least-squares solver, invariance under added planes, the ring is the only input of the
plane, and the fit after subtraction is unbiased on tilted backgrounds where the plain fit
is not."""
import numpy as np
import pytest

from paper_2106_02045_gb300 import synth


def _ring(W, H, border):
    x, y = np.meshgrid(np.arange(W), np.arange(H))
    return ((x < border) | (x >= W - border) | (y < border) | (y >= H - border)).ravel()


def _coords(W, H):
    x, y = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
    return (x - (W - 1) / 2).ravel(), (y - (H - 1) / 2).ravel()


def _pack(rois):
    offs = np.cumsum([0] + [r.size for r in rois[:-1]]).astype(np.int64)
    return np.concatenate(rois), offs


def test_plane_is_recovered_exactly(oracle_mod):
    rng = np.random.default_rng(3)
    rois, dims, planes, spots = [], [], [], []
    for W, H in ((21, 21), (15, 9), (64, 16), (8, 128), (33, 31), (3, 3)):
        c = rng.uniform(50, 500), rng.uniform(-5, 5), rng.uniform(-5, 5)
        xc, yc = _coords(W, H)
        s = 0.6
        spot = 800 * np.exp(-0.5 * (xc ** 2 + yc ** 2) / s ** 2)
        spot[_ring(W, H, 1)] = 0.0        # nothing of the spot on the ring
        rois.append(c[0] + c[1] * xc + c[2] * yc + spot)
        dims.append((W, H))
        planes.append(c)
        spots.append(spot)
    img, offs = _pack(rois)
    out, plane = oracle_mod.subtract_background(img, offs, dims)
    for k, (W, H) in enumerate(dims):
        assert np.allclose(plane[k], planes[k], rtol=0, atol=1e-9)
        got = out[offs[k]:offs[k] + W * H]
        assert np.allclose(got, spots[k] + planes[k][0], rtol=0, atol=1e-9)


@pytest.mark.parametrize("border", [1, 2, 3])
def test_plane_matches_a_generic_least_squares_solver(oracle_mod, border):
    rng = np.random.default_rng(10 + border)
    rois, dims = [], []
    for _ in range(40):
        W, H = int(rng.integers(3 + 2 * border, 40)), int(rng.integers(3 + 2 * border, 25))
        rois.append(rng.poisson(rng.uniform(20, 2000), W * H).astype(np.float32))
        dims.append((W, H))
    img, offs = _pack(rois)
    out, plane = oracle_mod.subtract_background(img, offs, dims, border=border)
    for k, (W, H) in enumerate(dims):
        m = _ring(W, H, border)
        xc, yc = _coords(W, H)
        A = np.stack([np.ones(W * H), xc, yc], axis=1)
        g = rois[k].astype(np.float64)
        c, *_ = np.linalg.lstsq(A[m], g[m], rcond=None)
        assert np.allclose(plane[k], c, rtol=1e-10, atol=1e-9)
        assert np.allclose(out[offs[k]:offs[k] + W * H], g - c[1] * xc - c[2] * yc,
                           rtol=0, atol=1e-9 * np.abs(g).max())


def test_added_planes_change_only_the_level(oracle_mod):
    """subtract(g + a + b x + c y) = subtract(g) + a, pixel by pixel, and only the ring
    decides the plane."""
    rng = np.random.default_rng(21)
    rois, dims, added = [], [], []
    for _ in range(30):
        W, H = int(rng.integers(5, 33)), int(rng.integers(5, 33))
        rois.append(rng.uniform(0, 1000, W * H))
        dims.append((W, H))
        added.append((rng.uniform(-100, 100), rng.uniform(-3, 3), rng.uniform(-3, 3)))
    img, offs = _pack(rois)
    out0, pl0 = oracle_mod.subtract_background(img, offs, dims, border=2)
    tilted = []
    for k, (W, H) in enumerate(dims):
        xc, yc = _coords(W, H)
        a, b, c = added[k]
        tilted.append(rois[k] + a + b * xc + c * yc)
    img1, _ = _pack(tilted)
    out1, pl1 = oracle_mod.subtract_background(img1, offs, dims, border=2)
    for k, (W, H) in enumerate(dims):
        sl = slice(offs[k], offs[k] + W * H)
        assert np.allclose(out1[sl], out0[sl] + added[k][0], rtol=0, atol=1e-9)
        assert np.allclose(pl1[k] - pl0[k], added[k], rtol=0, atol=1e-9)
    # changing interior pixels leaves the plane alone; changing a ring pixel does not
    W, H = dims[0]
    inner = np.nonzero(~_ring(W, H, 2))[0]
    img2 = img.copy()
    img2[offs[0] + inner] += 5000.0
    _, pl2 = oracle_mod.subtract_background(img2, offs[:1], dims[:1], border=2)
    assert np.array_equal(pl2[0], pl0[0])
    img2[offs[0]] += 5000.0
    _, pl3 = oracle_mod.subtract_background(img2, offs[:1], dims[:1], border=2)
    assert not np.allclose(pl3[0], pl0[0])


def test_invalid_rois_get_nan(oracle_mod):
    img = np.ones(1000, np.float32)
    offs = np.array([0, 0, 0, 990, 0], np.int64)
    dims = np.array([[2, 10], [10, 10], [10, 10], [4, 4], [1025, 1]], np.int32)
    for border, bad in ((1, [0, 3, 4]), (0, [0, 1, 2, 3, 4]), (9, [0, 1, 2, 3, 4])):
        _, pl = oracle_mod.subtract_background(img, offs, dims, border=border)
        assert np.isnan(pl[bad]).all()
        good = [k for k in range(5) if k not in bad]
        assert np.isfinite(pl[good]).all()


def test_fit_after_subtraction_is_unbiased_on_tilted_backgrounds(oracle_mod):
    """tilted workload (21 x 21, slopes up to 6 counts / px): after subtraction the centre
    errors have no measurable bias and no correlation with the slope; fitted directly, the
    spots are pulled along the slope."""
    b = synth.make_workload("tilted", 2000)
    d = b.numpy()
    img = synth.as_numpy_images(b)
    t = b.truth["params"].numpy()
    tilt = b.truth["tilt"].numpy()
    sub, plane = oracle_mod.subtract_background(img, d["offsets"], d["dims"])
    # slope noise: about sqrt(300) counts over sqrt(sum (x - xc)^2) = 73 on the ring, 0.25
    se = plane[:, 1:] - tilt
    assert np.sqrt((se ** 2).mean()) < 0.35 and np.abs(se.mean(0)).max() < 0.03
    assert np.abs((plane[:, 0] - b.truth["beta"].numpy()).mean()) < 1.0
    fit = lambda g: oracle_mod.fit_spots(g, d["offsets"], d["dims"], d["init"], d["model"])
    o_sub, o_raw = fit(sub), fit(img)
    err_sub = o_sub["params"][:, :2] - t[:, :2]
    err_raw = o_raw["params"][:, :2] - t[:, :2]
    corr = lambda e, s: np.corrcoef(e, s)[0, 1]
    assert np.isin(o_sub["state"], (1, 2, 3, 4)).mean() > 0.99
    assert np.abs(err_sub.mean(0)).max() < 0.01
    assert abs(corr(err_sub[:, 0], tilt[:, 0])) < 0.1 and abs(corr(err_sub[:, 1], tilt[:, 1])) < 0.1
    assert corr(err_raw[:, 0], tilt[:, 0]) > 0.5 and corr(err_raw[:, 1], tilt[:, 1]) > 0.5
    assert np.all(np.sqrt((err_sub ** 2).mean(0)) < 0.7 * np.sqrt((err_raw ** 2).mean(0)))
    assert np.abs(o_sub["beta"] - plane[:, 0]).mean() < 3.0
