"""Pins of the start-value oracle (``oracle/start.py``) to cases the definition fixes by
hand, and a cross-check against the independent PyTorch rules that made the workloads'
start values."""
import math

import numpy as np
import torch

from oracle import start as st
from paper_2106_02045_gb300 import synth


def test_single_bright_pixel():
    W, H = 32, 32
    g = np.full(W * H, 100.0)
    g[12 * W + 10] = 5000.0
    x0, y0, s0, s1 = st.start_one(g, W, H, st.CENTROID)
    assert (x0, y0) == (10.0, 12.0)                     # all the weight sits on one pixel
    assert s0 == s1 == math.sqrt(1 / math.pi)           # M = 1
    # the nine 3x3 neighbourhoods that hold the pixel tie; the lowest index wins
    x0, y0, _, _ = st.start_one(g, W, H, st.PAPER)
    assert (x0, y0) == (9.0, 11.0)


def test_flat_roi():
    W, H = 7, 5
    g = np.full(W * H, 42.0)
    assert np.array_equal(st.start_one(g, W, H, st.CENTROID),
                          [3.0, 2.0, math.sqrt(1 / math.pi), math.sqrt(1 / math.pi)])
    assert tuple(st.start_one(g, W, H, st.PAPER)[:2]) == (0.0, 0.0)


def test_clipped_neighbourhood_means_favour_the_corner():
    """Near a border the clipped 3x3 mean divides by fewer pixels: a bright pixel at (1, 1)
    gives the corner (0, 0) the mean (b + 3 f) / 4 > (8 f + b) / 9 of its own neighbourhood."""
    W = H = 6
    g = np.full(W * H, 10.0)
    g[1 * W + 1] = 910.0
    assert tuple(st.start_one(g, W, H, st.PAPER)[:2]) == (0.0, 0.0)


def test_symmetric_gaussian():
    """A noise-free Gaussian centred on the ROI's axis of symmetry: the centroid is the
    centre, the neighbourhood rule the nearer of the two central pixels, and M counts the
    pixels inside one sigma, ~ pi sigma^2."""
    W, H, sig = 32, 25, 5.0
    ys, xs = np.mgrid[0:H, 0:W]
    g = (1000.0 * np.exp(-0.5 * ((xs - 15.5) ** 2 + (ys - 12.0) ** 2) / sig**2)).astype(np.float32)
    x0, y0, s0, _ = st.start_one(g.ravel(), W, H, st.CENTROID)
    assert abs(x0 - 15.5) < 1e-9 and abs(y0 - 12.0) < 1e-9
    assert abs(s0 - sig) < 0.3
    x0, y0, _, _ = st.start_one(g.ravel(), W, H, st.PAPER)
    assert (x0, y0) == (15.0, 12.0)


def test_invalid_rois_give_nan():
    out = st.start_values(np.zeros(100), [0, 90, 0], [[10, 10], [5, 5], [40, 2]])
    assert np.isfinite(out[0]).all() and np.isnan(out[1]).all() and np.isnan(out[2]).all()


def test_matches_the_workload_generators():
    """synth computes the same rules with PyTorch (FP64 threshold and means): identical
    centres; widths identical wherever the FP32 and FP64 thresholds split the pixels alike."""
    b = synth.make_workload("iso15", 400)
    img = b.images.numpy()
    ref = b.init.numpy()
    out = st.start_values(img, b.offsets.numpy(), b.dims.numpy(), st.CENTROID)
    assert np.allclose(out[:, :2], ref[:, :2], atol=1e-5)
    assert np.mean(np.abs(out[:, 2] - ref[:, 2]) < 1e-5) >= 0.995
    p = synth.make_paper(200, 9, 1000.0, 100.0, seed=11)
    ref = synth.paper_start_values(p.images.reshape(p.n, -1), 9).numpy()
    out = st.start_values(p.images.numpy(), p.offsets.numpy(), p.dims.numpy(), st.PAPER)
    assert np.array_equal(out[:, :2], ref[:, :2])


def _noisy_spot(rng, W, H):
    ys, xs = np.mgrid[0:H, 0:W]
    x, y = rng.uniform(3, W - 4), rng.uniform(3, H - 4)
    s = rng.uniform(1.2, 2.5)
    lam = 1500.0 * np.exp(-0.5 * ((xs - x) ** 2 + (ys - y) ** 2) / s**2) + 60.0
    return rng.poisson(lam).astype(np.float64)


def test_exact_invariances():
    """Properties both rules have by definition, on integer-valued noisy spots (every FP32
    decision exact): embedding the ROI in a larger one filled with its own minimum moves the
    centre by the offset and leaves M alone (for the 3x3 rule when its best neighbourhood is
    away from the border, where the clipped means change); a constant added to every pixel
    leaves everything alone, a positive integer scale leaves the width (and the centroid)
    alone; transposing the ROI swaps the centroid's x0 and y0 and keeps the width."""
    rng = np.random.default_rng(21)
    for _ in range(40):
        W, H = int(rng.integers(9, 21)), int(rng.integers(9, 21))
        g = _noisy_spot(rng, W, H)
        for rule in (st.CENTROID, st.PAPER):
            base = st.start_one(g.ravel(), W, H, rule)
            # the extra pixels take the ROI's minimum: the centroid's weights (measured from
            # the minimum) and M are unchanged; a lower fill would move the minimum
            dx, dy = int(rng.integers(1, 32 - W + 1)), int(rng.integers(1, 32 - H + 1))
            big = np.full((H + dy + 1, W + dx + 1), g.min())
            big[dy:dy + H, dx:dx + W] = g.reshape(H, W)
            emb = st.start_one(big.ravel(), W + dx + 1, H + dy + 1, rule)
            if rule == st.CENTROID:
                assert np.allclose(emb, base + [dx, dy, 0, 0], rtol=0, atol=1e-9)
            else:
                # the clipped border means of the small ROI are not those of the embedded
                # one; the argmax agrees whenever it lies inside, away from the border
                if 1 <= base[0] <= W - 2 and 1 <= base[1] <= H - 2:
                    assert np.array_equal(emb, base + [dx, dy, 0, 0])
            assert np.array_equal(st.start_one(g.ravel() + 250.0, W, H, rule), base)
            assert np.array_equal(st.start_one(3.0 * g.ravel(), W, H, rule)[2:], base[2:])
            if rule == st.CENTROID:
                assert np.allclose(st.start_one(3.0 * g.ravel(), W, H, rule), base, atol=1e-9)
            gt = g.reshape(H, W).T.ravel()
            tr = st.start_one(gt, H, W, rule)
            if rule == st.CENTROID:
                assert np.allclose(tr, base[[1, 0, 2, 3]], atol=1e-9)
            else:
                assert tr[2] == base[2]
