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
