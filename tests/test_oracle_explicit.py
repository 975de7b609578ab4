"""Pins of the oracle's explicit-amplitude LM: exact recovery of noise-free spots, and the
same minimum as the implicit-amplitude fit (a different algorithm over the same model)."""
import numpy as np

from paper_2106_02045_gb300 import synth


def _spot(model, W, H, p, amp, bg):
    ys, xs = np.mgrid[0:H, 0:W]
    sy = p[2] if model == 0 else p[3]
    f = np.exp(-0.5 * ((xs - p[0]) / p[2]) ** 2 - 0.5 * ((ys - p[1]) / sy) ** 2)
    return (amp * f + bg).ravel()


def test_explicit_recovers_noise_free_spots(oracle_mod):
    cases = [(0, 15, 15, [7.3, 6.8, 1.7, 1.7], 900.0, 120.0),
             (1, 20, 13, [9.6, 6.2, 2.5, 1.4], 400.0, 30.0),
             (1, 32, 32, [15.1, 16.7, 3.1, 2.2], 2500.0, 300.0)]
    for m, W, H, p, amp, bg in cases:
        g = _spot(m, W, H, p, amp, bg)
        init = np.array([[p[0] + 0.6, p[1] - 0.5, p[2] * 1.25, p[3] * 0.8]], np.float32)
        o = oracle_mod.fit_spots_explicit(g, [0], [[W, H]], init, np.array([m], np.uint8),
                                          max_iter=200, min_delta=0.0, min_step=1e-14)
        assert o["state"][0] in (1, 2, 4), o["state"]
        assert np.allclose(o["params"][0][:2], p[:2], atol=1e-9)
        assert np.allclose(o["params"][0][2:], p[2:] if m else [p[2], p[2]], rtol=1e-9)
        assert abs(o["alpha"][0] / amp - 1) < 1e-9 and abs(o["beta"][0] / bg - 1) < 1e-9


def test_explicit_and_implicit_reach_the_same_minimum(oracle_mod):
    b = synth.make_paper(500, 9, 1600.0, 40.0, seed=21)
    d = b.numpy()
    kw = dict(max_iter=100, min_delta=0.0, min_step=1e-12)
    imp = oracle_mod.fit_spots(d["images"], d["offsets"], d["dims"], d["init"], d["model"], **kw)
    exp = oracle_mod.fit_spots_explicit(d["images"], d["offsets"], d["dims"], d["init"],
                                        d["model"], **kw)
    both = np.isin(imp["state"], (1, 2, 3, 4)) & np.isin(exp["state"], (1, 2, 3, 4))
    assert both.mean() > 0.99
    assert np.abs(imp["params"][both] - exp["params"][both]).max() < 1e-6
    assert np.abs(imp["chi2"][both] / exp["chi2"][both] - 1).max() < 1e-10
    assert np.abs(imp["alpha"][both] / exp["alpha"][both] - 1).max() < 1e-6
