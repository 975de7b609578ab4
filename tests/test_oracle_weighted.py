"""Pins of the oracle's variance-weighted fit: unit weights give the unweighted fit (a
separately written algorithm), noise-free spots are recovered exactly whatever the
weights, and on high-count Poisson spots the weighted fit is the more accurate one."""
import numpy as np

from paper_2106_02045_gb300 import synth


def test_unit_weights_reproduce_the_unweighted_fit(oracle_mod):
    b = synth.make_paper(400, 9, 400.0, 40.0, seed=41)
    d = b.numpy()
    u = oracle_mod.fit_spots(d["images"], d["offsets"], d["dims"], d["init"], d["model"])
    w = oracle_mod.fit_spots_weighted(d["images"], d["offsets"], d["dims"], d["init"],
                                      d["model"], unit_weights=True)
    assert np.array_equal(u["state"], w["state"]) and np.array_equal(u["iters"], w["iters"])
    for k in ("params", "alpha", "beta", "chi2"):
        assert np.allclose(u[k], w[k], rtol=1e-10, atol=1e-10), k


def test_weighted_recovers_noise_free_spots(oracle_mod):
    ys, xs = np.mgrid[0:13, 0:17]
    for m, p in ((0, [8.3, 6.1, 1.9, 1.9]), (1, [7.6, 5.7, 2.4, 1.6])):
        g = 800.0 * np.exp(-0.5 * ((xs - p[0]) / p[2]) ** 2 - 0.5 * ((ys - p[1]) / p[3]) ** 2) + 50.0
        init = np.array([[p[0] + 0.4, p[1] - 0.3, p[2] * 1.2, p[3] * 0.85]], np.float32)
        o = oracle_mod.fit_spots_weighted(g.ravel(), [0], [[17, 13]], init, np.array([m], np.uint8),
                                          max_iter=200, min_delta=0.0, min_step=1e-14)
        assert o["state"][0] in (1, 2, 4)
        assert np.allclose(o["params"][0], p, atol=1e-8)
        assert abs(o["alpha"][0] - 800.0) < 1e-6 and abs(o["beta"][0] - 50.0) < 1e-6


def test_weighting_helps_at_high_counts(oracle_mod):
    """Peak 1000, background 100 (iso15): the weights estimate the Poisson variance well and
    the weighted fit's centre and width errors are smaller; at low counts (9x9, 400:40) the
    data-based weights are biased and it is the other way round (not asserted)."""
    b = synth.make_workload("iso15", 3000)
    d = b.numpy()
    img = synth.as_numpy_images(b)
    tp = b.truth["params"].numpy()
    res = []
    for fit in (oracle_mod.fit_spots, oracle_mod.fit_spots_weighted):
        o = fit(img, d["offsets"], d["dims"], d["init"], d["model"])
        c = np.isin(o["state"], (1, 2, 3, 4))
        ex = np.sqrt(np.mean(((o["params"][c, 0] - tp[c, 0]) / tp[c, 2]) ** 2))
        es = np.sqrt(np.mean(((o["params"][c, 2] - tp[c, 2]) / tp[c, 2]) ** 2))
        res.append((ex, es))
    assert res[1][0] < 0.95 * res[0][0] and res[1][1] < 0.95 * res[0][1], res
