"""Pins of the FP64 oracle to facts outside itself (no GPU needed).

Each test checks the oracle against something the paper or mathematics fixes: a generic
least-squares solver, finite differences, exact recovery of noise-free spots, a
brute-force grid plus a library optimiser, symmetries, and the accuracy figures the
paper prints in Table 1.
"""
import math
from pathlib import Path

import numpy as np
import pytest

from paper_2106_02045_gb300 import synth

ISO, ELL = 0, 1
GOLDEN = Path(__file__).parent / "golden"


def _spot(model, W, H, p, amp, bg, rng=None, noise=True):
    x = np.arange(W)[None, :]
    y = np.arange(H)[:, None]
    sx, sy = (p[2], p[2]) if model == ISO else (p[2], p[3])
    f = np.exp(-0.5 * ((x - p[0]) / sx) ** 2 - 0.5 * ((y - p[1]) / sy) ** 2).ravel()
    g = amp * f + bg
    if noise:
        g = rng.poisson(g).astype(np.float64)
    return g


# ---------------------------------------------------------------- Eq. 5-6 amplitudes
def test_amplitudes_equal_generic_least_squares(oracle_mod):
    """alpha^, beta^ of Eq. 6 equal a generic least-squares solve of [f, 1] c = g."""
    rng = np.random.default_rng(1)
    for trial in range(50):
        N = int(rng.integers(9, 1025))
        f = rng.uniform(0.0, 1.0, N) ** 3
        g = 500.0 * f + 40.0 + rng.normal(0, 5, N)
        a, b = oracle_mod.amplitudes(f, g)
        c, *_ = np.linalg.lstsq(np.stack([f, np.ones(N)], 1), g, rcond=None)
        assert abs(a - c[0]) <= 1e-11 * abs(c[0])
        assert abs(b - c[1]) <= 1e-11 * max(abs(c[1]), 1.0)
        r = g - (a * f + b)                      # Eq. 4: the residual is orthogonal to f and 1
        assert abs(r.sum()) <= 1e-12 * np.abs(g).sum()
        assert abs((r * f).sum()) <= 1e-12 * np.abs(g).sum()


def test_amplitudes_undefined_for_constant_profile(oracle_mod):
    """N F(bold) - F^2 vanishes only for a constant profile (text after Eq. 6)."""
    assert oracle_mod.amplitudes(np.full(25, 0.5), np.arange(25.0)) is None
    f = np.linspace(0.1, 1.0, 25)
    assert oracle_mod.amplitudes(f, np.arange(25.0)) is not None


# ---------------------------------------------------------------- Eq. 10-11 profile
@pytest.mark.parametrize("model", [ISO, ELL])
def test_profile_derivatives_match_finite_differences(oracle_mod, model):
    rng = np.random.default_rng(2)
    for _ in range(10):
        W, H = int(rng.integers(5, 33)), int(rng.integers(5, 33))
        p = np.array([rng.uniform(1, W - 2), rng.uniform(1, H - 2), rng.uniform(0.8, 4),
                      rng.uniform(0.8, 4)])
        if model == ISO:
            p[3] = p[2]
        f, d = oracle_mod.profile(model, W, H, p, with_derivs=True)
        assert np.all(f > 0) and abs(f.max() - 1.0) < 0.5
        P = 3 if model == ISO else 4
        for j in range(P):
            h = 1e-6 * max(1.0, abs(p[j]))
            pp, pm = p.copy(), p.copy()
            pp[j] += h
            pm[j] -= h
            if model == ISO and j == 2:
                pp[3], pm[3] = pp[2], pm[2]
            fd = (oracle_mod.profile(model, W, H, pp) - oracle_mod.profile(model, W, H, pm)) / (2 * h)
            assert np.max(np.abs(fd - d[j])) <= 1e-7 * np.max(np.abs(d[j]))


# ---------------------------------------------------------------- Eq. 7-9 Jacobian
def _h(oracle_mod, model, W, H, g, p):
    f = oracle_mod.profile(model, W, H, p)
    a, b = oracle_mod.amplitudes(f, g)
    return a * f + b


def _chi2(oracle_mod, model, W, H, g, p):
    return float(((g - _h(oracle_mod, model, W, H, g, p)) ** 2).sum())


def _set(p, j, v, model):
    q = p.copy()
    q[j] = v
    if model == ISO and j == 2:
        q[3] = v
    return q


@pytest.mark.parametrize("model", [ISO, ELL])
def test_jacobian_matches_finite_differences(oracle_mod, model):
    """J_ij = dh_i/dp_j including the implicit amplitude derivatives of Eq. 8."""
    rng = np.random.default_rng(3)
    for _ in range(8):
        W, H = int(rng.integers(5, 33)), int(rng.integers(5, 33))
        p = np.array([(W - 1) / 2 + rng.uniform(-1, 1), (H - 1) / 2 + rng.uniform(-1, 1),
                      rng.uniform(1, 2.5), rng.uniform(1, 2.5)])
        if model == ISO:
            p[3] = p[2]
        g = _spot(model, W, H, p + rng.normal(0, 0.3, 4), 800, 60, rng)
        J, a, b, da, db = oracle_mod.jacobian(model, W, H, g, p)
        for j in range(J.shape[0]):
            h = 1e-6 * max(1.0, abs(p[j]))
            fd = (_h(oracle_mod, model, W, H, g, _set(p, j, p[j] + h, model)) -
                  _h(oracle_mod, model, W, H, g, _set(p, j, p[j] - h, model))) / (2 * h)
            assert np.max(np.abs(fd - J[j])) <= 2e-7 * np.max(np.abs(J[j]))
            # Eq. 8 alone: the amplitude derivatives
            fp = oracle_mod.profile(model, W, H, _set(p, j, p[j] + h, model))
            fm = oracle_mod.profile(model, W, H, _set(p, j, p[j] - h, model))
            ap, bp = oracle_mod.amplitudes(fp, g)
            am, bm = oracle_mod.amplitudes(fm, g)
            assert abs((ap - am) / (2 * h) - da[j]) <= 1e-6 * (abs(da[j]) + 1e-3 * abs(a))
            assert abs((bp - bm) / (2 * h) - db[j]) <= 1e-6 * (abs(db[j]) + 1e-3 * abs(a))


@pytest.mark.parametrize("model", [ISO, ELL])
def test_gradient_is_minus_half_chi2_slope(oracle_mod, model):
    """b = J^T (g - h) = -1/2 d chi^2 / dp (Eq. 9 with the sign reading of Eq. 12)."""
    rng = np.random.default_rng(4)
    for _ in range(8):
        W, H = int(rng.integers(6, 25)), int(rng.integers(6, 25))
        p = np.array([(W - 1) / 2 + rng.uniform(-1, 1), (H - 1) / 2 + rng.uniform(-1, 1),
                      rng.uniform(1, 2.5), rng.uniform(1, 2.5)])
        if model == ISO:
            p[3] = p[2]
        g = _spot(model, W, H, p, 900, 50, rng)
        q = p + np.array([0.4, -0.3, 0.2, -0.15])
        if model == ISO:
            q[3] = q[2]
        ev = oracle_mod.evaluate(model, W, H, g, q)
        for j in range(len(ev["b"])):
            h = 1e-5 * max(1.0, abs(q[j]))
            slope = (_chi2(oracle_mod, model, W, H, g, _set(q, j, q[j] + h, model)) -
                     _chi2(oracle_mod, model, W, H, g, _set(q, j, q[j] - h, model))) / (2 * h)
            assert abs(-0.5 * slope - ev["b"][j]) <= 1e-6 * np.max(np.abs(ev["b"])) + 1e-9


@pytest.mark.parametrize("model", [ISO, ELL])
def test_normal_matrix_is_half_hessian_at_zero_residual(oracle_mod, model):
    """With g = h(p) exactly, 1/2 d^2 chi^2/dp^2 = J^T J (Gauss-Newton is exact there)."""
    rng = np.random.default_rng(5)
    W, H = 13, 11
    p = np.array([6.2, 4.7, 1.7, 1.3])
    if model == ISO:
        p[3] = p[2]
    g = _spot(model, W, H, p, 700, 80, noise=False)
    A = oracle_mod.evaluate(model, W, H, g, p)["A"]
    P = A.shape[0]
    hs = 1e-4
    for j in range(P):
        for k in range(P):
            def c(dj, dk):
                q = _set(p, j, p[j] + dj, model)
                q = _set(q, k, q[k] + dk, model)
                return _chi2(oracle_mod, model, W, H, g, q)
            hess = (c(hs, hs) - c(hs, -hs) - c(-hs, hs) + c(-hs, -hs)) / (4 * hs * hs)
            assert abs(0.5 * hess - A[j, k]) <= 1e-5 * np.max(np.abs(A))
    del rng


def test_damped_solve_matches_numpy(oracle_mod):
    """Eq. 14 on random SPD systems."""
    rng = np.random.default_rng(6)
    for P in (3, 4):
        for lam in (0.0, 1e-3, 0.01, 1.0, 1e3):
            X = rng.normal(size=(20, P)) * rng.uniform(0.1, 10, P)
            A = X.T @ X
            b = rng.normal(size=P)
            d = oracle_mod.solve_damped(A, b, lam)
            ref = np.linalg.solve(A + lam * np.diag(np.diag(A)), b)
            assert np.allclose(d, ref, rtol=1e-10, atol=1e-14)
    assert oracle_mod.solve_damped(np.zeros((3, 3)), np.ones(3), 0.01) is None


# ---------------------------------------------------------------- the whole LM
def _pack(spots, dims, dtype=np.float64):
    offs = np.cumsum([0] + [len(s) for s in spots[:-1]])
    return np.concatenate(spots).astype(dtype), offs, np.array(dims, np.int32)


@pytest.mark.parametrize("model", [ISO, ELL])
def test_exact_recovery_of_noise_free_spots(oracle_mod, model):
    """Noise-free spots are recovered to better than 1e-9 (px, relative in amplitudes)."""
    rng = np.random.default_rng(7)
    spots, dims, init, truth = [], [], [], []
    for _ in range(60):
        W, H = int(rng.integers(5, 33)), int(rng.integers(5, 33))
        cap = min(W, H) / 4
        p = np.array([(W - 1) / 2 + rng.uniform(-1, 1), (H - 1) / 2 + rng.uniform(-1, 1),
                      rng.uniform(0.8, max(0.9, min(2.5, cap))),
                      rng.uniform(0.8, max(0.9, min(2.5, cap)))])
        if model == ISO:
            p[3] = p[2]
        amp, bg = rng.uniform(100, 5000), rng.uniform(0, 500)
        spots.append(_spot(model, W, H, p, amp, bg, noise=False))
        dims.append((W, H))
        q = p + np.array([rng.uniform(-1, 1), rng.uniform(-1, 1), 0, 0])
        q[2] *= rng.uniform(0.75, 1.3)
        q[3] = q[2] if model == ISO else q[3] * rng.uniform(0.75, 1.3)
        init.append(q)
        truth.append((p, amp, bg))
    img, offs, dims = _pack(spots, dims)
    o = oracle_mod.fit_spots(img, offs, dims, np.array(init, np.float32),
                             np.full(len(spots), model, np.uint8), max_iter=100,
                             min_delta=0.0, min_step=1e-12)
    for s, (p, amp, bg) in enumerate(truth):
        assert np.max(np.abs(o["params"][s] - p)) < 1e-9, (s, o["state"][s], o["params"][s], p)
        assert abs(o["alpha"][s] - amp) < 1e-9 * amp
        assert abs(o["beta"][s] - bg) < 1e-9 * max(amp, 1.0)


@pytest.mark.parametrize("model", [ISO, ELL])
def test_exact_recovery_of_elongated_spots(oracle_mod, model):
    """ROIs with a side above 32 (up to 1024 pixels, the paper's bound on one fit): noise-free
    spots are recovered to better than 1e-9, in both orientations."""
    rng = np.random.default_rng(17 + model)
    shapes = [(64, 16), (16, 64), (128, 8), (8, 128), (341, 3), (3, 341), (40, 25), (100, 10)]
    spots, dims, init, truth = [], [], [], []
    for W, H in shapes * 2:
        cap = min(W, H) / 4
        p = np.array([(W - 1) / 2 + rng.uniform(-1, 1), (H - 1) / 2 + rng.uniform(-1, 1),
                      rng.uniform(0.6, max(0.7, min(2.5, cap))),
                      rng.uniform(0.6, max(0.7, min(2.5, cap)))])
        if model == ISO:
            p[3] = p[2]
        amp, bg = rng.uniform(500, 5000), rng.uniform(0, 500)
        spots.append(_spot(model, W, H, p, amp, bg, noise=False))
        dims.append((W, H))
        q = p + np.array([rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5), 0, 0])
        q[2] *= rng.uniform(0.85, 1.15)
        q[3] = q[2] if model == ISO else q[3] * rng.uniform(0.85, 1.15)
        init.append(q)
        truth.append((p, amp, bg))
    img, offs, dims = _pack(spots, dims)
    o = oracle_mod.fit_spots(img, offs, dims, np.array(init, np.float32),
                             np.full(len(spots), model, np.uint8), max_iter=100,
                             min_delta=0.0, min_step=1e-12)
    for s, (p, amp, bg) in enumerate(truth):
        assert np.max(np.abs(o["params"][s] - p)) < 1e-9, (s, o["state"][s], o["params"][s], p)
        assert abs(o["alpha"][s] - amp) < 1e-9 * amp
        assert abs(o["beta"][s] - bg) < 1e-9 * max(amp, 1.0)


def test_transpose_symmetry_on_elongated_spots(oracle_mod):
    """A wide ROI and its transpose (64x16 / 16x64, 128x8 / 8x128) give the same fit with x and
    y swapped: the elongated ROIs keep the exact symmetry of the method."""
    rng = np.random.default_rng(23)
    for W, H in ((64, 16), (128, 8), (200, 5)):
        p = np.array([(W - 1) / 2 + 0.7, (H - 1) / 2 - 0.4, 1.8, 1.3])
        g = _spot(ELL, W, H, p, 900, 80, rng).reshape(H, W)
        s0 = np.array([p[0] + 0.3, p[1] - 0.2, 1.5, 1.5], np.float32)
        img, offs, dd = _pack([g.ravel(), g.T.copy().ravel()], [(W, H), (H, W)])
        init = np.array([s0, s0[[1, 0, 3, 2]]], np.float32)
        o = oracle_mod.fit_spots(img, offs, dd, init, np.full(2, ELL, np.uint8), max_iter=300,
                                 min_delta=0.0, min_step=1e-10)
        q = o["params"]
        assert np.isin(o["state"], (1, 2, 3, 4)).all()
        assert np.allclose(q[1], q[0][[1, 0, 3, 2]], atol=1e-7)
        assert abs(o["alpha"][1] - o["alpha"][0]) < 1e-7 * o["alpha"][0]


def test_accepted_steps_never_increase_chi2(oracle_mod):
    b = synth.make_workload("ell32", 400)
    d = b.numpy()
    o = oracle_mod.fit_spots(d["images"], d["offsets"], d["dims"], d["init"], d["model"],
                             trace=True)
    tr = o["trace"]
    for s in range(tr.shape[0]):
        t = tr[s][~np.isnan(tr[s])]
        assert np.all(np.diff(t) <= 0.0), (s, t)


def _explicit_fit(model, W, H, g, p0, amp0, bg0):
    """scipy's trust-region least squares on the explicit model (p, alpha, beta)."""
    from scipy.optimize import least_squares
    x = np.arange(W)[None, :]
    y = np.arange(H)[:, None]

    def res(v):
        if model == ISO:
            x0, y0, s, a, b = v
            sx = sy = s
        else:
            x0, y0, sx, sy, a, b = v
        f = np.exp(-0.5 * ((x - x0) / sx) ** 2 - 0.5 * ((y - y0) / sy) ** 2).ravel()
        return a * f + b - g

    v0 = list(p0[:3] if model == ISO else p0[:4]) + [amp0, bg0]
    sol = least_squares(res, v0, method="lm", xtol=1e-15, ftol=1e-15, gtol=1e-15, max_nfev=20000)
    return sol.x, float((sol.fun ** 2).sum())


@pytest.mark.parametrize("model", [ISO, ELL])
def test_converged_fit_is_the_least_squares_minimum(oracle_mod, model):
    """The LM fixed point equals the explicit 5/6-parameter minimum found by scipy."""
    rng = np.random.default_rng(8)
    spots, dims, init, cases = [], [], [], []
    for _ in range(24):
        W, H = int(rng.integers(7, 33)), int(rng.integers(7, 33))
        p = np.array([(W - 1) / 2 + rng.uniform(-1, 1), (H - 1) / 2 + rng.uniform(-1, 1),
                      rng.uniform(1.0, 2.0), rng.uniform(1.0, 2.0)])
        if model == ISO:
            p[3] = p[2]
        g = _spot(model, W, H, p, 1500, 100, rng)
        spots.append(g)
        dims.append((W, H))
        init.append(p + np.array([0.3, -0.2, 0.1, 0.1]) * (1 if model == ELL else [1, 1, 1, 1]))
        cases.append((W, H, g, p))
    init = np.array(init)
    if model == ISO:
        init[:, 3] = init[:, 2]
    img, offs, dims = _pack(spots, dims)
    o = oracle_mod.fit_spots(img, offs, dims, init.astype(np.float32),
                             np.full(len(spots), model, np.uint8), max_iter=200,
                             min_delta=0.0, min_step=1e-13)
    P = 3 if model == ISO else 4
    for s, (W, H, g, p) in enumerate(cases):
        xs, chi_s = _explicit_fit(model, W, H, g, o["params"][s] + 0.05, o["alpha"][s] * 0.9,
                                  o["beta"][s] + 3)
        assert np.max(np.abs(xs[:P] - o["params"][s][:P])) < 1e-6
        assert abs(xs[P] - o["alpha"][s]) < 1e-6 * abs(xs[P])
        chi_o = o["chi2"][s] * (W * H - P - 2)
        assert chi_o <= chi_s * (1 + 1e-10)


def _grid_chi2_min(W, H, g, xs, ys, ss):
    """Brute force: min over the grid of the projection residual ||(I - QQ^T) g||^2."""
    x = np.arange(W)[None, None, :]
    y = np.arange(H)[None, :, None]
    best = (np.inf, None)
    for s in ss:
        X0, Y0 = np.meshgrid(xs, ys, indexing="ij")
        X0, Y0 = X0.ravel(), Y0.ravel()
        f = np.exp(-0.5 * ((x - X0[:, None, None]) ** 2 + (y - Y0[:, None, None]) ** 2) / s ** 2)
        Phi = np.stack([f.reshape(len(X0), -1), np.ones((len(X0), W * H))], axis=2)
        Q, _ = np.linalg.qr(Phi)
        proj = np.einsum("kni,n->ki", Q, g)
        chi = g @ g - (proj ** 2).sum(1)
        k = int(np.argmin(chi))
        if chi[k] < best[0]:
            best = (chi[k], (X0[k], Y0[k], s))
    return best


@pytest.mark.parametrize("S", [5, 7])
def test_tiny_roi_fit_is_the_global_minimum(oracle_mod, S):
    """5x5 / 7x7 noisy spots: the LM result beats a brute-force grid and equals the
    library optimiser started from the grid's best point."""
    rng = np.random.default_rng(9 + S)
    c = (S - 1) / 2
    spots, init, cases = [], [], []
    for _ in range(6):
        p = np.array([c + rng.uniform(-0.7, 0.7), c + rng.uniform(-0.7, 0.7),
                      rng.uniform(0.9, 1.3), 0.0])
        p[3] = p[2]
        g = _spot(ISO, S, S, p, 2000, 50, rng)
        spots.append(g)
        init.append([c, c, 1.2, 1.2])
        cases.append(g)
    img, offs, dims = _pack(spots, [(S, S)] * len(spots))
    o = oracle_mod.fit_spots(img, offs, dims, np.array(init, np.float32),
                             np.zeros(len(spots), np.uint8), max_iter=200, min_delta=0.0,
                             min_step=1e-13)
    for s, g in enumerate(cases):
        gx = np.arange(c - 1.5, c + 1.5001, 0.05)
        chi_grid, (x0, y0, s0) = _grid_chi2_min(S, S, g, gx, gx, np.arange(0.6, 2.0001, 0.05))
        chi_lm = o["chi2"][s] * (S * S - 5)
        assert chi_lm <= chi_grid * (1 + 1e-12)
        xs, chi_s = _explicit_fit(ISO, S, S, g, np.array([x0, y0, s0, s0]), g.max() - g.min(),
                                  g.min())
        assert np.max(np.abs(xs[:3] - o["params"][s][:3])) < 1e-6
        assert abs(chi_lm - chi_s) <= 1e-9 * chi_s


def test_symmetries(oracle_mod):
    """Transpose, mirror, constant offset and scale act on the fit as they must."""
    rng = np.random.default_rng(10)
    W, H = 19, 13
    p = np.array([9.3, 5.8, 1.9, 1.4])
    g = _spot(ELL, W, H, p, 1200, 90, rng).reshape(H, W)
    variants = [g, g.T.copy(), g[:, ::-1].copy(), g + 37.0, g * 2.5]
    dims = [(W, H), (H, W), (W, H), (W, H), (W, H)]
    init = np.array([[9, 6, 1.6, 1.6], [6, 9, 1.6, 1.6], [W - 1 - 9, 6, 1.6, 1.6],
                     [9, 6, 1.6, 1.6], [9, 6, 1.6, 1.6]], np.float32)
    img, offs, dd = _pack([v.ravel() for v in variants], dims)
    o = oracle_mod.fit_spots(img, offs, dd, init, np.full(5, ELL, np.uint8), max_iter=200,
                             min_delta=0.0, min_step=1e-13)
    q, a, b, c = o["params"], o["alpha"], o["beta"], o["chi2"]
    tol = 1e-8
    assert np.allclose(q[1], [q[0][1], q[0][0], q[0][3], q[0][2]], atol=tol)
    assert np.allclose(q[2], [W - 1 - q[0][0], q[0][1], q[0][2], q[0][3]], atol=tol)
    assert np.allclose(q[3], q[0], atol=tol) and abs(b[3] - b[0] - 37.0) < tol
    assert abs(a[3] - a[0]) < tol * a[0] and abs(c[3] - c[0]) < 1e-7 * c[0]
    assert np.allclose(q[4], q[0], atol=tol)
    assert abs(a[4] - 2.5 * a[0]) < tol * a[4] and abs(b[4] - 2.5 * b[0]) < tol * a[4]
    assert abs(c[4] - 6.25 * c[0]) < 1e-7 * c[4]


@pytest.mark.parametrize("model", [ISO, ELL])
def test_symmetries_on_random_spots(oracle_mod, model):
    """The same symmetries (transpose, both mirrors, offset, scale) on random sizes and
    spots of both models, each variant fitted from the correspondingly moved start."""
    rng = np.random.default_rng(60 + model)
    for _ in range(8):
        W, H = int(rng.integers(7, 33)), int(rng.integers(7, 33))
        p = np.array([(W - 1) / 2 + rng.uniform(-1.5, 1.5), (H - 1) / 2 + rng.uniform(-1.5, 1.5),
                      rng.uniform(1.2, 2.4), rng.uniform(1.2, 2.4)])
        if model == ISO:
            p[3] = p[2]
        g = _spot(model, W, H, p, 1500, 70, rng).reshape(H, W)
        s0 = np.array([p[0] + 0.3, p[1] - 0.2, p[2] * 1.1, p[3] * 0.9])
        if model == ISO:
            s0[3] = s0[2]
        off = float(rng.integers(5, 200))
        variants = [(g, (W, H), s0),
                    (g.T.copy(), (H, W), s0[[1, 0, 3, 2]]),
                    (g[:, ::-1].copy(), (W, H), [W - 1 - s0[0], s0[1], s0[2], s0[3]]),
                    (g[::-1, :].copy(), (W, H), [s0[0], H - 1 - s0[1], s0[2], s0[3]]),
                    (g + off, (W, H), s0), (g * 3.0, (W, H), s0)]
        img, offs, dd = _pack([v[0].ravel() for v in variants], [v[1] for v in variants])
        init = np.array([v[2] for v in variants], np.float32)
        # min_step 1e-10: tight enough for the 1e-7 comparisons, loose enough that every fit
        # ends on the step test rather than climbing to the damping cap at the FP64 floor
        o = oracle_mod.fit_spots(img, offs, dd, init, np.full(6, model, np.uint8),
                                 max_iter=300, min_delta=0.0, min_step=1e-10)
        q, a, b = o["params"], o["alpha"], o["beta"]
        assert np.isin(o["state"], (1, 2, 3, 4)).all()
        tol = 1e-7
        assert np.allclose(q[1], q[0][[1, 0, 3, 2]], atol=tol)
        assert np.allclose(q[2], [W - 1 - q[0][0], q[0][1], q[0][2], q[0][3]], atol=tol)
        assert np.allclose(q[3], [q[0][0], H - 1 - q[0][1], q[0][2], q[0][3]], atol=tol)
        assert np.allclose(q[4], q[0], atol=tol) and abs(b[4] - b[0] - off) < 1e-6
        assert np.allclose(q[5], q[0], atol=tol)
        assert abs(a[5] - 3 * a[0]) < 1e-7 * a[5] and abs(a[4] - a[0]) < 1e-7 * a[0]


def test_invalid_spots_are_flagged(oracle_mod):
    img = np.ones(4096, np.float32)
    offs = np.array([0, 100, 200, 300, 4000], np.int64)
    # too narrow, 1089 pixels (above 1024), too flat, unknown model, past the end
    dims = np.array([[2, 10], [33, 33], [3, 2], [5, 5], [10, 10]], np.int32)
    model = np.array([0, 0, 1, 7, 0], np.uint8)
    o = oracle_mod.fit_spots(img, offs, dims, np.ones((5, 4), np.float32), model)
    assert list(o["state"]) == [-2] * 5
    assert np.all(np.isnan(o["alpha"])) and list(o["iters"]) == [0] * 5


# ---------------------------------------------------------------- Table 1 and Fig. 8
def _golden_table1():
    rows = []
    for line in (GOLDEN / "table1_fit2dgaussian.txt").read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            rows.append([float(v) for v in line.split()])
    return rows


@pytest.mark.parametrize("row", range(3))
def test_reproduces_table1_accuracy(oracle_mod, row):
    """100,000 fits with the paper's simulation protocol reproduce the Fit2DGaussian rows
    of Table 1. Centre errors agree within 3 % (statistical error ~0.3 %); width errors
    within 7 % (our widths scatter 1-5 % more than printed, from protocol details the
    text does not fix)."""
    sig, bg, *ref = _golden_table1()[row]
    b = synth.make_paper(100_000, 9, sig, bg, seed=synth.SEED_BASE + 10 + row)
    d = b.numpy()
    o = oracle_mod.fit_spots(d["images"], d["offsets"], d["dims"], d["init"], d["model"])
    tp = b.truth["params"].numpy()
    st = tp[:, 2]
    ex = np.concatenate([np.abs(o["params"][:, 0] - tp[:, 0]), np.abs(o["params"][:, 1] - tp[:, 1])])
    ex = ex / np.concatenate([st, st])
    es = np.abs(np.abs(o["params"][:, 2]) - st) / st
    got = [np.median(ex), ex.mean(), ex.std(), np.median(es), es.mean(), es.std()]
    for k in range(3):
        assert abs(got[k] / ref[k] - 1) < 0.03, (k, got, ref)
    for k in range(3, 6):
        assert abs(got[k] / ref[k] - 1) < 0.07, (k, got, ref)
    if row == 1:   # "typically terminated after 4 or 5 iterations" at 1600:40 (Fig. 8)
        hist = np.bincount(o["iters"])
        assert int(np.argmax(hist)) in (4, 5)
        assert (hist[4] + hist[5]) / hist.sum() > 0.8


def _golden_stop():
    out = {}
    for line in (GOLDEN / "stop_conditions_fit2dgaussian.txt").read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            name, lo, hi = line.split()
            out[name] = (float(lo), float(hi))
    return out


def test_paper_arithmetic_reproduces_the_stop_conditions(oracle_mod):
    """The stop conditions the paper reports for 1600:40 pin the LM control flow (damping
    escalation, the no-decrease exit, the order of the stop tests). They come from the
    paper's own arithmetic: its FP32 chi^2 has a rounding floor near the 1e-6 minDelta
    threshold, so some final trials fail to decrease, and its minStep test is relative to
    coordinates near zero. The oracle's second build, with FP32 chi^2 over pixel threads and
    the minStep test relative to the ROI centre, reproduces the reported shares; the FP64
    build reaches the same fits but has no rounding floor, so it shows no such exits."""
    codes = {"MIN_DELTA": 1, "MIN_STEP": 2, "NO_DECREASE": 4, "MAX_ITER": 0}
    bands = _golden_stop()
    b = synth.make_paper(100_000, 9, 1600, 40, seed=synth.SEED_BASE + 11)
    d = b.numpy()
    paper = oracle_mod.fit_spots(d["images"], d["offsets"], d["dims"], d["init"], d["model"],
                                 paper_arithmetic=True)
    shares = {k: float(np.mean(paper["state"] == c)) for k, c in codes.items()}
    for name, (lo, hi) in bands.items():
        assert lo <= shares[name] <= hi, (name, shares)
    assert np.isin(paper["state"], (1, 2, 3, 4)).mean() >= 0.995, shares
    fp64 = oracle_mod.fit_spots(d["images"], d["offsets"], d["dims"], d["init"], d["model"])
    assert np.mean(fp64["state"] == 4) < 0.005
    # both builds end at the same fits (to well inside the spots' statistical errors)
    conv = np.isin(paper["state"], (1, 2, 4)) & np.isin(fp64["state"], (1, 2, 4))
    dx = np.abs(paper["params"][conv, :2] - fp64["params"][conv, :2])
    assert np.median(dx) < 1e-3 and np.percentile(dx, 99) < 2e-2


@pytest.mark.parametrize("model,S", [(0, 9), (1, 15)])
def test_normalised_chi2_is_the_residual_variance(oracle_mod, model, S):
    """Reading R9 (the paper names a normalised chi^2 without its divisor): chi^2 / (N - P - 2)
    is the unbiased estimate of the pixel noise variance at the minimum over the P shape
    parameters and the two amplitudes. With white Gaussian noise of variance 1 its mean over
    many well-determined fits is 1 to within sampling error, which the other candidate
    divisors (N, N - P) miss by several standard errors."""
    rng = np.random.default_rng(91 + S)
    n, N = 6000, S * S
    P = 3 if model == 0 else 4
    ys, xs = np.mgrid[0:S, 0:S]
    imgs, inits = [], []
    for _ in range(n):
        c = (S - 1) / 2
        p = np.array([c + rng.uniform(-0.5, 0.5), c + rng.uniform(-0.5, 0.5),
                      rng.uniform(1.2, 2.0), rng.uniform(1.2, 2.0)])
        if model == 0:
            p[3] = p[2]
        f = np.exp(-0.5 * ((xs - p[0]) / p[2]) ** 2 - 0.5 * ((ys - p[1]) / p[3]) ** 2)
        imgs.append((400.0 * f + 20.0 + rng.normal(size=f.shape)).ravel())
        inits.append(p * np.array([1.0, 1.0, 1.05, 0.95]))
    img = np.concatenate(imgs)
    out = oracle_mod.fit_spots(img, np.arange(n, dtype=np.int64) * N,
                               np.tile(np.array([[S, S]], np.int32), (n, 1)),
                               np.array(inits, np.float32), np.full(n, model, np.uint8),
                               max_iter=100, min_delta=0.0, min_step=1e-10)
    ok = np.isin(out["state"], (1, 2, 4))
    assert ok.mean() > 0.99
    c2n = out["chi2"][ok]
    se = c2n.std() / np.sqrt(c2n.size)
    mean = c2n.mean()
    print(f"model {model}, {S}x{S}: mean chi2/(N-P-2) {mean:.4f} +- {se:.4f}")
    assert abs(mean - 1.0) < 4 * se
    for dof in (N, N - P):   # the alternatives are off by (P + 2) / N or 2 / N
        assert abs(mean * (N - P - 2) / dof - 1.0) > 4 * se
