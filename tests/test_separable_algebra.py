"""The separable reformulation the CUDA kernels use, checked in FP64 on the host.

The kernels never form the per-pixel Jacobian of Eq. 9. Because f = e_x(x) e_y(y), they
reduce each evaluation to 17 one-dimensional moments of e_x and e_y, one bilinear sum
e_x^T G e_y, and five row/column-weighted sums of the residual; the LM step assembles
alpha^, beta^ (Eq. 6), J^T r and J^T J (Eq. 12-14) from those. This test writes that
assembly out in numpy (double precision, same sums and formulas as the kernel's LM step) and
compares it with the oracle's explicit per-pixel normal equations, so an algebra slip in
the reformulation would show here apart from any FP32 rounding. The backward kernel's
separable system (13 bilinear data sums, 1-D moments, the 6 x 6 system of the
implicit-function theorem and its per-pixel gradient formula) is checked the same way
against the oracle's backward."""
import numpy as np
import pytest

ISO, ELL = 0, 1


def _sums(g, W, H, R, pe, iso, shift):
    """The kernel's per-evaluation sums at trial point pe (x0, y0, sx, sy); R >= H is the
    compiled row count of the configuration (padding rows contribute nothing), on whose
    centre R / 2 the row weights are taken."""
    sx, sy = pe[2], (pe[2] if iso else pe[3])
    x = np.arange(W, dtype=np.float64)
    y = np.arange(H, dtype=np.float64)
    dx, dy = x - pe[0], y - pe[1]
    ex = np.exp(-0.5 * dx**2 / sx**2)
    ey = np.exp(-0.5 * dy**2 / sy**2)
    G = g.reshape(H, W) - shift                       # g' = g - shift, [y][x]
    X = dict(X01=ex.sum(), X02=(ex**2).sum(), X11=(dx * ex).sum(), X21=(dx**2 * ex).sum(),
             X12=(dx * ex**2).sum(), X22=(dx**2 * ex**2).sum(), X32=(dx**3 * ex**2).sum(),
             X42=(dx**4 * ex**2).sum())
    Y = dict(Y01=ey.sum(), Y02=(ey**2).sum(), Y11=(dy * ey).sum(), Y21=(dy**2 * ey).sum(),
             Y12=(dy * ey**2).sum(), Y22=(dy**2 * ey**2).sum(), Y32=(dy**3 * ey**2).sum(),
             Y42=(dy**4 * ey**2).sum())
    FG = ex @ G.T @ ey                                # pass 1: e_x^T G' e_y
    Gs = G.sum()
    N = W * H
    F, FF = X["X01"] * Y["Y01"], X["X02"] * Y["Y02"]
    D = N * FF - F * F
    alpha = (N * FG - F * Gs) / D                     # Eq. 6
    bp = (Gs * FF - F * FG) / D                       # beta^ - shift
    U = G - alpha * np.outer(ey, ex)                  # pass 2: u = g' - alpha e_x e_y
    yt = y - 0.5 * R
    t0 = ey @ U                                       # per column: sum_y e_y u
    t1 = (yt * ey) @ U
    t2 = (yt**2 * ey) @ U
    T = dict(chiu=(U**2).sum(), Tf=ex @ t0, Tx=(dx * ex) @ t0, Txx=(dx**2 * ex) @ t0,
             Ty1=ex @ t1, Ty2=ex @ t2)
    return X, Y, T, alpha, bp, Gs, F, FF, N, R


def _assemble(X, Y, T, alpha, bp, Gs, F, FF, N, R, pe, iso):
    """J^T J (packed upper triangle of 4 x 4) and J^T r, the kernel's LM-step formulas."""
    D = N * FF - F * F
    sx, sy = pe[2], (pe[2] if iso else pe[3])
    ivx, ivy = 1 / sx**2, 1 / sy**2
    cx, cy = ivx / sx, ivy / sy
    eta = pe[1] - 0.5 * R
    Sfdy = T["Ty1"] - eta * T["Tf"]
    Sfdy2 = T["Ty2"] - 2 * eta * T["Ty1"] + eta**2 * T["Tf"]
    Rd = np.array([ivx * (T["Tx"] - bp * X["X11"] * Y["Y01"]),
                   ivy * (Sfdy - bp * X["X01"] * Y["Y11"]),
                   cx * (T["Txx"] - bp * X["X21"] * Y["Y01"]),
                   cy * (Sfdy2 - bp * X["X01"] * Y["Y21"])])
    D1 = np.array([X["X11"] * Y["Y01"] * ivx, X["X01"] * Y["Y11"] * ivy,
                   X["X21"] * Y["Y01"] * cx, X["X01"] * Y["Y21"] * cy])
    Fd = np.array([X["X12"] * Y["Y02"] * ivx, X["X02"] * Y["Y12"] * ivy,
                   X["X22"] * Y["Y02"] * cx, X["X02"] * Y["Y22"] * cy])
    aa = (N * Rd - alpha * (N * Fd - F * D1)) / D
    bb = (alpha * (F * Fd - FF * D1) - F * Rd) / D
    Dd = np.array([X["X22"] * Y["Y02"] * ivx * ivx, X["X12"] * Y["Y12"] * ivx * ivy,
                   X["X32"] * Y["Y02"] * ivx * cx, X["X12"] * Y["Y22"] * ivx * cy,
                   X["X02"] * Y["Y22"] * ivy * ivy, X["X22"] * Y["Y12"] * ivy * cx,
                   X["X02"] * Y["Y32"] * ivy * cy, X["X42"] * Y["Y02"] * cx * cx,
                   X["X22"] * Y["Y22"] * cx * cy, X["X02"] * Y["Y42"] * cy * cy])
    M = np.empty(10)
    idx = 0
    for r in range(4):
        for k in range(r, 4):
            M[idx] = aa[r] * Rd[k] + alpha * (Fd[r] * aa[k] + D1[r] * bb[k]) + alpha**2 * Dd[idx]
            idx += 1
    if iso:
        A = np.array([[M[0], M[1], M[2] + M[3]],
                      [M[1], M[4], M[5] + M[6]],
                      [M[2] + M[3], M[5] + M[6], M[7] + 2 * M[8] + M[9]]])
        b = alpha * np.array([Rd[0], Rd[1], Rd[2] + Rd[3]])
    else:
        up = np.zeros((4, 4))
        up[np.triu_indices(4)] = M
        A = up + np.triu(up, 1).T
        b = alpha * Rd
    return A, b


@pytest.mark.parametrize("model", [ISO, ELL])
def test_separable_normal_equations_equal_the_per_pixel_form(oracle_mod, model):
    rng = np.random.default_rng(31 + model)
    for _ in range(30):
        W, H = int(rng.integers(5, 33)), int(rng.integers(5, 33))
        truth = [(W - 1) / 2 + rng.uniform(-1, 1), (H - 1) / 2 + rng.uniform(-1, 1),
                 rng.uniform(1.0, 3.0), rng.uniform(1.0, 3.0)]
        ys, xs = np.mgrid[0:H, 0:W]
        sy_t = truth[2] if model == ISO else truth[3]
        lam = 900 * np.exp(-0.5 * ((xs - truth[0]) / truth[2]) ** 2
                           - 0.5 * ((ys - truth[1]) / sy_t) ** 2) + 120
        g = rng.poisson(lam).astype(np.float64).ravel()
        # away from the minimum: J^T r does not vanish there
        pe = np.array(truth) + rng.uniform(-0.5, 0.5, 4) * [1, 1, 0.3, 0.3]
        if model == ISO:
            pe[3] = pe[2]
        shift = float(np.rint(g.min()))
        R = int(rng.integers(H, 33))
        X, Y, T, alpha, bp, Gs, F, FF, N, R = _sums(g, W, H, R, pe, model == ISO, shift)
        A, b = _assemble(X, Y, T, alpha, bp, Gs, F, FF, N, R, pe, model == ISO)
        ref = oracle_mod.evaluate(model, W, H, g, pe)
        assert abs(alpha - ref["alpha"]) <= 1e-10 * abs(ref["alpha"])
        assert abs(bp + shift - ref["beta"]) <= 1e-9 * abs(ref["beta"])
        # chi^2 = sum (u - beta')^2 = chi_u - 2 beta' sum u + N beta'^2, sum u = G' - alpha F
        Su = Gs - alpha * F
        chi = T["chiu"] - 2 * bp * Su + N * bp * bp
        assert abs(chi - ref["chi2"]) <= 1e-9 * ref["chi2"]
        scale = np.sqrt(np.outer(np.diag(ref["A"]), np.diag(ref["A"])))
        assert np.max(np.abs(A - ref["A"]) / scale) < 1e-9
        assert np.max(np.abs(b - ref["b"]) / np.sqrt(np.diag(ref["A"]) * ref["chi2"])) < 1e-9


def _backward_separable(g, W, H, p, al, beta, up, iso):
    """The backward kernel's path in FP64: 13 data sums G_ab = sum g' e_x dx^a e_y dy^b, the
    1-D moments, M over q = (x0, y0, sx, sy, alpha, beta) with the isotropic fold, M v = u,
    then grad = e_x e_y (alpha (A(x) + B(y)) + v_alpha) + v_beta + c (g - alpha f - beta)."""
    sh = float(np.rint(beta))
    bp = beta - sh
    sx, sy = p[2], (p[2] if iso else p[3])
    ivx, ivy = 1 / sx**2, 1 / sy**2
    cx, cy = ivx / sx, ivy / sy
    dx = np.arange(W) - p[0]
    dy = np.arange(H) - p[1]
    ex = np.exp(-0.5 * dx**2 * ivx)
    ey = np.exp(-0.5 * dy**2 * ivy)
    Gp = g.reshape(H, W) - sh
    G = {(a, b): (ex * dx**a) @ Gp.T @ (ey * dy**b)
         for a, b in ((0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2), (3, 0), (2, 1), (1, 2),
                      (0, 3), (4, 0), (2, 2), (0, 4))}
    E = [(ex * dx**m).sum() for m in range(5)]
    P = [(ex**2 * dx**m).sum() for m in range(5)]
    F = [(ey * dy**m).sum() for m in range(5)]
    Q = [(ey**2 * dy**m).sum() for m in range(5)]
    N = W * H
    DD = [ivx * ivx * P[2] * Q[0], ivx * ivy * P[1] * Q[1], ivx * cx * P[3] * Q[0],
          ivx * cy * P[1] * Q[2], ivy * ivy * P[0] * Q[2], ivy * cx * P[2] * Q[1],
          ivy * cy * P[0] * Q[3], cx * cx * P[4] * Q[0], cx * cy * P[2] * Q[2],
          cy * cy * P[0] * Q[4]]
    FD = [ivx * P[1] * Q[0], ivy * P[0] * Q[1], cx * P[2] * Q[0], cy * P[0] * Q[2]]
    SD = [ivx * E[1] * F[0], ivy * E[0] * F[1], cx * E[2] * F[0], cy * E[0] * F[2]]
    GD = [ivx * G[1, 0], ivy * G[0, 1], cx * G[2, 0], cy * G[0, 2]]
    # sum g' h_jk, sum f h_jk, sum h_jk for the second derivatives h_jk of f / f
    def hsum(s2):   # s2(a, b): the family's sum weighted by dx^a dy^b
        return [ivx * ivx * s2(2, 0) - ivx * s2(0, 0), ivx * ivy * s2(1, 1),
                ivx * cx * s2(3, 0) - 2 * cx * s2(1, 0), ivx * cy * s2(1, 2),
                ivy * ivy * s2(0, 2) - ivy * s2(0, 0), ivy * cx * s2(2, 1),
                ivy * cy * s2(0, 3) - 2 * cy * s2(0, 1),
                cx * cx * s2(4, 0) - 3 * ivx * ivx * s2(2, 0), cx * cy * s2(2, 2),
                cy * cy * s2(0, 4) - 3 * ivy * ivy * s2(0, 2)]
    GH = hsum(lambda a, b: G[a, b])
    FH = hsum(lambda a, b: P[a] * Q[b])
    SH = hsum(lambda a, b: E[a] * F[b])
    M = np.zeros((6, 6))
    t = 0
    for j in range(4):
        for k in range(j, 4):
            rh = GH[t] - al * FH[t] - bp * SH[t]
            M[j, k] = M[k, j] = al * (al * DD[t] - rh)
            t += 1
    for j in range(4):
        rd = GD[j] - al * FD[j] - bp * SD[j]
        M[j, 4] = M[4, j] = al * FD[j] - rd
        M[j, 5] = M[5, j] = al * SD[j]
    M[4, 4], M[4, 5], M[5, 4], M[5, 5] = P[0] * Q[0], E[0] * F[0], E[0] * F[0], N
    v = np.array(up[:6], dtype=np.float64)
    if iso:
        M[2, :] += M[3, :]
        M[:, 2] += M[:, 3]
        v[2] += v[3]
        M[3, :] = 0
        M[:, 3] = 0
        M[3, 3] = 1
        v[3] = 0
    v = np.linalg.solve(M, v)
    Ps = 3 if iso else 4
    vx, vy, vsx, vsy = v[0] * ivx, v[1] * ivy, v[2] * cx, (v[2] if iso else v[3]) * cy
    cchi = 2 * up[6] / (N - Ps - 2)
    Ax = dx * (vx + vsx * dx)
    By = dy * (vy + vsy * dy)
    f = np.outer(ey, ex)
    grad = f * (al * (Ax[None, :] + By[:, None]) + v[4]) + v[5] \
        + cchi * (g.reshape(H, W) - al * f - beta)
    return grad.ravel()


@pytest.mark.parametrize("model", [ISO, ELL])
def test_separable_backward_equals_the_oracle_ift(oracle_mod, model):
    """The backward kernel's separable system and gradient formula, in FP64, against the
    oracle's implicit-function-theorem VJP (explicit per-pixel K, second derivatives)."""
    rng = np.random.default_rng(41 + model)
    for _ in range(20):
        W, H = int(rng.integers(5, 33)), int(rng.integers(5, 33))
        truth = [(W - 1) / 2 + rng.uniform(-1, 1), (H - 1) / 2 + rng.uniform(-1, 1),
                 rng.uniform(1.2, 2.5), rng.uniform(1.2, 2.5)]
        sy_t = truth[2] if model == ISO else truth[3]
        ys, xs = np.mgrid[0:H, 0:W]
        lam = 1500 * np.exp(-0.5 * ((xs - truth[0]) / truth[2]) ** 2
                            - 0.5 * ((ys - truth[1]) / sy_t) ** 2) + 90
        g = rng.poisson(lam).astype(np.float64).ravel()
        init = np.array([truth], np.float32)
        if model == ISO:
            init[0, 3] = init[0, 2]
        o = oracle_mod.fit_spots(g, [0], [[W, H]], init, np.array([model], np.uint8),
                                 max_iter=200, min_delta=0.0, min_step=1e-13)
        p, al, be = o["params"][0], o["alpha"][0], o["beta"][0]
        up = rng.standard_normal(7)
        ref = oracle_mod.backward(model, W, H, g, p, al, be, up)
        assert ref is not None
        got = _backward_separable(g, W, H, p, al, be, up, model == ISO)
        assert np.linalg.norm(got - ref) <= 1e-9 * np.linalg.norm(ref)


@pytest.mark.parametrize("model", [ISO, ELL])
def test_tie_refinement_equals_the_chi2_difference(oracle_mod, model):
    """The kernels' refinement of a near-tie decision: with b the best point and t the trial,
    h_t - h_b = f_b (alpha_t tt + alpha_t - alpha_b) + beta'_t - beta'_b, where
    1 + tt = f_t / f_b = (1 + m_x)(1 + m_y) is formed from the exponent differences
    m = expm1(d0 (dt + db) iv_t / 2 + db^2 (iv_b - iv_t) / 2) per axis, and
    chi2_t - chi2_b = sum dh (dh - 2 r_b). Written out in FP64, it equals the difference of
    the oracle's chi^2 at the two points."""
    rng = np.random.default_rng(51 + model)
    for _ in range(30):
        W, H = int(rng.integers(5, 33)), int(rng.integers(5, 33))
        truth = np.array([(W - 1) / 2 + rng.uniform(-1, 1), (H - 1) / 2 + rng.uniform(-1, 1),
                          rng.uniform(1.2, 2.5), rng.uniform(1.2, 2.5)])
        if model == ISO:
            truth[3] = truth[2]
        ys, xs = np.mgrid[0:H, 0:W]
        lam = 1200 * np.exp(-0.5 * ((xs - truth[0]) / truth[2]) ** 2
                            - 0.5 * ((ys - truth[1]) / truth[3]) ** 2) + 80
        g = rng.poisson(lam).astype(np.float64).ravel()
        pb = truth + rng.uniform(-0.05, 0.05, 4) * [1, 1, 0.2, 0.2]
        pt = pb + rng.uniform(-1e-3, 1e-3, 4) * [1, 1, 0.1, 0.1]
        if model == ISO:
            pb[3], pt[3] = pb[2], pt[2]
        eb, et = oracle_mod.evaluate(model, W, H, g, pb), oracle_mod.evaluate(model, W, H, g, pt)
        ab, bb_, at, bt = eb["alpha"], eb["beta"], et["alpha"], et["beta"]

        def mvec(n, c_t, c_b, s_t, s_b):
            pos = np.arange(n, dtype=np.float64)
            dt, db = pos - c_t, pos - c_b
            ivt, ivb = 1 / s_t**2, 1 / s_b**2
            return np.expm1(0.5 * ((c_t - c_b) * (dt + db) * ivt + db**2 * (ivb - ivt))), db, ivb
        mx, dbx, ivbx = mvec(W, pt[0], pb[0], pt[2], pb[2])
        my, dby, ivby = mvec(H, pt[1], pb[1], pt[3], pb[3])
        exb, eyb = np.exp(-0.5 * dbx**2 * ivbx), np.exp(-0.5 * dby**2 * ivby)
        fb = np.outer(eyb, exb)
        tt = np.outer(my, 1 + mx) + mx[None, :]
        dh = fb * (at * tt + (at - ab)) + (bt - bb_)
        rb = g.reshape(H, W) - ab * fb - bb_
        delta = (dh * (dh - 2 * rb)).sum()
        exact = et["chi2"] - eb["chi2"]
        assert abs(delta - exact) <= 1e-7 * abs(exact) + 1e-12 * eb["chi2"]


def test_fp32_separable_normal_matrix_loses_digits_only_on_flat_profiles(oracle_mod):
    """Why FP32 fits part from the FP64 oracle on flat chi^2 surfaces: the separable J^T J is a
    small difference of large products of 1-D moments when the profile is nearly flat over
    the ROI (widths near the ROI size), so the same formulas evaluated from FP32-rounded sums
    in FP32 lose digits there and not on compact spots. (The GPU kernels form these sums and
    this assembly in FP32.)"""
    rng = np.random.default_rng(77)
    W = H = 32
    ys, xs = np.mgrid[0:H, 0:W]

    def rel_err(s_true):
        errs = []
        for _ in range(20):
            p = np.array([15.5 + rng.uniform(-1, 1), 15.5 + rng.uniform(-1, 1),
                          s_true * rng.uniform(0.9, 1.1), s_true * rng.uniform(0.9, 1.1)])
            f = np.exp(-0.5 * ((xs - p[0]) / p[2]) ** 2 - 0.5 * ((ys - p[1]) / p[3]) ** 2)
            g = rng.poisson(60.0 * f + 300.0).astype(np.float64).ravel()
            ref = oracle_mod.evaluate(ELL, W, H, g, p)
            shift = float(np.rint(ref["beta"]))
            X, Y, T, alpha, bp, Gs, F, FF, N, R = _sums(g, W, H, 32, p, False, shift)
            f32 = lambda v: ({k: np.float32(x) for k, x in v.items()} if isinstance(v, dict)
                             else np.float32(v))
            A32, _ = _assemble(f32(X), f32(Y), f32(T), f32(alpha), f32(bp), f32(Gs), f32(F),
                               f32(FF), N, R, p.astype(np.float32), False)
            d = np.abs(np.diag(A32) - np.diag(ref["A"])) / np.abs(np.diag(ref["A"]))
            errs.append(d.max())
        return float(np.median(errs))

    compact, flat = rel_err(2.0), rel_err(20.0)
    print(f"FP32 separable J^T J, max relative diagonal error: compact spots {compact:.1e}, "
          f"flat spots {flat:.1e}")
    assert compact < 1e-5
    assert flat > 10 * compact   # measured: about 35 times
