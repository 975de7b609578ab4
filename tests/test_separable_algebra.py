"""The separable reformulation the CUDA kernels use, checked in FP64 on the host.

The kernels never form the per-pixel Jacobian of Eq. 9. Because f = e_x(x) e_y(y), they
reduce each evaluation to 17 one-dimensional moments of e_x and e_y, one bilinear sum
e_x^T G e_y, and five row/column-weighted sums of the residual; the LM step assembles
alpha^, beta^ (Eq. 6), J^T r and J^T J (Eq. 12-14) from those. This test writes that
assembly out in numpy (double precision, same sums and formulas as the kernel's LM step) and
compares it with the oracle's explicit per-pixel normal equations, so an algebra slip in
the reformulation would show here apart from any FP32 rounding."""
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
