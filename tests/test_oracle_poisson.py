"""Pins of the oracle's Poisson-likelihood fit (deviance objective, amplitudes at their
Poisson maximum likelihood for each profile): the amplitudes solve the score equations and
equal a generic optimiser's, noise-free spots are recovered exactly, a converged fit is the
maximum of the Poisson likelihood over all explicit unknowns (scipy), its gradient is the
deviance slope, and on Poisson spots it reaches the Cramer-Rao bound."""
import numpy as np
import pytest

from paper_2106_02045_gb300 import synth
from tests.test_oracle_weighted import _cramer_rao

ISO, ELL = 0, 1


def _profile(W, H, p):
    x, y = np.arange(W)[None, :], np.arange(H)[:, None]
    return np.exp(-0.5 * ((x - p[0]) / p[2]) ** 2 - 0.5 * ((y - p[1]) / p[3]) ** 2).ravel()


def _nll(h, g):
    """Poisson negative log-likelihood up to a constant."""
    return float(np.sum(h - g * np.log(h)))


def test_amplitudes_solve_the_score_equations(oracle_mod):
    from scipy.optimize import minimize
    rng = np.random.default_rng(5)
    for _ in range(20):
        W, H = int(rng.integers(7, 20)), int(rng.integers(7, 20))
        p = [(W - 1) / 2 + rng.uniform(-1, 1), (H - 1) / 2 + rng.uniform(-1, 1),
             rng.uniform(1.0, 2.5), rng.uniform(1.0, 2.5)]
        f = _profile(W, H, p)
        g = rng.poisson(rng.uniform(50, 2000) * f + rng.uniform(2, 200)).astype(np.float64)
        # at a profile that is not the data's: the amplitudes are still the likelihood optimum
        fq = _profile(W, H, [p[0] + 0.3, p[1] - 0.2, p[2] * 1.1, p[3] * 0.9])
        a, b = oracle_mod.poisson_amplitudes(fq, g)
        h = a * fq + b
        score = np.array([np.sum((g / h - 1) * fq), np.sum(g / h - 1)])
        scale = np.array([np.sum(g / h * fq), np.sum(g / h)])
        assert np.all(np.abs(score) <= 1e-10 * scale)
        sol = minimize(lambda v: _nll(np.maximum(v[0] * fq + v[1], 1e-300), g), [0.8 * a, 1.1 * b],
                       method="Nelder-Mead", options=dict(xatol=1e-10, fatol=1e-14, maxiter=20000))
        assert abs(sol.x[0] - a) <= 1e-5 * abs(a) + 1e-6 and abs(sol.x[1] - b) <= 1e-5 * abs(b)
        assert _nll(h, g) <= sol.fun + 1e-9 * abs(sol.fun)


@pytest.mark.parametrize("model", [ISO, ELL])
def test_poisson_fit_recovers_noise_free_spots(oracle_mod, model):
    rng = np.random.default_rng(9 + model)
    spots, dims, init, truth = [], [], [], []
    for _ in range(30):
        W, H = int(rng.integers(7, 33)), int(rng.integers(7, 33))
        p = np.array([(W - 1) / 2 + rng.uniform(-1, 1), (H - 1) / 2 + rng.uniform(-1, 1),
                      rng.uniform(1.0, min(2.5, min(W, H) / 4)), rng.uniform(1.0, min(2.5, min(W, H) / 4))])
        if model == ISO:
            p[3] = p[2]
        amp, bg = rng.uniform(100, 5000), rng.uniform(1, 300)
        spots.append(amp * _profile(W, H, p) + bg)
        dims.append((W, H))
        q = p + np.array([rng.uniform(-0.7, 0.7), rng.uniform(-0.7, 0.7), 0, 0])
        q[2] *= rng.uniform(0.8, 1.25)
        q[3] = q[2] if model == ISO else q[3] * rng.uniform(0.8, 1.25)
        init.append(q)
        truth.append((p, amp, bg))
    offs = np.cumsum([0] + [s.size for s in spots[:-1]])
    o = oracle_mod.fit_spots_poisson(np.concatenate(spots), offs, dims, np.array(init, np.float32),
                                     np.full(len(spots), model, np.uint8), max_iter=200,
                                     min_delta=0.0, min_step=1e-13)
    for s, (p, amp, bg) in enumerate(truth):
        assert np.max(np.abs(o["params"][s] - p)) < 1e-8, (s, o["params"][s], p)
        assert abs(o["alpha"][s] - amp) < 1e-8 * amp and abs(o["beta"][s] - bg) < 1e-7 * amp
        assert abs(o["chi2"][s]) < 1e-9   # the deviance of a perfect model is 0


def _explicit_mle(model, W, H, g, v0):
    """The Poisson maximum likelihood over all explicit unknowns (shape, alpha, beta)."""
    from scipy.optimize import minimize

    def nll(v):
        if model == ISO:
            x0, y0, s, a, b = v
            sx = sy = s
        else:
            x0, y0, sx, sy, a, b = v
        h = a * _profile(W, H, [x0, y0, sx, sy]) + b
        return _nll(h, g) if np.all(h > 0) else 1e300
    sol = minimize(nll, v0, method="Nelder-Mead",
                   options=dict(xatol=1e-9, fatol=1e-13, maxiter=200000, maxfev=200000))
    sol = minimize(nll, sol.x, method="Nelder-Mead",
                   options=dict(xatol=1e-10, fatol=1e-14, maxiter=200000, maxfev=200000))
    return sol.x, sol.fun


@pytest.mark.parametrize("model", [ISO, ELL])
def test_converged_fit_is_the_poisson_maximum_likelihood(oracle_mod, model):
    """The fixed point maximises the Poisson likelihood over all 5 / 6 explicit unknowns
    (scipy's simplex on the explicit likelihood), its deviance is twice the log-likelihood
    ratio against the saturated model, and it differs from the least-squares minimum."""
    rng = np.random.default_rng(31 + model)
    moved = 0.0
    for _ in range(6):
        W, H = int(rng.integers(9, 17)), int(rng.integers(9, 17))
        p = np.array([(W - 1) / 2 + rng.uniform(-1, 1), (H - 1) / 2 + rng.uniform(-1, 1),
                      rng.uniform(1.2, 2.2), rng.uniform(1.2, 2.2)])
        if model == ISO:
            p[3] = p[2]
        g = rng.poisson(600.0 * _profile(W, H, p) + 20.0).astype(np.float64)
        init = np.array([[p[0] + 0.3, p[1] - 0.2, p[2] * 1.1, p[3] * (1.1 if model else 1.1)]],
                        np.float32)
        if model == ISO:
            init[0, 3] = init[0, 2]
        o = oracle_mod.fit_spots_poisson(g, [0], [[W, H]], init, np.array([model], np.uint8),
                                         max_iter=300, min_delta=0.0, min_step=1e-13)
        u = oracle_mod.fit_spots(g, [0], [[W, H]], init, np.array([model], np.uint8),
                                 max_iter=300, min_delta=0.0, min_step=1e-13)
        assert o["state"][0] in (1, 2, 4)
        P = 3 if model == ISO else 4
        pw, a, b = o["params"][0], o["alpha"][0], o["beta"][0]
        v0 = list(pw[:P] + 0.03) + [0.95 * a, 1.05 * b]
        xv, nll_s = _explicit_mle(model, W, H, g, v0)
        h = a * _profile(W, H, pw) + b
        assert _nll(h, g) <= nll_s + 1e-9 * abs(nll_s)
        assert np.max(np.abs(xv[:P] - pw[:P])) < 2e-5
        gp = np.where(g > 0, g * np.log(np.where(g > 0, g, 1) / h), 0.0)
        dev = 2 * float(np.sum(h - g + gp))
        assert abs(dev - o["chi2"][0] * (W * H - P - 2)) <= 1e-9 * dev
        moved = max(moved, float(np.max(np.abs(u["params"][0][:P] - pw[:P]))))
    assert moved > 1e-3   # the likelihood's maximum is not the least-squares minimum


def test_poisson_fit_reaches_the_cramer_rao_bound(oracle_mod):
    """Poisson spots (iso15: peak 1000, background 100): the Poisson fit's centre and width
    errors have the spread the Cramer-Rao bound allows, without bias; the unweighted fit's
    spread is 13-20 % larger."""
    b = synth.make_workload("iso15", 4000)
    d = b.numpy()
    img = synth.as_numpy_images(b)
    tp = b.truth["params"].numpy()
    bound = _cramer_rao(15, 15, tp, b.truth["alpha"].numpy(), b.truth["beta"].numpy())
    o = oracle_mod.fit_spots_poisson(img, d["offsets"], d["dims"], d["init"], d["model"])
    assert np.isin(o["state"], (1, 2, 3, 4)).all()
    z = (o["params"][:, :3] - tp[:, :3]) / bound
    assert np.all(np.abs(z.mean(0)) < 0.08), z.mean(0)
    sp = z.std(0)
    assert np.all(sp > 0.97) and np.all(sp < 1.04), sp
    u = oracle_mod.fit_spots(img, d["offsets"], d["dims"], d["init"], d["model"])
    su = ((u["params"][:, :3] - tp[:, :3]) / bound).std(0)
    assert np.all(su > 1.08 * sp), (su, sp)
