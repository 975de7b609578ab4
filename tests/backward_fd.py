"""Finite-difference vector-Jacobian products of the fit, from polished FP64 oracle refits
(test code only).

For a spot with pixels g and an upstream vector u over the fitted (x0, y0, sigma_x, sigma_y,
alpha, beta, chi2_n), the derivative of u . q(g) with respect to pixel i is taken as the
central difference (u . q(g + h_i e_i) - u . q(g - h_i e_i)) / 2 h_i, where q is the FP64
oracle fit polished to the rounding floor (min_delta 0, min_step 1e-13, up to 300
iterations) from the unperturbed fit, and h_i = 1e-2 max(1, sqrt|g_i|), about 1 % of the
pixel's Poisson noise. The fit is the minimum of Eq. 2 with the amplitudes of Eq. 6, so this
is the derivative that the implicit-function-theorem backward must reproduce.
"""
from __future__ import annotations

import numpy as np

POLISH = dict(max_iter=300, min_delta=0.0, min_step=1e-13)


def polished(images, offsets, dims, init, model):
    import oracle
    return oracle.fit_spots(images, offsets, dims, init, model, **POLISH)


def fd_vjp(img: np.ndarray, offsets, dims, model, params, upstream, chunk_spots: int = 32):
    """Central-difference VJPs of spots with equal W x H, one row of ``upstream`` (7 values)
    per spot; ``params`` are the polished fits the refits start from. Returns an (n, W*H)
    FP64 array and the states of all refits."""
    offsets = np.asarray(offsets, np.int64)
    dims = np.asarray(dims, np.int32)
    n = len(offsets)
    W, H = int(dims[0, 0]), int(dims[0, 1])
    assert (dims == [W, H]).all(), "one ROI size per call"
    N = W * H
    out = np.empty((n, N))
    states = []
    eye = np.eye(N)
    for c0 in range(0, n, chunk_spots):
        c1 = min(n, c0 + chunk_spots)
        m = c1 - c0
        g = np.stack([img[offsets[s]:offsets[s] + N].astype(np.float64) for s in range(c0, c1)])
        h = 1e-2 * np.maximum(1.0, np.sqrt(np.abs(g)))               # (m, N)
        # (m, N pixels perturbed, 2 signs, N) ROIs: + h e_i then - h e_i
        pert = np.stack([g[:, None, :] + (h[:, :, None] * eye[None]),
                         g[:, None, :] - (h[:, :, None] * eye[None])], axis=2)
        M = m * N * 2
        o = polished(pert.reshape(-1), np.arange(M, dtype=np.int64) * N,
                     np.tile(np.array([[W, H]], np.int32), (M, 1)),
                     np.repeat(np.asarray(params[c0:c1], np.float32), N * 2, axis=0),
                     np.repeat(np.asarray(model[c0:c1], np.uint8), N * 2))
        states.append(o["state"])
        q = np.concatenate([o["params"], o["alpha"][:, None], o["beta"][:, None],
                            o["chi2"][:, None]], axis=1).reshape(m, N, 2, 7)
        u = np.asarray(upstream[c0:c1], np.float64)[:, None, None, :]
        val = (q * u).sum(-1)                                           # (m, N, 2)
        out[c0:c1] = (val[..., 0] - val[..., 1]) / (2 * h)
    return out, np.concatenate(states)


def rel_err(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Per-row ||a - b|| / ||b||."""
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)
