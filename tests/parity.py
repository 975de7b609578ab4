"""Helpers that compare the CUDA path's outputs with the FP64 oracle (test code only)."""
from __future__ import annotations

import numpy as np

CONVERGED = (1, 2, 3, 4)
# the accuracy bar for converged fits: centre to 1e-3 px, sigma / alpha / beta to 1e-4
XY_TOL, REL_TOL = 1e-3, 1e-4


def run_oracle(batch, **kw):
    import oracle
    from paper_2106_02045_gb300 import synth
    d = batch.numpy()
    return oracle.fit_spots(synth.as_numpy_images(batch), d["offsets"], d["dims"], d["init"],
                            d["model"], **kw)


def to_numpy(out: dict) -> dict:
    return {k: v.detach().cpu().numpy() for k, v in out.items()}


def well_posed(ref: dict, dims: np.ndarray) -> np.ndarray:
    """Spots whose FP64 fit is a meaningful estimate: converged, positive amplitude, no
    parameter held at the limit() box, peak amplitude above the residual noise."""
    p = ref["params"]
    W = dims[:, 0].astype(np.float64)
    H = dims[:, 1].astype(np.float64)
    smax = np.maximum(W, H)
    eps = 1e-6
    inside = ((p[:, 0] > -0.5 + eps) & (p[:, 0] < W - 0.5 - eps) & (p[:, 1] > -0.5 + eps) &
              (p[:, 1] < H - 0.5 - eps) & (p[:, 2] > 0.25 + eps) & (p[:, 2] < smax - eps) &
              (p[:, 3] > 0.25 + eps) & (p[:, 3] < smax - eps))
    conv = np.isin(ref["state"], CONVERGED)
    snr = ref["alpha"] / np.sqrt(np.maximum(ref["chi2"], 1e-30))
    return conv & inside & (ref["alpha"] > 0) & (snr >= 1.0)


def fisher_se(batch, ref: dict) -> np.ndarray:
    """Standard errors of (x0, y0, sigma_x, sigma_y) of each FP64 fit from the oracle's
    normal matrix at the fitted point: sqrt(chi2_n * diag((J^T J)^-1)); inf if undefined."""
    import oracle
    from paper_2106_02045_gb300 import synth
    img = synth.as_numpy_images(batch)
    offs, dims, model = batch.offsets.numpy(), batch.dims.numpy(), batch.model.numpy()
    se = np.full((batch.n, 4), np.inf)
    for s in np.nonzero(np.isin(ref["state"], CONVERGED))[0]:
        W, H = int(dims[s, 0]), int(dims[s, 1])
        m = int(model[s])
        g = img[offs[s]:offs[s] + W * H].astype(np.float64)
        ev = oracle.evaluate(m, W, H, g, ref["params"][s])
        if ev is None:
            continue
        try:
            ai = np.linalg.inv(ev["A"])
        except np.linalg.LinAlgError:
            continue
        d = np.sqrt(np.maximum(ref["chi2"][s] * np.diag(ai), 0.0))
        se[s, :len(d)] = d
        if m == 0:
            se[s, 3] = d[2]
    return se


def determined(batch, ref: dict, se_px: float = 0.1, se_rel: float = 0.1) -> np.ndarray:
    """Well-posed spots whose FP64 fit is statistically determined: centre standard error
    <= se_px pixels and width standard error <= se_rel of the width. Elsewhere the chi^2
    surface is so flat that the stop rule leaves rounding-sensitive end points."""
    se = fisher_se(batch, ref)
    rel = se[:, 2:] / np.abs(ref["params"][:, 2:])
    return (well_posed(ref, batch.dims.numpy()) & (se[:, 0] <= se_px) & (se[:, 1] <= se_px) &
            (rel.max(axis=1) <= se_rel))


def compare(out: dict, ref: dict, dims: np.ndarray, det: np.ndarray | None = None) -> dict:
    """Per-spot agreement metrics (out: numpy dict from the GPU, ref: oracle dict)."""
    st, rs = out["state"], ref["state"]
    conv, rconv = np.isin(st, CONVERGED), np.isin(rs, CONVERGED)
    both = conv & rconv
    P, RP = out["params"].astype(np.float64), ref["params"]
    dxy = np.abs(P[:, :2] - RP[:, :2]).max(1)
    ds = (np.abs(P[:, 2:] - RP[:, 2:]) / np.abs(RP[:, 2:])).max(1)
    da = np.abs(out["alpha"] - ref["alpha"]) / np.abs(ref["alpha"])
    db = np.abs(out["beta"] - ref["beta"]) / np.abs(ref["beta"])
    ok = (dxy < XY_TOL) & (ds < REL_TOL) & (da < REL_TOL) & (db < REL_TOL)
    wp = well_posed(ref, dims) if det is None else det
    res = dict(n=len(st), class_agree=float(np.mean(conv == rconv)),
               state_agree=float(np.mean(st == rs)),
               bar_converged=float(ok[both].mean()) if both.any() else 1.0,
               n_well_posed=int(wp.sum()),
               class_agree_wp=float(np.mean((conv == rconv)[wp])) if wp.any() else 1.0,
               bar_wp=float(ok[wp & both].mean()) if (wp & both).any() else 1.0,
               max_dxy_wp=float(dxy[wp & both].max()) if (wp & both).any() else 0.0)
    return res
