"""FP64 CPU oracle for implicit-amplitude Levenberg-Marquardt spot fitting.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the library itself never does.
The arithmetic lives in ``fitspots_oracle.c`` (plain C, double precision, one spot at a
time, OpenMP across spots); this module compiles it with gcc and marshals numpy arrays.

parity unpinned: the limit() box, the maxError default and the damping schedule's
constants are conventions or readings that no printed value pins (see the header of
``fitspots_oracle.c``); the normalised chi^2 divisor is pinned statistically (the unbiased
residual variance). The NO_DECREASE exit and the order of the stop
tests are pinned by the paper's stop-condition shares through a second build of the same
source with the paper's FP32 chi^2 (``paper_arithmetic=True``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "fitspots_oracle.c"
_LIB = _HERE / "_build" / "liboracle.so"
# the same source built with the paper's chi^2 arithmetic and minStep origin, for the pin
# of the stop conditions the paper reports (see the header of fitspots_oracle.c)
_LIB_PAPER = _HERE / "_build" / "liboracle_paper.so"
# the same source with the profile values rounded to FP32 and everything after them in FP64,
# to measure how far FP32 model values alone move a fit (see the header of fitspots_oracle.c)
_LIB_FP32_PROFILE = _HERE / "_build" / "liboracle_fp32profile.so"

MODEL_ISO, MODEL_ELLIPTIC = 0, 1
U16, F32, F64 = 0, 1, 2
STATE_NAMES = {0: "MAX_ITER", 1: "MIN_DELTA", 2: "MIN_STEP", 3: "MAX_ERROR",
               4: "NO_DECREASE", -1: "NOT_CONVERGED", -2: "INVALID"}

_libs = {}


def build(force: bool = False, paper_arithmetic: bool = False,
          fp32_profile: bool = False) -> Path:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, -O2, OpenMP); with
    ``paper_arithmetic`` the second build, ``liboracle_paper.so`` (-DOR_PAPER_ARITHMETIC);
    with ``fp32_profile`` the third, ``liboracle_fp32profile.so`` (-DOR_FP32_PROFILE)."""
    lib_path = _LIB_PAPER if paper_arithmetic else _LIB_FP32_PROFILE if fp32_profile else _LIB
    lib_path.parent.mkdir(exist_ok=True)
    if force or not lib_path.exists() or lib_path.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = lib_path.with_suffix(f".{os.getpid()}.tmp")
        defines = (["-DOR_PAPER_ARITHMETIC"] if paper_arithmetic else
                   ["-DOR_FP32_PROFILE"] if fp32_profile else [])
        subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", *defines,
                        "-o", str(tmp), str(_SRC), "-lm"], check=True)
        os.replace(tmp, lib_path)
    return lib_path


def _load(paper_arithmetic: bool = False, fp32_profile: bool = False):
    key = (paper_arithmetic, fp32_profile)
    if key not in _libs:
        lib = ctypes.CDLL(str(build(paper_arithmetic=paper_arithmetic, fp32_profile=fp32_profile)))
        d, i, i64, vp = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
        lib.or_fit_spots.argtypes = [vp, i, i64, vp, vp, vp, vp, i64, i, d, d, d,
                                     vp, vp, vp, vp, vp, vp, vp, vp, i]
        lib.or_fit_spots.restype = None
        lib.or_fit_spots_explicit.argtypes = [vp, i, i64, vp, vp, vp, vp, i64, i, d, d, d,
                                              vp, vp, vp, vp, vp, vp, vp, i]
        lib.or_fit_spots_explicit.restype = None
        lib.or_fit_spots_weighted.argtypes = [vp, i, i64, vp, vp, vp, vp, i64, i, d, d, d,
                                              vp, vp, vp, vp, vp, vp, vp, i, i]
        lib.or_fit_spots_weighted.restype = None
        lib.or_fit_spots_poisson.argtypes = [vp, i, i64, vp, vp, vp, vp, i64, i, d, d, d,
                                             vp, vp, vp, vp, vp, vp, vp, i]
        lib.or_fit_spots_poisson.restype = None
        lib.or_subtract_background.argtypes = [vp, i, i64, vp, vp, i64, i, vp, vp]
        lib.or_subtract_background.restype = None
        lib.or_poisson_amplitudes.argtypes = [i, vp, vp, vp, vp]
        lib.or_poisson_amplitudes.restype = i
        lib.or_evaluate.argtypes = [i, i, i, vp, vp, vp, vp, vp, vp, vp]
        lib.or_evaluate.restype = i
        lib.or_profile.argtypes = [i, i, i, vp, vp, vp]
        lib.or_profile.restype = None
        lib.or_amplitudes.argtypes = [i, vp, vp, vp, vp]
        lib.or_amplitudes.restype = i
        lib.or_jacobian.argtypes = [i, i, i, vp, vp, vp, vp, vp, vp, vp]
        lib.or_jacobian.restype = i
        lib.or_solve_damped.argtypes = [i, vp, vp, d, vp]
        lib.or_solve_damped.restype = i
        lib.or_limit.argtypes = [i, i, i, vp]
        lib.or_limit.restype = None
        lib.or_profile_second.argtypes = [i, i, i, vp, vp]
        lib.or_profile_second.restype = None
        lib.or_backward.argtypes = [i, i, i, vp, vp, d, d, vp, vp]
        lib.or_backward.restype = i
        _libs[key] = lib
    return _libs[key]


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def nparams(model: int) -> int:
    return 3 if model == MODEL_ISO else 4


def profile(model: int, W: int, H: int, p, with_derivs: bool = False):
    """f_i(p) (Eq. 10) and optionally df_i/dp_j (Eq. 11), shape (N,) and (P, N)."""
    lib = _load()
    pp = _f64(p)
    N = W * H
    f = np.empty(N)
    d = np.empty((nparams(model), N)) if with_derivs else None
    lib.or_profile(model, W, H, _p(pp), _p(f), _p(d) if d is not None else None)
    return (f, d) if with_derivs else f


def amplitudes(f, g):
    """alpha^, beta^ of Eq. 6 (None if undefined)."""
    lib = _load()
    f, g = _f64(f), _f64(g)
    a, b = ctypes.c_double(), ctypes.c_double()
    if lib.or_amplitudes(f.size, _p(f), _p(g), ctypes.byref(a), ctypes.byref(b)):
        return None
    return a.value, b.value


def jacobian(model: int, W: int, H: int, g, p):
    """Per-pixel J (P, N) = dh/dp with alpha^, beta^ and their derivatives (Eq. 8-9)."""
    lib = _load()
    g, pp = _f64(g), _f64(p)
    P = nparams(model)
    J = np.empty((P, W * H))
    da, db = np.empty(P), np.empty(P)
    a, b = ctypes.c_double(), ctypes.c_double()
    rc = lib.or_jacobian(model, W, H, _p(g), _p(pp), _p(J), ctypes.byref(a), ctypes.byref(b),
                         _p(da), _p(db))
    if rc:
        return None
    return J, a.value, b.value, da, db


def evaluate(model: int, W: int, H: int, g, p, with_normal: bool = True):
    """alpha^, beta^, chi^2 and (A = J^T J, b = J^T (g-h)) at p."""
    lib = _load()
    g, pp = _f64(g), _f64(p)
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    A = np.zeros(16)
    bb = np.zeros(4)
    rc = lib.or_evaluate(model, W, H, _p(g), _p(pp), ctypes.byref(a), ctypes.byref(b),
                         ctypes.byref(c), _p(A) if with_normal else None, _p(bb))
    if rc:
        return None
    P = nparams(model)
    out = dict(alpha=a.value, beta=b.value, chi2=c.value)
    if with_normal:
        out["A"] = A.reshape(4, 4)[:P, :P].copy()
        out["b"] = bb[:P].copy()
    return out


def solve_damped(A, b, lam: float):
    lib = _load()
    A = _f64(A)
    P = A.shape[0]
    A16 = np.zeros((4, 4))
    A16[:P, :P] = A
    A16 = A16.ravel().copy()
    bb = np.zeros(4)
    bb[:P] = _f64(b)
    delta = np.zeros(4)
    if lib.or_solve_damped(P, _p(A16), _p(bb), float(lam), _p(delta)):
        return None
    return delta[:P]


def limit(model: int, W: int, H: int, p):
    lib = _load()
    pp = _f64(p).copy()
    lib.or_limit(model, W, H, _p(pp))
    return pp


def fit_spots(images: np.ndarray, offsets, dims, init, model, *, max_iter: int = 20,
              max_error: float = 0.0, min_delta: float = 1e-6, min_step: float = 1e-4,
              trace: bool = False, nthreads: int = 0, paper_arithmetic: bool = False,
              fp32_profile: bool = False) -> dict:
    """Fit every spot in FP64. ``images`` is a flat uint16, float32 or float64 array.
    ``paper_arithmetic`` runs the second build (FP32 chi^2 over pixel threads, minStep
    relative to the ROI centre), used only to pin the paper's stop-condition shares;
    ``fp32_profile`` the third (profile values rounded to FP32), used only to measure how far
    FP32 model values alone move the fits."""
    lib = _load(paper_arithmetic, fp32_profile)
    images = np.ascontiguousarray(images)
    dtype = {np.dtype(np.uint16): U16, np.dtype(np.float32): F32,
             np.dtype(np.float64): F64}[images.dtype]
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    dims = np.ascontiguousarray(dims, dtype=np.int32).reshape(-1, 2)
    init = np.ascontiguousarray(init, dtype=np.float32).reshape(-1, 4)
    model = np.ascontiguousarray(model, dtype=np.uint8)
    n = offsets.size
    assert dims.shape[0] == n and init.shape[0] == n and model.size == n
    out = dict(params=np.empty((n, 4)), alpha=np.empty(n), beta=np.empty(n), chi2=np.empty(n),
               state=np.empty(n, np.int32), iters=np.empty(n, np.int32),
               evals=np.empty(n, np.int32))
    tr = np.empty((n, max_iter + 1)) if trace else None
    lib.or_fit_spots(_p(images), dtype, images.size, _p(offsets), _p(dims), _p(init), _p(model),
                     n, int(max_iter), float(max_error), float(min_delta), float(min_step),
                     _p(out["params"]), _p(out["alpha"]), _p(out["beta"]), _p(out["chi2"]),
                     _p(out["state"]), _p(out["iters"]), _p(out["evals"]),
                     _p(tr) if tr is not None else None, int(nthreads))
    if trace:
        out["trace"] = tr
    return out


def fit_spots_explicit(images: np.ndarray, offsets, dims, init, model, *, max_iter: int = 20,
                       max_error: float = 0.0, min_delta: float = 1e-6, min_step: float = 1e-4,
                       nthreads: int = 0) -> dict:
    """Plain LM over (shape, alpha, beta) in FP64, the explicit-amplitude comparison."""
    lib = _load()
    images = np.ascontiguousarray(images)
    dtype = {np.dtype(np.uint16): U16, np.dtype(np.float32): F32,
             np.dtype(np.float64): F64}[images.dtype]
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    dims = np.ascontiguousarray(dims, dtype=np.int32).reshape(-1, 2)
    init = np.ascontiguousarray(init, dtype=np.float32).reshape(-1, 4)
    model = np.ascontiguousarray(model, dtype=np.uint8)
    n = offsets.size
    out = dict(params=np.empty((n, 4)), alpha=np.empty(n), beta=np.empty(n), chi2=np.empty(n),
               state=np.empty(n, np.int32), iters=np.empty(n, np.int32),
               evals=np.empty(n, np.int32))
    lib.or_fit_spots_explicit(_p(images), dtype, images.size, _p(offsets), _p(dims), _p(init),
                              _p(model), n, int(max_iter), float(max_error), float(min_delta),
                              float(min_step), _p(out["params"]), _p(out["alpha"]),
                              _p(out["beta"]), _p(out["chi2"]), _p(out["state"]),
                              _p(out["iters"]), _p(out["evals"]), int(nthreads))
    return out


def fit_spots_weighted(images: np.ndarray, offsets, dims, init, model, *, max_iter: int = 20,
                       max_error: float = 0.0, min_delta: float = 1e-6, min_step: float = 1e-4,
                       unit_weights: bool = False, nthreads: int = 0) -> dict:
    """The variance-weighted implicit-amplitude fit (weights 1 / max(g, 1), or all 1)."""
    lib = _load()
    images = np.ascontiguousarray(images)
    dtype = {np.dtype(np.uint16): U16, np.dtype(np.float32): F32,
             np.dtype(np.float64): F64}[images.dtype]
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    dims = np.ascontiguousarray(dims, dtype=np.int32).reshape(-1, 2)
    init = np.ascontiguousarray(init, dtype=np.float32).reshape(-1, 4)
    model = np.ascontiguousarray(model, dtype=np.uint8)
    n = offsets.size
    out = dict(params=np.empty((n, 4)), alpha=np.empty(n), beta=np.empty(n), chi2=np.empty(n),
               state=np.empty(n, np.int32), iters=np.empty(n, np.int32),
               evals=np.empty(n, np.int32))
    lib.or_fit_spots_weighted(_p(images), dtype, images.size, _p(offsets), _p(dims), _p(init),
                              _p(model), n, int(max_iter), float(max_error), float(min_delta),
                              float(min_step), _p(out["params"]), _p(out["alpha"]),
                              _p(out["beta"]), _p(out["chi2"]), _p(out["state"]),
                              _p(out["iters"]), _p(out["evals"]), int(unit_weights), int(nthreads))
    return out


def subtract_background(images: np.ndarray, offsets, dims, border: int = 1):
    """Tilt of the least-squares plane on each ROI's border ring subtracted: (images as
    float64, untouched outside the ROIs as NaN; plane [n, 3] = c0, cx, cy)."""
    lib = _load()
    images = np.ascontiguousarray(images)
    dtype = {np.dtype(np.uint16): U16, np.dtype(np.float32): F32,
             np.dtype(np.float64): F64}[images.dtype]
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    dims = np.ascontiguousarray(dims, dtype=np.int32).reshape(-1, 2)
    n = offsets.size
    out = np.full(images.size, np.nan)
    plane = np.empty((n, 3))
    lib.or_subtract_background(_p(images), dtype, images.size, _p(offsets), _p(dims), n,
                               int(border), _p(out), _p(plane))
    return out, plane


def poisson_amplitudes(f, g):
    """Poisson maximum-likelihood alpha, beta for the profile f (None if none is found)."""
    lib = _load()
    f, g = _f64(f), _f64(g)
    a, b = ctypes.c_double(), ctypes.c_double()
    if lib.or_poisson_amplitudes(f.size, _p(f), _p(g), ctypes.byref(a), ctypes.byref(b)):
        return None
    return a.value, b.value


def fit_spots_poisson(images: np.ndarray, offsets, dims, init, model, *, max_iter: int = 20,
                      max_error: float = 0.0, min_delta: float = 1e-6, min_step: float = 1e-4,
                      nthreads: int = 0) -> dict:
    """The Poisson-likelihood implicit-amplitude fit (deviance objective); "chi2" is the
    deviance over N - P - 2."""
    lib = _load()
    images = np.ascontiguousarray(images)
    dtype = {np.dtype(np.uint16): U16, np.dtype(np.float32): F32,
             np.dtype(np.float64): F64}[images.dtype]
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    dims = np.ascontiguousarray(dims, dtype=np.int32).reshape(-1, 2)
    init = np.ascontiguousarray(init, dtype=np.float32).reshape(-1, 4)
    model = np.ascontiguousarray(model, dtype=np.uint8)
    n = offsets.size
    out = dict(params=np.empty((n, 4)), alpha=np.empty(n), beta=np.empty(n), chi2=np.empty(n),
               state=np.empty(n, np.int32), iters=np.empty(n, np.int32),
               evals=np.empty(n, np.int32))
    lib.or_fit_spots_poisson(_p(images), dtype, images.size, _p(offsets), _p(dims), _p(init),
                             _p(model), n, int(max_iter), float(max_error), float(min_delta),
                             float(min_step), _p(out["params"]), _p(out["alpha"]),
                             _p(out["beta"]), _p(out["chi2"]), _p(out["state"]),
                             _p(out["iters"]), _p(out["evals"]), int(nthreads))
    return out


def profile_second(model: int, W: int, H: int, p):
    """d^2 f_i / dp_j dp_k, shape (P, P, N)."""
    lib = _load()
    pp = _f64(p)
    P, N = nparams(model), W * H
    d2 = np.empty((P, P, N))
    lib.or_profile_second(model, W, H, _p(pp), _p(d2))
    return d2


def backward(model: int, W: int, H: int, g, p, alpha: float, beta: float, upstream):
    """Implicit-function-theorem VJP of one fit: d loss / d g (N values), or None."""
    lib = _load()
    g, pp, up = _f64(g), _f64(p), _f64(upstream)
    assert up.size == 7
    out = np.empty(W * H)
    if lib.or_backward(model, W, H, _p(g), _p(pp), float(alpha), float(beta), _p(up), _p(out)):
        return None
    return out
