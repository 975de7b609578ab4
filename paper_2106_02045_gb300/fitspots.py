"""Thin Python binding of ``include/fitspots.h`` (ctypes; argument marshalling only).

Every step of the fit runs in the CUDA library ``_build/libfitspots.so``. PyTorch only
provides device memory and the stream. There is no CPU fallback: if the library is not
built, or a tensor is not on a CUDA device, the call raises.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

import torch

from .build import LIB

MODEL_ISO, MODEL_ELLIPTIC = 0, 1
U16, F32 = 0, 1
STATE = {"MAX_ITER": 0, "MIN_DELTA": 1, "MIN_STEP": 2, "MAX_ERROR": 3, "NO_DECREASE": 4,
         "NOT_CONVERGED": -1, "INVALID_ROI": -2}
CONVERGED_STATES = (1, 2, 3, 4)
# largest spot count per call (FS_MAX_SPOTS of the C header: 2^31 - 2^24, headroom for the
# kernels' 32-bit work counters)
MAX_SPOTS = 2_130_706_432


class FitSpotsError(RuntimeError):
    pass


def _check_count(n: int) -> None:
    if n > MAX_SPOTS:
        raise FitSpotsError(f"{n} spots in one call; at most {MAX_SPOTS} (split the batch)")


_lib = None


def library() -> ctypes.CDLL:
    """The loaded C library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not Path(LIB).exists():
            raise FitSpotsError(f"{LIB} is missing: build it with __graft_entry__.build()")
        lib = ctypes.CDLL(str(LIB))
        vp, i, i64, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
        lib.fit_spots.argtypes = [vp, i, i64, vp, vp, vp, vp, i64, i, d, d, d,
                                  vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]
        lib.fit_spots.restype = i
        lib.fit_spots_per_class.argtypes = lib.fit_spots.argtypes
        lib.fit_spots_per_class.restype = i
        lib.fit_spots_uniform.argtypes = [vp, i, i, i, i, vp, i64, i, d, d, d,
                                          vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]
        lib.fit_spots_uniform.restype = i
        lib.fit_spots_explicit.argtypes = [vp, i, i64, vp, vp, vp, vp, i64, i, d, d, d,
                                           vp, vp, vp, vp, vp, vp, vp, vp]
        lib.fit_spots_explicit.restype = i
        lib.fit_spots_weighted.argtypes = lib.fit_spots_explicit.argtypes
        lib.fit_spots_weighted.restype = i
        lib.fit_spots_poisson.argtypes = lib.fit_spots_explicit.argtypes
        lib.fit_spots_poisson.restype = i
        lib.fit_spots_subtract_background.argtypes = [vp, i, i64, vp, vp, i64, i, vp, vp, vp]
        lib.fit_spots_subtract_background.restype = i
        lib.fit_spots_start.argtypes = [vp, i, i64, vp, vp, i64, i, vp, vp]
        lib.fit_spots_start.restype = i
        lib.fit_spots_uniform_host.argtypes = [vp, i, i, i, i, vp, i64, i, d, d, d,
                                               vp, vp, vp, vp, vp, vp, vp, i64, vp, sz, vp]
        lib.fit_spots_uniform_host.restype = i
        lib.fit_spots_noalloc.argtypes = [vp, i, i64, vp, vp, vp, vp, i64, i, d, d, d,
                                          vp, vp, vp, vp, vp, vp, vp, vp]
        lib.fit_spots_noalloc.restype = i
        lib.fit_spots_noalloc_max_spots.argtypes = []
        lib.fit_spots_noalloc_max_spots.restype = i64
        lib.fit_spots_uniform_host_workspace.argtypes = [i64, i, i, i]
        lib.fit_spots_uniform_host_workspace.restype = sz
        lib.fit_spots_uniform_workspace.argtypes = []
        lib.fit_spots_uniform_workspace.restype = sz
        lib.fit_spots_default_config.argtypes = [i]
        lib.fit_spots_default_config.restype = i
        lib.fit_spots_config_batched.argtypes = [i]
        lib.fit_spots_config_batched.restype = i
        lib.fit_spots_probe_scratch_bytes.argtypes = [i]
        lib.fit_spots_probe_scratch_bytes.restype = sz
        lib.fit_spots_probe_rates.argtypes = [i, vp, sz, ctypes.POINTER(d), ctypes.POINTER(d),
                                              ctypes.POINTER(d), vp]
        lib.fit_spots_probe_rates.restype = i
        lib.fit_spots_config_generic.argtypes = [i]
        lib.fit_spots_config_generic.restype = i
        lib.fit_spots_config_fits.argtypes = [i, i]
        lib.fit_spots_config_fits.restype = i
        lib.fit_spots_backward.argtypes = [vp, i, i64, vp, vp, vp, i64, vp, vp, vp, vp,
                                           vp, vp, vp, vp, vp, vp]
        lib.fit_spots_backward.restype = i
        lib.fit_spots_workspace.argtypes = [i64]
        lib.fit_spots_workspace.restype = sz
        lib.fit_spots_strerror.argtypes = [i]
        lib.fit_spots_strerror.restype = ctypes.c_char_p
        lib.fit_spots_last_cuda_error.argtypes = []
        lib.fit_spots_last_cuda_error.restype = i
        lib.fit_spots_num_classes.restype = i
        lib.fit_spots_num_configs.restype = i
        lib.fit_spots_config_info.argtypes = [i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]
        lib.fit_spots_config_info.restype = i
        lib.fit_spots_get_config.argtypes = [i]
        lib.fit_spots_get_config.restype = i
        lib.fit_spots_set_config.argtypes = [i, i]
        lib.fit_spots_set_config.restype = i
        _lib = lib
    return _lib


def check(rc: int, what: str = "fit_spots") -> None:
    if rc != 0:
        lib = library()
        msg = lib.fit_spots_strerror(rc).decode()
        if rc == -7:
            msg += f" (cudaError {lib.fit_spots_last_cuda_error()})"
        raise FitSpotsError(f"{what} failed: {msg} [{rc}]")


def _ptr(t: torch.Tensor | None):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _need(t: torch.Tensor, dtype, name: str, device) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
        raise FitSpotsError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise FitSpotsError(f"{name} must be {dtype}, got {t.dtype}")
    if t.device != device:
        raise FitSpotsError(f"{name} is on {t.device}, expected {device}")
    if not t.is_contiguous():
        raise FitSpotsError(f"{name} must be contiguous")
    return t


def workspace_bytes(n: int) -> int:
    return int(library().fit_spots_workspace(int(n)))


def uniform_workspace_bytes() -> int:
    return int(library().fit_spots_uniform_workspace())


def alloc_outputs(n: int, device) -> dict:
    return dict(params=torch.empty((n, 4), dtype=torch.float32, device=device),
                alpha=torch.empty(n, dtype=torch.float32, device=device),
                beta=torch.empty(n, dtype=torch.float32, device=device),
                chi2=torch.empty(n, dtype=torch.float32, device=device),
                state=torch.empty(n, dtype=torch.int32, device=device),
                iters=torch.empty(n, dtype=torch.int32, device=device),
                evals=torch.empty(n, dtype=torch.int32, device=device))


def fit(images: torch.Tensor, offsets: torch.Tensor, dims: torch.Tensor, init: torch.Tensor,
        model: torch.Tensor, *, max_iter: int = 20, max_error: float = 0.0,
        min_delta: float = 1e-6, min_step: float = 1e-4, out: dict | None = None,
        workspace: torch.Tensor | None = None, stream: torch.cuda.Stream | None = None,
        per_class: bool = False) -> dict:
    """Fit all spots; returns (or fills ``out``) params [n,4], alpha, beta, chi2 (normalised),
    state, iters, evals. Asynchronous on ``stream`` (default: the current stream).
    ``per_class`` runs fit_spots_per_class (one persistent launch per size class, each with
    its configured kernel) instead of the single generic launch of fit_spots."""
    dev = images.device
    if dev.type != "cuda":
        raise FitSpotsError("images must be a CUDA tensor")
    if images.dtype == torch.uint16:
        dtype = U16
    elif images.dtype == torch.float32:
        dtype = F32
    else:
        raise FitSpotsError(f"images must be uint16 or float32, got {images.dtype}")
    _need(images, images.dtype, "images", dev)
    n = int(offsets.numel())
    _check_count(n)
    _need(offsets, torch.int64, "offsets", dev)
    _need(dims, torch.int32, "dims", dev)
    _need(init, torch.float32, "init", dev)
    _need(model, torch.uint8, "model", dev)
    if dims.numel() != 2 * n or init.numel() != 4 * n or model.numel() != n:
        raise FitSpotsError("offsets, dims, init and model disagree on the spot count")
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    # temporaries and outputs are allocated on the launch stream, so that the caching
    # allocator never reuses their memory while the kernels may still run
    with torch.cuda.device(dev), torch.cuda.stream(s):
        o = out if out is not None else alloc_outputs(n, dev)
        if workspace is None:
            workspace = torch.empty(max(workspace_bytes(n), 16), dtype=torch.uint8, device=dev)
        fn = library().fit_spots_per_class if per_class else library().fit_spots
        rc = fn(
            _ptr(images), dtype, images.numel(), _ptr(offsets), _ptr(dims), _ptr(init), _ptr(model),
            n, int(max_iter), float(max_error), float(min_delta), float(min_step),
            _ptr(o["params"]), _ptr(o["alpha"]), _ptr(o["beta"]), _ptr(o["chi2"]), _ptr(o["state"]),
            _ptr(o["iters"]), _ptr(o.get("evals")), _ptr(workspace), workspace.numel(),
            ctypes.c_void_p(s.cuda_stream))
    check(rc)
    return o


def fit_uniform(images: torch.Tensor, width: int, height: int, model: int, init: torch.Tensor, *,
                max_iter: int = 20, max_error: float = 0.0, min_delta: float = 1e-6,
                min_step: float = 1e-4, out: dict | None = None,
                workspace: torch.Tensor | None = None,
                stream: torch.cuda.Stream | None = None) -> dict:
    """Fit n spots of one size and model stored back to back (spot s at s*W*H)."""
    dev = images.device
    if dev.type != "cuda":
        raise FitSpotsError("images must be a CUDA tensor")
    if images.dtype == torch.uint16:
        dtype = U16
    elif images.dtype == torch.float32:
        dtype = F32
    else:
        raise FitSpotsError(f"images must be uint16 or float32, got {images.dtype}")
    _need(images, images.dtype, "images", dev)
    _need(init, torch.float32, "init", dev)
    n = init.numel() // 4
    _check_count(n)
    if init.numel() != 4 * n or images.numel() < n * width * height:
        raise FitSpotsError("init must be [n, 4] and images must hold n*W*H elements")
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    with torch.cuda.device(dev), torch.cuda.stream(s):
        o = out if out is not None else alloc_outputs(n, dev)
        if workspace is None:
            workspace = torch.empty(max(int(library().fit_spots_uniform_workspace()), 16),
                                    dtype=torch.uint8, device=dev)
        rc = library().fit_spots_uniform(
            _ptr(images), dtype, int(width), int(height), int(model), _ptr(init), n,
            int(max_iter), float(max_error), float(min_delta), float(min_step),
            _ptr(o["params"]), _ptr(o["alpha"]), _ptr(o["beta"]), _ptr(o["chi2"]), _ptr(o["state"]),
            _ptr(o["iters"]), _ptr(o.get("evals")), _ptr(workspace), workspace.numel(),
            ctypes.c_void_p(s.cuda_stream))
    check(rc, "fit_spots_uniform")
    return o


def alloc_host_outputs(n: int) -> dict:
    """Pinned host buffers for the outputs of ``fit_uniform_host``."""
    return {k: torch.empty(v, dtype=t, pin_memory=True) for k, (v, t) in dict(
        params=((n, 4), torch.float32), alpha=(n, torch.float32), beta=(n, torch.float32),
        chi2=(n, torch.float32), state=(n, torch.int32), iters=(n, torch.int32),
        evals=(n, torch.int32)).items()}


def host_workspace_bytes(chunk: int, width: int, height: int, dtype: int) -> int:
    return int(library().fit_spots_uniform_host_workspace(int(chunk), int(width), int(height),
                                                          int(dtype)))


def fit_uniform_host(images: torch.Tensor, width: int, height: int, model: int,
                     init: torch.Tensor, *, chunk: int = 131072, max_iter: int = 20,
                     max_error: float = 0.0, min_delta: float = 1e-6, min_step: float = 1e-4,
                     out: dict | None = None, workspace: torch.Tensor | None = None,
                     device=None, stream: torch.cuda.Stream | None = None) -> dict:
    """``fit_uniform`` on HOST tensors (pinned for overlap): chunks of ``chunk`` spots are
    copied up, fitted and copied back with the copies overlapping the fits. Returns (or
    fills ``out``) host tensors, valid once ``stream`` has completed."""
    if images.device.type != "cpu" or init.device.type != "cpu":
        raise FitSpotsError("images and init must be host (CPU) tensors")
    if images.dtype == torch.uint16:
        dtype = U16
    elif images.dtype == torch.float32:
        dtype = F32
    else:
        raise FitSpotsError(f"images must be uint16 or float32, got {images.dtype}")
    if init.dtype != torch.float32 or not init.is_contiguous() or not images.is_contiguous():
        raise FitSpotsError("images and init must be contiguous; init float32")
    n = init.numel() // 4
    _check_count(n)
    if init.numel() != 4 * n or images.numel() < n * width * height:
        raise FitSpotsError("init must be [n, 4] and images must hold n*W*H elements")
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    o = out if out is not None else alloc_host_outputs(n)
    for k, t in o.items():
        if t is not None and t.device.type != "cpu":
            raise FitSpotsError(f"out[{k!r}] must be a host tensor")
    need = host_workspace_bytes(min(chunk, max(n, 1)), width, height, dtype)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    with torch.cuda.device(dev), torch.cuda.stream(s):
        if workspace is None:
            workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
        rc = library().fit_spots_uniform_host(
            _ptr(images), dtype, int(width), int(height), int(model), _ptr(init), n,
            int(max_iter), float(max_error), float(min_delta), float(min_step),
            _ptr(o["params"]), _ptr(o["alpha"]), _ptr(o["beta"]), _ptr(o["chi2"]), _ptr(o["state"]),
            _ptr(o["iters"]), _ptr(o.get("evals")), int(chunk), _ptr(workspace),
            workspace.numel(), ctypes.c_void_p(s.cuda_stream))
    check(rc, "fit_spots_uniform_host")
    return o


def fit_explicit(images: torch.Tensor, offsets: torch.Tensor, dims: torch.Tensor,
                 init: torch.Tensor, model: torch.Tensor, *, max_iter: int = 20,
                 max_error: float = 0.0, min_delta: float = 1e-6, min_step: float = 1e-4,
                 out: dict | None = None, stream: torch.cuda.Stream | None = None,
                 _entry: str = "fit_spots_explicit") -> dict:
    """The explicit-amplitude LM (comparison method), same arguments and outputs as fit."""
    dev = images.device
    if dev.type != "cuda":
        raise FitSpotsError("images must be a CUDA tensor")
    dtype = U16 if images.dtype == torch.uint16 else F32 if images.dtype == torch.float32 else None
    if dtype is None:
        raise FitSpotsError(f"images must be uint16 or float32, got {images.dtype}")
    _need(offsets, torch.int64, "offsets", dev)
    _need(dims, torch.int32, "dims", dev)
    _need(init, torch.float32, "init", dev)
    _need(model, torch.uint8, "model", dev)
    n = offsets.numel()
    _check_count(n)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    with torch.cuda.device(dev), torch.cuda.stream(s):
        o = out if out is not None else alloc_outputs(n, dev)
        rc = getattr(library(), _entry)(
            _ptr(images), dtype, images.numel(), _ptr(offsets), _ptr(dims), _ptr(init),
            _ptr(model), n, int(max_iter), float(max_error), float(min_delta), float(min_step),
            _ptr(o["params"]), _ptr(o["alpha"]), _ptr(o["beta"]), _ptr(o["chi2"]), _ptr(o["state"]),
            _ptr(o["iters"]), _ptr(o.get("evals")), ctypes.c_void_p(s.cuda_stream))
    check(rc, _entry)
    return o


def fit_weighted(images: torch.Tensor, offsets: torch.Tensor, dims: torch.Tensor,
                 init: torch.Tensor, model: torch.Tensor, **kw) -> dict:
    """The variance-weighted implicit-amplitude fit (weights 1 / max(g, 1)); same arguments
    and outputs as fit (chi2 is the weighted one)."""
    return fit_explicit(images, offsets, dims, init, model, _entry="fit_spots_weighted", **kw)


def fit_poisson(images: torch.Tensor, offsets: torch.Tensor, dims: torch.Tensor,
                init: torch.Tensor, model: torch.Tensor, **kw) -> dict:
    """The Poisson-likelihood implicit-amplitude fit (deviance objective, amplitudes at their
    likelihood optimum); same arguments and outputs as fit ("chi2" is the deviance over
    N - P - 2)."""
    return fit_explicit(images, offsets, dims, init, model, _entry="fit_spots_poisson", **kw)


START_CENTROID, START_PAPER = 0, 1


def start_values(images: torch.Tensor, offsets: torch.Tensor, dims: torch.Tensor,
                 rule: int = START_CENTROID, *, out: torch.Tensor | None = None,
                 stream: torch.cuda.Stream | None = None) -> torch.Tensor:
    """Start values [n, 4] (x0, y0, s0, s0) from each ROI's pixels, on the device."""
    dev = images.device
    if dev.type != "cuda":
        raise FitSpotsError("images must be a CUDA tensor")
    dtype = U16 if images.dtype == torch.uint16 else F32 if images.dtype == torch.float32 else None
    if dtype is None:
        raise FitSpotsError(f"images must be uint16 or float32, got {images.dtype}")
    _need(images, images.dtype, "images", dev)
    _need(offsets, torch.int64, "offsets", dev)
    _need(dims, torch.int32, "dims", dev)
    n = offsets.numel()
    _check_count(n)
    if dims.numel() != 2 * n:
        raise FitSpotsError("dims must be [n, 2]")
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    with torch.cuda.device(dev), torch.cuda.stream(s):
        o = out if out is not None else torch.empty((n, 4), dtype=torch.float32, device=dev)
        _need(o, torch.float32, "out", dev)
        rc = library().fit_spots_start(_ptr(images), dtype, images.numel(), _ptr(offsets),
                                       _ptr(dims), n, int(rule), _ptr(o),
                                       ctypes.c_void_p(s.cuda_stream))
    check(rc, "fit_spots_start")
    return o


def subtract_background(images: torch.Tensor, offsets: torch.Tensor, dims: torch.Tensor,
                        border: int = 1, *, out: torch.Tensor | None = None,
                        plane: torch.Tensor | None = None,
                        stream: torch.cuda.Stream | None = None):
    """Each ROI minus the tilt of the least-squares plane on its border ring
    (fit_spots_subtract_background): (float32 images of the same layout, plane [n, 3] =
    c0, cx, cy). Elements outside the ROIs of a freshly allocated output are 0."""
    dev = images.device
    if dev.type != "cuda":
        raise FitSpotsError("images must be a CUDA tensor")
    dtype = U16 if images.dtype == torch.uint16 else F32 if images.dtype == torch.float32 else None
    if dtype is None:
        raise FitSpotsError(f"images must be uint16 or float32, got {images.dtype}")
    _need(images, images.dtype, "images", dev)
    _need(offsets, torch.int64, "offsets", dev)
    _need(dims, torch.int32, "dims", dev)
    n = offsets.numel()
    _check_count(n)
    if dims.numel() != 2 * n:
        raise FitSpotsError("dims must be [n, 2]")
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    with torch.cuda.device(dev), torch.cuda.stream(s):
        o = out if out is not None else torch.zeros(images.numel(), dtype=torch.float32, device=dev)
        pl = plane if plane is not None else torch.empty((n, 3), dtype=torch.float32, device=dev)
        _need(o, torch.float32, "out", dev)
        _need(pl, torch.float32, "plane", dev)
        if o.numel() < images.numel() or pl.numel() < 3 * n:
            raise FitSpotsError("out or plane too small")
        rc = library().fit_spots_subtract_background(
            _ptr(images), dtype, images.numel(), _ptr(offsets), _ptr(dims), n, int(border),
            _ptr(o), _ptr(pl), ctypes.c_void_p(s.cuda_stream))
    check(rc, "fit_spots_subtract_background")
    return o, pl


def fit_batch(batch, **kw) -> dict:
    """``fit`` on a :class:`synth.SpotBatch` living on a CUDA device."""
    return fit(batch.images, batch.offsets, batch.dims, batch.init, batch.model, **kw)


def configs() -> list[tuple[int, int, int, int]]:
    """(lanes, cols, rows, batched) of every compiled configuration, by id."""
    lib = library()
    out = []
    for c in range(lib.fit_spots_num_configs()):
        L, C, R = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(lib.fit_spots_config_info(c, ctypes.byref(L), ctypes.byref(C), ctypes.byref(R)),
              "fit_spots_config_info")
        b = lib.fit_spots_config_batched(c)
        check(min(b, 0), "fit_spots_config_batched")
        out.append((L.value, C.value, R.value, b))
    return out


def get_config(size_class: int) -> int:
    return int(library().fit_spots_get_config(int(size_class)))


def default_config(size_class: int) -> int:
    """The library's built-in configuration for a size class."""
    c = int(library().fit_spots_default_config(int(size_class)))
    check(min(c, 0), "fit_spots_default_config")
    return c


def config_generic(config: int) -> bool:
    """Whether ``config`` is the generic configuration (fit_spots' single launch)."""
    c = int(library().fit_spots_config_generic(int(config)))
    check(min(c, 0), "fit_spots_config_generic")
    return bool(c)


def probe_rates(device="cuda:0") -> dict:
    """Measured lane-operations per second of FP32 FMA, MUFU exp2 and FP64 FMA on ``device``
    (the roofline denominators of the fit kernels); see fit_spots_probe_rates."""
    dev = torch.device(device)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    lib = library()
    scratch = torch.empty(int(lib.fit_spots_probe_scratch_bytes(sms)), dtype=torch.uint8, device=dev)
    f, e, dd = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    s = torch.cuda.current_stream(dev)
    check(lib.fit_spots_probe_rates(sms, _ptr(scratch), scratch.numel(), ctypes.byref(f),
                                    ctypes.byref(e), ctypes.byref(dd), ctypes.c_void_p(s.cuda_stream)),
          "fit_spots_probe_rates")
    return {"ffma": f.value, "ex2": e.value, "dfma": dd.value, "sms": sms}


def num_classes() -> int:
    return int(library().fit_spots_num_classes())


def config_fits(size_class: int, config: int) -> bool:
    return bool(library().fit_spots_config_fits(int(size_class), int(config)))


def set_config(size_class: int, config: int) -> None:
    check(library().fit_spots_set_config(int(size_class), int(config)), "fit_spots_set_config")


def backward(images: torch.Tensor, offsets: torch.Tensor, dims: torch.Tensor,
             model: torch.Tensor, fit_out: dict, grad_params=None, grad_alpha=None,
             grad_beta=None, grad_chi2=None, grad_images: torch.Tensor | None = None,
             stream: torch.cuda.Stream | None = None) -> torch.Tensor:
    """d loss / d images for upstream gradients of a fit (implicit-function theorem)."""
    dev = images.device
    if dev.type != "cuda":
        raise FitSpotsError("images must be a CUDA tensor")
    dtype = U16 if images.dtype == torch.uint16 else F32 if images.dtype == torch.float32 else None
    if dtype is None:
        raise FitSpotsError(f"images must be uint16 or float32, got {images.dtype}")
    _need(images, images.dtype, "images", dev)
    _need(offsets, torch.int64, "offsets", dev)
    _need(dims, torch.int32, "dims", dev)
    _need(model, torch.uint8, "model", dev)
    n = int(offsets.numel())
    _check_count(n)
    if dims.numel() != 2 * n or model.numel() != n:
        raise FitSpotsError("offsets, dims and model disagree on the spot count")
    for k, t, m in (("params", torch.float32, 4 * n), ("alpha", torch.float32, n),
                    ("beta", torch.float32, n), ("state", torch.int32, n)):
        _need(fit_out[k], t, f"fit_out[{k!r}]", dev)
        if fit_out[k].numel() != m:
            raise FitSpotsError(f"fit_out[{k!r}] has the wrong size")
    if grad_images is not None:
        _need(grad_images, torch.float32, "grad_images", dev)
        if grad_images.numel() != images.numel():
            raise FitSpotsError("grad_images must have as many elements as images")

    def opt(t, shape):
        if t is None:
            return None
        t = t.to(device=dev, dtype=torch.float32).contiguous()
        if t.numel() != shape:
            raise FitSpotsError("upstream gradient has the wrong size")
        return t
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    # conversions and the zeroed output are made on the launch stream: ordered before the
    # kernel, and their memory is not reused while it runs
    with torch.cuda.device(dev), torch.cuda.stream(s):
        if grad_images is None:
            grad_images = torch.zeros(images.numel(), dtype=torch.float32, device=dev)
        gp, ga = opt(grad_params, 4 * n), opt(grad_alpha, n)
        gb, gc = opt(grad_beta, n), opt(grad_chi2, n)
        rc = library().fit_spots_backward(
            _ptr(images), dtype, images.numel(), _ptr(offsets), _ptr(dims), _ptr(model), n,
            _ptr(fit_out["params"]), _ptr(fit_out["alpha"]), _ptr(fit_out["beta"]),
            _ptr(fit_out["state"]), _ptr(gp), _ptr(ga), _ptr(gb), _ptr(gc), _ptr(grad_images),
            ctypes.c_void_p(s.cuda_stream))
    check(rc, "fit_spots_backward")
    return grad_images


class FitSpotsFunction(torch.autograd.Function):
    """Differentiable batched fit: (images, init) -> (params, alpha, beta, chi2).

    The backward pass is the implicit-function-theorem kernel; the gradient with respect
    to the start parameters is zero (the minimum does not depend on where the search
    started). state and iters are returned as non-differentiable tensors."""

    @staticmethod
    def forward(ctx, images, init, offsets, dims, model, max_iter=20, max_error=0.0,
                min_delta=1e-6, min_step=1e-4):
        out = fit(images.detach(), offsets, dims, init.detach().contiguous(), model,
                  max_iter=max_iter, max_error=max_error, min_delta=min_delta,
                  min_step=min_step)
        ctx.save_for_backward(images.detach(), offsets, dims, model, out["params"], out["alpha"],
                              out["beta"], out["state"])
        ctx.init_shape = init.shape
        ctx.mark_non_differentiable(out["state"], out["iters"])
        return out["params"], out["alpha"], out["beta"], out["chi2"], out["state"], out["iters"]

    @staticmethod
    def backward(ctx, g_params, g_alpha, g_beta, g_chi2, g_state, g_iters):
        images, offsets, dims, model, params, alpha, beta, state = ctx.saved_tensors
        grad_images = None
        if ctx.needs_input_grad[0]:
            fo = dict(params=params, alpha=alpha, beta=beta, state=state)
            grad_images = backward(images, offsets, dims, model, fo, g_params, g_alpha, g_beta,
                                   g_chi2).view(images.shape)
        grad_init = torch.zeros(ctx.init_shape, dtype=torch.float32, device=params.device) \
            if ctx.needs_input_grad[1] else None
        return grad_images, grad_init, None, None, None, None, None, None, None


def fit_differentiable(images, init, offsets, dims, model, **kw):
    """FitSpotsFunction.apply with keyword tolerances."""
    return FitSpotsFunction.apply(images, init, offsets, dims, model, kw.get("max_iter", 20),
                                  kw.get("max_error", 0.0), kw.get("min_delta", 1e-6),
                                  kw.get("min_step", 1e-4))
