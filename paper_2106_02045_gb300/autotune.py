"""Per-size-class kernel configuration autotuner.

Every size class (ceil(W/8), ceil(H/8)) can run several compiled configurations (lanes
per spot, columns per lane, rows, per-spot or batched): ``fitspots.configs()`` lists them and
``fitspots.config_fits`` says which serve a class. The library's built-in defaults were
timed on one GPU with FP32 samples; the best choice also depends on the GPU, the pixel type
and the fit statistics of the data. ``autotune`` times every usable configuration on a synthetic
sample of each class (the class's bound size, so the whole class fits it), keeps the
fastest with ``fitspots.set_config`` and can cache the choice per device.

Timing uses CUDA events around ``fit_spots_uniform`` launches on the current stream;
the sample stays resident on the device. The sample must fill the GPU for every candidate:
the batched configuration (one lane per spot) keeps 16 spots per warp in flight, about
58,000 on a 152-SM GPU, so samples much smaller than twice that favour the per-spot kernels. Results of a spot depend on the configuration
only through the order of FP32 sums (within the parity tolerances either way).
"""
from __future__ import annotations

import json
from pathlib import Path

import torch

from . import fitspots, synth

# the classes with a choice: W, H <= 32 (class 16, a side above 32, has one configuration)
NUM_CLASSES = 16
ELONGATED_CLASS = 16


def class_of(W: int, H: int) -> int:
    """Size class of a W x H spot."""
    if W > 32 or H > 32:
        return ELONGATED_CLASS
    return ((W + 7) // 8 - 1) * 4 + ((H + 7) // 8 - 1)


def class_bounds(cls: int) -> tuple[int, int]:
    """Largest (W, H) of a size class."""
    return (cls // 4 + 1) * 8, (cls % 4 + 1) * 8


def _sample(cls: int, n: int, dtype: int, device, seed: int) -> synth.SpotBatch:
    W, H = class_bounds(cls)
    b = synth.make_ell32(n, seed=seed, device=device, W=W, H=H, name=f"class{cls}")
    if dtype == fitspots.F32:
        b.images = b.images.to(torch.float32)
    return b


def _time_uniform(b: synth.SpotBatch, W: int, H: int, reps: int) -> float:
    stream = torch.cuda.current_stream(b.images.device)
    out = fitspots.alloc_outputs(b.n, b.images.device)
    fitspots.fit_uniform(b.images, W, H, int(b.model[0]), b.init, out=out, stream=stream)
    best = float("inf")
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fitspots.fit_uniform(b.images, W, H, int(b.model[0]), b.init, out=out, stream=stream)
        e1.record(stream)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def autotune(classes=None, n: int = 131072, reps: int = 3, dtype: int = fitspots.F32,
             device="cuda:0", cache: str | Path | None = None, seed: int = 20210610) -> dict:
    """Time every usable configuration of each class; keep and return the fastest.

    The choice applies where a class runs in a launch of its own (fit_spots_uniform and
    fit_spots_per_class); fit_spots runs every class in one launch of the generic kernel.

    Returns {class: {"config": c, "ms": t, "tried": {config: ms}}} and, with ``cache``,
    merges the choice into that JSON file under the device's name and the pixel type.
    """
    device = torch.device(device)
    classes = range(NUM_CLASSES) if classes is None else classes
    n_cfg = len(fitspots.configs())
    result = {}
    for cls in classes:
        W, H = class_bounds(cls)
        b = _sample(cls, n, dtype, device, seed + cls)
        tried = {}
        for cfg in range(n_cfg):
            if not fitspots.config_fits(cls, cfg):
                continue
            fitspots.set_config(cls, cfg)
            tried[cfg] = _time_uniform(b, W, H, reps)
        best = min(tried, key=tried.get)
        fitspots.set_config(cls, best)
        result[int(cls)] = {"config": best, "ms": tried[best], "tried": tried}
        del b
    if cache is not None:
        save(cache, result, dtype, device)
    return result


def _key(dtype: int, device) -> str:
    name = torch.cuda.get_device_name(torch.device(device))
    return f"{name}|{'u16' if dtype == fitspots.U16 else 'f32'}"


def save(cache: str | Path, result: dict, dtype: int, device) -> None:
    path = Path(cache)
    data = json.loads(path.read_text()) if path.exists() else {}
    data[_key(dtype, device)] = {str(c): r["config"] for c, r in result.items()}
    path.write_text(json.dumps(data, indent=1, sort_keys=True))


def load(cache: str | Path, dtype: int = fitspots.F32, device="cuda:0") -> dict:
    """Apply a cached choice for this device and pixel type; returns {class: config}."""
    path = Path(cache)
    if not path.exists():
        return {}
    choice = json.loads(path.read_text()).get(_key(dtype, device), {})
    applied = {}
    for c, cfg in choice.items():
        if fitspots.config_fits(int(c), int(cfg)):
            fitspots.set_config(int(c), int(cfg))
            applied[int(c)] = int(cfg)
    return applied


def defaults() -> None:
    """Restore the built-in configuration of every class."""
    for cls in range(fitspots.num_classes()):
        fitspots.set_config(cls, default_config(cls))


def default_config(cls: int) -> int:
    """The library's built-in configuration of a size class."""
    return fitspots.default_config(cls)
