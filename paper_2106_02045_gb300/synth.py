"""Seeded synthetic spot workloads.

This module only draws inputs: true spot parameters, noisy pixel data and the start
parameters that both the CUDA path and the oracle receive. It holds none of the fitting
arithmetic. Seeds are ``20210603 + workload index``; a workload drawn on a given device
with a given PyTorch build is reproducible bit for bit.

Workloads (pixel (x, y) of a W x H spot sits at element y*W + x, x = 0 is the first
pixel centre):

* ``iso15``   10,000 spots, 15x15 float32, isotropic; centre 7 +- U(1) px,
  sigma ~ U(1.2, 2.0), peak amplitude 1000, background 100, Poisson noise.
* ``ell32``   1,000,000 spots, 32x32 uint16, elliptic; centre 15.5 +- U(1) px,
  sigma_x, sigma_y ~ U(1, 4), photons log-uniform in [200, 20000] (amplitude
  N/(2 pi sx sy)), background U(50, 500), Poisson + N(0, 2^2) read noise + offset 100,
  rounded and clipped to [0, 65535].
* ``mixed``   2,000,000 spots, W, H uniform in 5..32 each, models 50/50, float32;
  isotropic spots draw like ``iso15``, elliptic ones like ``ell32``; every sigma is
  capped at min(W, H)/4; centre (W-1)/2, (H-1)/2 +- U(1); spot offsets are padded to
  4-element (16-byte) boundaries.
* ``iso16``   262,144 spots, 16x16 float32, isotropic like ``iso15``, centre 7.5 +- U(1).
* ``elongated`` 200,000 spots with a side above 32 and at most 1024 pixels (64x16, 128x8,
  40x25, 100x10, 256x4, 341x3, 33x31 and their transposes, uniformly), both models, drawn
  like ``mixed``.
* ``tilted``  1,000,000 spots, 21x21 uint16, isotropic, on a tilted background plane:
  centre 10 +- U(1) px, sigma ~ U(1.0, 1.8), peak amplitude 800, background
  beta + tx (x - 10) + ty (y - 10) with beta ~ U(150, 400) and slopes tx, ty ~ U(-6, 6)
  counts per pixel, Poisson noise; start values are the true parameters moved by
  U(-0.5, 0.5) px and sigma scaled by U(0.8, 1.25) (the fixed rule below would be pulled
  towards the bright side of the tilt).
* ``paper``   the accuracy protocol of the paper's Results section: S x S, centre
  N(0, S/20) around the ROI centre, sigma ~ U(1, 2), integrated signal and total
  background given in counts, Gaussian noise of variance equal to the pixel value,
  rounded to non-negative integers; start values by the paper's rule (3x3 moving
  average maximum, min / max amplitudes, sigma = sqrt(M / pi)).

Start parameters for all other workloads follow one fixed rule: beta0 = min g,
alpha0 = max g - beta0, centre = centroid of max(g - beta0, 0), sigma0 = sqrt(M / pi)
with M = #{g > alpha0 exp(-1/2) + beta0}; elliptic spots start with sigma_x = sigma_y.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

MODEL_ISO, MODEL_ELLIPTIC = 0, 1
SEED_BASE = 20210603
WORKLOADS = ("iso15", "ell32", "mixed", "iso16", "elongated", "tilted")
FULL_SIZES = {"iso15": 10_000, "ell32": 1_000_000, "mixed": 2_000_000, "iso16": 262_144,
              "elongated": 200_000, "tilted": 1_000_000}


@dataclass
class SpotBatch:
    """A packed batch of spots. Tensors live on one device."""

    images: torch.Tensor        # flat uint16 or float32
    offsets: torch.Tensor       # int64 [n], element offset of each spot
    dims: torch.Tensor          # int32 [n, 2] = (W, H)
    model: torch.Tensor         # uint8 [n]
    init: torch.Tensor          # float32 [n, 4] = (x, y, sigma_x, sigma_y)
    truth: dict = field(default_factory=dict)  # float64 tensors: params [n,4], alpha, beta
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.offsets.numel())

    def to(self, device) -> "SpotBatch":
        return SpotBatch(self.images.to(device), self.offsets.to(device), self.dims.to(device),
                         self.model.to(device), self.init.to(device),
                         {k: v.to(device) for k, v in self.truth.items()}, self.name)

    def numpy(self) -> dict:
        return dict(images=self.images.cpu().numpy(), offsets=self.offsets.cpu().numpy(),
                    dims=self.dims.cpu().numpy(), model=self.model.cpu().numpy(),
                    init=self.init.cpu().numpy())

    def head(self, n: int) -> "SpotBatch":
        """The first n spots, sharing storage (spots are packed in index order)."""
        n = int(n)
        if n == 0:
            end = 0
        else:
            last = n - 1
            end = int(self.offsets[last].item() + self.dims[last, 0].item() * self.dims[last, 1].item())
        return SpotBatch(self.images[:end], self.offsets[:n], self.dims[:n], self.model[:n],
                         self.init[:n], {k: v[:n] for k, v in self.truth.items()}, self.name)

    def subset(self, idx) -> "SpotBatch":
        """Spots ``idx`` repacked densely (each keeps its own padding rule)."""
        idx = torch.as_tensor(idx, dtype=torch.int64, device=self.offsets.device)
        dims = self.dims[idx]
        n_el = (dims[:, 0] * dims[:, 1]).to(torch.int64)
        span = (n_el + 3) // 4 * 4
        new_off = torch.cumsum(span, 0) - span
        total = int(span.sum().item()) if idx.numel() else 0
        imgs = torch.zeros(total, dtype=self.images.dtype, device=self.images.device)
        src_off, n_cpu, new_cpu = self.offsets[idx].cpu(), n_el.cpu(), new_off.cpu()
        for k in range(idx.numel()):
            a, m, b = int(src_off[k]), int(n_cpu[k]), int(new_cpu[k])
            imgs[b:b + m] = self.images[a:a + m]
        return SpotBatch(imgs, new_off, dims.clone(), self.model[idx].clone(),
                         self.init[idx].clone(), {k: v[idx].clone() for k, v in self.truth.items()},
                         self.name)


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return g


def _uniform(n, lo, hi, gen, device):
    return lo + (hi - lo) * torch.rand(n, generator=gen, device=device, dtype=torch.float64)


def _render(W: int, H: int, params: torch.Tensor, amp: torch.Tensor, bg: torch.Tensor):
    """Noise-free pixel values amp * exp(-dx^2/2sx^2 - dy^2/2sy^2) + bg, shape [n, H*W]."""
    dev = params.device
    x = torch.arange(W, device=dev, dtype=torch.float64)
    y = torch.arange(H, device=dev, dtype=torch.float64)
    ex = torch.exp(-0.5 * ((x[None, :] - params[:, 0:1]) / params[:, 2:3]) ** 2)   # [n, W]
    ey = torch.exp(-0.5 * ((y[None, :] - params[:, 1:2]) / params[:, 3:4]) ** 2)   # [n, H]
    img = ey[:, :, None] * ex[:, None, :]                                         # [n, H, W]
    return (amp[:, None, None] * img + bg[:, None, None]).reshape(params.shape[0], H * W)


def start_values(g: torch.Tensor, W: int, H: int) -> torch.Tensor:
    """The fixed start rule (module docstring) for spots of one size; g is [n, H*W]."""
    g = g.to(torch.float64)
    n = g.shape[0]
    dev = g.device
    b0 = g.min(dim=1).values
    a0 = g.max(dim=1).values - b0
    w = (g - b0[:, None]).clamp_min(0.0)
    xs = torch.arange(W, device=dev, dtype=torch.float64).repeat(H)
    ys = torch.arange(H, device=dev, dtype=torch.float64).repeat_interleave(W)
    sw = w.sum(dim=1).clamp_min(1e-30)
    x0 = (w * xs).sum(dim=1) / sw
    y0 = (w * ys).sum(dim=1) / sw
    M = (g > (a0 * math.exp(-0.5) + b0)[:, None]).sum(dim=1).to(torch.float64)
    s0 = torch.sqrt(M.clamp_min(1.0) / math.pi)
    out = torch.stack([x0, y0, s0, s0], dim=1)
    return out.to(torch.float32).reshape(n, 4)


def paper_start_values(g: torch.Tensor, S: int) -> torch.Tensor:
    """The paper's start rule (Results section): argmax of the 3x3 moving average, min and
    max amplitudes, sigma = sqrt(M / pi)."""
    g = g.to(torch.float64)
    n = g.shape[0]
    img = g.reshape(n, 1, S, S)
    sm = torch.nn.functional.avg_pool2d(img, 3, stride=1, padding=1, count_include_pad=False)
    k = sm.reshape(n, -1).argmax(dim=1)
    x0 = (k % S).to(torch.float64)
    y0 = (k // S).to(torch.float64)
    b0 = g.min(dim=1).values
    a0 = g.max(dim=1).values - b0
    M = (g > (a0 * math.exp(-0.5) + b0)[:, None]).sum(dim=1).to(torch.float64)
    s0 = torch.sqrt(M.clamp_min(1.0) / math.pi)
    return torch.stack([x0, y0, s0, s0], dim=1).to(torch.float32)


def _pack_uniform(vals: torch.Tensor, W: int, H: int, model: int, init, truth, name):
    n = vals.shape[0]
    dev = vals.device
    N = W * H
    offsets = torch.arange(n, device=dev, dtype=torch.int64) * N
    dims = torch.tensor([W, H], dtype=torch.int32, device=dev).repeat(n, 1)
    models = torch.full((n,), model, dtype=torch.uint8, device=dev)
    return SpotBatch(vals.reshape(-1).contiguous(), offsets, dims, models, init, truth, name)


def make_iso(n: int, S: int, centre: float, seed: int, device="cpu", name="iso") -> SpotBatch:
    """Isotropic S x S float32 spots: peak 1000, background 100, Poisson noise."""
    gen = _gen(seed, device)
    x = centre + _uniform(n, -1.0, 1.0, gen, device)
    y = centre + _uniform(n, -1.0, 1.0, gen, device)
    s = _uniform(n, 1.2, 2.0, gen, device)
    params = torch.stack([x, y, s, s], dim=1)
    amp = torch.full((n,), 1000.0, dtype=torch.float64, device=device)
    bg = torch.full((n,), 100.0, dtype=torch.float64, device=device)
    lam = _render(S, S, params, amp, bg)
    g = torch.poisson(lam, generator=gen).to(torch.float32)
    init = start_values(g, S, S)
    truth = dict(params=params, alpha=amp, beta=bg)
    return _pack_uniform(g, S, S, MODEL_ISO, init, truth, name)


def make_ell32(n: int, seed: int = SEED_BASE + 2, device="cpu", W: int = 32, H: int = 32,
               name="ell32") -> SpotBatch:
    """Elliptic uint16 spots with camera-like noise (module docstring, ``ell32``)."""
    gen = _gen(seed, device)
    x = (W - 1) / 2 + _uniform(n, -1.0, 1.0, gen, device)
    y = (H - 1) / 2 + _uniform(n, -1.0, 1.0, gen, device)
    sx = _uniform(n, 1.0, 4.0, gen, device)
    sy = _uniform(n, 1.0, 4.0, gen, device)
    nph = torch.exp(_uniform(n, math.log(200.0), math.log(20000.0), gen, device))
    bg = _uniform(n, 50.0, 500.0, gen, device)
    params = torch.stack([x, y, sx, sy], dim=1)
    amp = nph / (2 * math.pi * sx * sy)
    lam = _render(W, H, params, amp, bg)
    e = torch.poisson(lam, generator=gen)
    read = 2.0 * torch.randn(lam.shape, generator=gen, device=device, dtype=torch.float64)
    g = torch.round(e + read + 100.0).clamp(0, 65535)
    init = start_values(g, W, H)
    truth = dict(params=params, alpha=amp, beta=bg + 100.0)
    g16 = g.to(torch.int32).to(torch.uint16)
    return _pack_uniform(g16, W, H, MODEL_ELLIPTIC, init, truth, name)


def make_tilted(n: int, seed: int = SEED_BASE + 6, device="cpu", S: int = 21,
                name="tilted") -> SpotBatch:
    """Isotropic uint16 spots on a tilted background plane (module docstring, ``tilted``)."""
    gen = _gen(seed, device)
    c = (S - 1) / 2
    x = c + _uniform(n, -1.0, 1.0, gen, device)
    y = c + _uniform(n, -1.0, 1.0, gen, device)
    s = _uniform(n, 1.0, 1.8, gen, device)
    bg = _uniform(n, 150.0, 400.0, gen, device)
    tilt = torch.stack([_uniform(n, -6.0, 6.0, gen, device),
                        _uniform(n, -6.0, 6.0, gen, device)], dim=1)
    params = torch.stack([x, y, s, s], dim=1)
    amp = torch.full((n,), 800.0, dtype=torch.float64, device=device)
    lam = _render(S, S, params, amp, bg)
    xs = torch.arange(S, device=device, dtype=torch.float64) - c
    plane = (tilt[:, 0:1, None] * xs[None, None, :] + tilt[:, 1:2, None] * xs[None, :, None])
    lam = lam + plane.reshape(n, S * S)
    g = torch.poisson(lam, generator=gen).clamp(0, 65535)
    init = params.clone()
    init[:, :2] += _uniform(2 * n, -0.5, 0.5, gen, device).reshape(n, 2)
    init[:, 2] *= _uniform(n, 0.8, 1.25, gen, device)
    init[:, 3] = init[:, 2]
    truth = dict(params=params, alpha=amp, beta=bg, tilt=tilt)
    g16 = g.to(torch.int32).to(torch.uint16)
    return _pack_uniform(g16, S, S, MODEL_ISO, init.to(torch.float32), truth, name)


def make_mixed(n: int, seed: int = SEED_BASE + 3, device="cpu", name="mixed") -> SpotBatch:
    """Mixed sizes 5..32 per side, both models, float32, 16-byte aligned offsets."""
    gen = _gen(seed, device)
    Ws = torch.randint(5, 33, (n,), generator=gen, device=device)
    Hs = torch.randint(5, 33, (n,), generator=gen, device=device)
    models = (torch.rand(n, generator=gen, device=device) < 0.5).to(torch.uint8)
    return _pack_sized(Ws, Hs, models, gen, device, name)


# elongated shapes: a side above 32 and at most 1024 pixels, both orientations
ELONGATED_SHAPES = ((64, 16), (16, 64), (128, 8), (8, 128), (40, 25), (25, 40), (100, 10),
                    (10, 100), (256, 4), (4, 256), (341, 3), (3, 341), (33, 31), (31, 33))


def make_elongated(n: int, seed: int = SEED_BASE + 5, device="cpu",
                   shapes=ELONGATED_SHAPES, name="elongated") -> SpotBatch:
    """ROIs with a side above 32 (the paper's bound is 1024 pixels per fit, not a side):
    shapes drawn uniformly from ``shapes``, both models, drawn like ``mixed`` (float32)."""
    gen = _gen(seed, device)
    pick = torch.randint(0, len(shapes), (n,), generator=gen, device=device)
    table = torch.tensor(shapes, dtype=torch.int64, device=device)
    Ws, Hs = table[pick, 0], table[pick, 1]
    models = (torch.rand(n, generator=gen, device=device) < 0.5).to(torch.uint8)
    return _pack_sized(Ws, Hs, models, gen, device, name)


def _pack_sized(Ws, Hs, models, gen, device, name) -> SpotBatch:
    """Spots of the given sizes and models: isotropic ones drawn like ``iso15``, elliptic
    ones like ``ell32`` (as float32), every sigma capped at min(W, H) / 4, the centre within
    1 px of the ROI centre; offsets padded to 4-element (16-byte) boundaries."""
    n = Ws.numel()
    n_el = (Ws * Hs).to(torch.int64)
    span = (n_el + 3) // 4 * 4
    offsets = torch.cumsum(span, 0) - span
    images = torch.zeros(int(span.sum().item()), dtype=torch.float32, device=device)
    init = torch.empty((n, 4), dtype=torch.float32, device=device)
    tp = torch.empty((n, 4), dtype=torch.float64, device=device)
    ta = torch.empty(n, dtype=torch.float64, device=device)
    tb = torch.empty(n, dtype=torch.float64, device=device)
    key = (Ws * 1024 + Hs) * 2 + models.to(torch.int64)
    for k in torch.unique(key).tolist():
        idx = torch.nonzero(key == k).flatten()
        m = int(k % 2)
        W, H = int(k // 2 // 1024), int(k // 2 % 1024)
        cnt = idx.numel()
        cap = min(W, H) / 4.0
        x = (W - 1) / 2 + _uniform(cnt, -1.0, 1.0, gen, device)
        y = (H - 1) / 2 + _uniform(cnt, -1.0, 1.0, gen, device)
        if m == MODEL_ISO:
            s = _uniform(cnt, 1.2, 2.0, gen, device).clamp_max(cap)
            params = torch.stack([x, y, s, s], dim=1)
            amp = torch.full((cnt,), 1000.0, dtype=torch.float64, device=device)
            bg = torch.full((cnt,), 100.0, dtype=torch.float64, device=device)
            g = torch.poisson(_render(W, H, params, amp, bg), generator=gen)
            beta = bg
        else:
            sx = _uniform(cnt, 1.0, 4.0, gen, device).clamp_max(cap)
            sy = _uniform(cnt, 1.0, 4.0, gen, device).clamp_max(cap)
            nph = torch.exp(_uniform(cnt, math.log(200.0), math.log(20000.0), gen, device))
            bg = _uniform(cnt, 50.0, 500.0, gen, device)
            params = torch.stack([x, y, sx, sy], dim=1)
            amp = nph / (2 * math.pi * sx * sy)
            lam = _render(W, H, params, amp, bg)
            read = 2.0 * torch.randn(lam.shape, generator=gen, device=device, dtype=torch.float64)
            g = torch.poisson(lam, generator=gen) + read + 100.0
            beta = bg + 100.0
        gf = g.to(torch.float32)
        cols = offsets[idx][:, None] + torch.arange(W * H, device=device)[None, :]
        images[cols.reshape(-1)] = gf.reshape(-1)
        init[idx] = start_values(gf, W, H)
        tp[idx], ta[idx], tb[idx] = params, amp, beta
    dims = torch.stack([Ws, Hs], dim=1).to(torch.int32)
    return SpotBatch(images, offsets, dims, models, init, dict(params=tp, alpha=ta, beta=tb), name)


def make_paper(n: int, S: int, signal: float, background: float, seed: int, device="cpu",
               name="paper") -> SpotBatch:
    """Accuracy protocol of the paper's Results section (module docstring, ``paper``)."""
    gen = _gen(seed, device)
    c = (S - 1) / 2
    x = c + (S / 20.0) * torch.randn(n, generator=gen, device=device, dtype=torch.float64)
    y = c + (S / 20.0) * torch.randn(n, generator=gen, device=device, dtype=torch.float64)
    s = _uniform(n, 1.0, 2.0, gen, device)
    params = torch.stack([x, y, s, s], dim=1)
    amp = signal / (2 * math.pi * s * s)
    bg = torch.full((n,), background / (S * S), dtype=torch.float64, device=device)
    lam = _render(S, S, params, amp, bg)
    noisy = lam + torch.sqrt(lam) * torch.randn(lam.shape, generator=gen, device=device,
                                                dtype=torch.float64)
    g = torch.round(noisy).clamp_min(0.0).to(torch.float32)
    init = paper_start_values(g, S)
    truth = dict(params=params, alpha=amp, beta=bg)
    return _pack_uniform(g, S, S, MODEL_ISO, init, truth, name)


@dataclass
class CameraStream:
    """Synthetic camera frames with drifting fiducial markers (serving workload)."""

    frames: torch.Tensor      # uint16 [n_frames, H, W]
    truth: torch.Tensor       # float64 [n_frames, markers, 2] marker centres (x, y)
    sigma: torch.Tensor       # float64 [markers]
    start: torch.Tensor       # float32 [markers, 4] start state (x, y, s, s), ~0.3 px off


def make_camera_stream(n_frames: int, markers: int = 64, width: int = 2048, height: int = 2048,
                       seed: int = SEED_BASE + 5, device="cpu", photons: float = 20000.0,
                       background: float = 100.0, drift: float = 0.05) -> CameraStream:
    """uint16 frames: background + markers of sigma ~ U(1.2, 2.0) carrying ``photons``
    each, Poisson + N(0, 2^2) read noise + offset 100; marker centres at least 16 px from
    the border, moving as a Gaussian random walk of ``drift`` px per frame and axis."""
    gen = _gen(seed, device)
    f64 = torch.float64
    x0 = 16 + (width - 33) * torch.rand(markers, generator=gen, device=device, dtype=f64)
    y0 = 16 + (height - 33) * torch.rand(markers, generator=gen, device=device, dtype=f64)
    sig = 1.2 + 0.8 * torch.rand(markers, generator=gen, device=device, dtype=f64)
    steps = drift * torch.randn(n_frames, markers, 2, generator=gen, device=device, dtype=f64)
    steps[0] = 0.0
    pos = torch.stack([x0, y0], dim=1)[None] + torch.cumsum(steps, dim=0)
    pos[..., 0].clamp_(14, width - 15)
    pos[..., 1].clamp_(14, height - 15)
    amp = photons / (2 * math.pi * sig * sig)
    frames = torch.empty((n_frames, height, width), dtype=torch.uint16, device=device)
    half = 12
    ar = torch.arange(-half, half + 1, device=device)
    for k in range(n_frames):
        lam = torch.full((height, width), background, dtype=f64, device=device)
        cx = torch.round(pos[k, :, 0]).long()
        cy = torch.round(pos[k, :, 1]).long()
        xs = (cx[:, None] + ar[None, :]).clamp(0, width - 1)              # [m, 25]
        ys = (cy[:, None] + ar[None, :]).clamp(0, height - 1)
        fx = torch.exp(-0.5 * ((xs - pos[k, :, 0:1]) / sig[:, None]) ** 2)
        fy = torch.exp(-0.5 * ((ys - pos[k, :, 1:2]) / sig[:, None]) ** 2)
        spot = amp[:, None, None] * fy[:, :, None] * fx[:, None, :]        # [m, 25, 25]
        idx = (ys[:, :, None] * width + xs[:, None, :]).reshape(-1)
        lam.view(-1).index_add_(0, idx, spot.reshape(-1))
        noisy = torch.poisson(lam, generator=gen) + 2.0 * torch.randn(
            lam.shape, generator=gen, device=device, dtype=f64) + 100.0
        frames[k] = torch.round(noisy).clamp(0, 65535).to(torch.int32).to(torch.uint16)
    off = 0.3 * (2 * torch.rand(markers, 2, generator=gen, device=device, dtype=f64) - 1)
    start = torch.stack([pos[0, :, 0] + off[:, 0], pos[0, :, 1] + off[:, 1], sig * 1.1, sig * 1.1],
                        dim=1).to(torch.float32)
    return CameraStream(frames, pos, sig, start)


def make_workload(name: str, n: int | None = None, device="cpu") -> SpotBatch:
    """One of ``WORKLOADS`` at its full size, or its first ``n`` draws at size n."""
    n = FULL_SIZES[name] if n is None else int(n)
    if name == "iso15":
        return make_iso(n, 15, 7.0, SEED_BASE + 1, device, name)
    if name == "ell32":
        return make_ell32(n, SEED_BASE + 2, device, name=name)
    if name == "mixed":
        return make_mixed(n, SEED_BASE + 3, device, name)
    if name == "iso16":
        return make_iso(n, 16, 7.5, SEED_BASE + 4, device, name)
    if name == "elongated":
        return make_elongated(n, SEED_BASE + 5, device, name=name)
    if name == "tilted":
        return make_tilted(n, SEED_BASE + 6, device, name=name)
    raise KeyError(name)


def as_numpy_images(batch: SpotBatch) -> np.ndarray:
    """Pixel buffer as numpy (uint16 stays uint16)."""
    t = batch.images.cpu()
    if t.dtype == getattr(torch, "uint16", None):
        return t.view(torch.int16).numpy().view(np.uint16)
    return t.numpy()
