"""Real-time fiducial tracking with continuous batching (host orchestration).

Per frame the device work is one captured CUDA graph: ROI cut at the markers' previous
positions (``fs_serve_roi_cut``), the warm-started batched fit (``fit_spots_uniform``) and
the marker-state update (``fs_serve_update``); marker state stays on the device. Frames of
several sessions that are on the device at the same time form one batch (at most one
frame per session, because a session's next ROI placement needs its previous fit), so a
frame that arrives while a batch is running is admitted into a free frame slot, copied
in on a separate stream while the running batch computes, and joins the next batch.

Admission is by memory: ``frame_slots`` device frame buffers. A frame that finds no free
slot waits in a bounded queue; beyond ``queue_limit`` it is rejected (counted in
``dropped``). Latency = host arrival stamp -> results visible on the host.
"""
from __future__ import annotations

import collections
import gc
import ctypes
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import fitspots

CONVERGED = fitspots.CONVERGED_STATES


def _bind():
    lib = fitspots.library()
    if not hasattr(lib, "_serve_bound"):
        vp, i = ctypes.c_void_p, ctypes.c_int
        lib.fs_serve_roi_cut.argtypes = [vp, i, i, i, i, vp, i, vp, vp, vp, vp, vp]
        lib.fs_serve_roi_cut.restype = i
        lib.fs_serve_update.argtypes = [vp, i, i, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        lib.fs_serve_update.restype = i
        lib._serve_bound = True
    return lib


def _p(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr())


@dataclass
class FrameRecord:
    session: int
    index: int
    t_arrival: float
    host_frame: torch.Tensor
    slot: int = -1
    copied: torch.cuda.Event | None = None
    t_done: float = 0.0


@dataclass
class Batch:
    frames: list
    done: torch.cuda.Event
    results: torch.Tensor          # pinned host [k * markers, 8]
    desc: torch.Tensor             # pinned host descriptor used by this batch


@dataclass
class SessionLog:
    results: dict = field(default_factory=dict)   # frame index -> np.ndarray [markers, 8]
    latency: dict = field(default_factory=dict)   # frame index -> seconds


class TrackingServer:
    """Continuous-batching tracker for ``sessions`` camera streams of one frame size."""

    def __init__(self, frame_w: int, frame_h: int, markers: int = 64, roi: int = 21,
                 sessions: int = 1, max_batch: int = 8, frame_slots: int = 8,
                 queue_limit: int = 64, max_inflight: int = 2, device="cuda:0",
                 max_iter: int = 20, min_delta: float = 1e-6, min_step: float = 1e-4):
        self.dev = torch.device(device)
        self.fw, self.fh, self.m, self.roi = frame_w, frame_h, markers, roi
        self.max_batch = min(max_batch, sessions) if sessions > 0 else max_batch
        self.queue_limit, self.max_inflight = queue_limit, max_inflight
        self.tol = dict(max_iter=max_iter, min_delta=min_delta, min_step=min_step)
        self.lib = _bind()
        dev = self.dev
        self.frames = torch.zeros((frame_slots, frame_h, frame_w), dtype=torch.uint16, device=dev)
        self.free_slots = collections.deque(range(frame_slots))
        self.state = torch.zeros((sessions, markers, 4), dtype=torch.float32, device=dev)
        nmax = self.max_batch * markers
        self.rois = torch.zeros(nmax * roi * roi, dtype=torch.uint16, device=dev)
        self.init = torch.zeros((nmax, 4), dtype=torch.float32, device=dev)
        self.origin = torch.zeros((nmax, 2), dtype=torch.int32, device=dev)
        self.fit_out = fitspots.alloc_outputs(nmax, dev)
        self.results = torch.zeros((nmax, 8), dtype=torch.float32, device=dev)
        self.desc = torch.zeros(1 + 2 * self.max_batch, dtype=torch.int32, device=dev)
        # pinned staging for batch descriptors, one per batch in flight (a host buffer must
        # not change before its copy has executed)
        self.desc_pool = collections.deque(
            torch.zeros(1 + 2 * self.max_batch, dtype=torch.int32, pin_memory=True)
            for _ in range(max_inflight + 2))
        self.ws = torch.empty(max(int(self.lib.fit_spots_uniform_workspace()), 16),
                              dtype=torch.uint8, device=dev)
        self.compute = torch.cuda.Stream(dev)
        self.copy = torch.cuda.Stream(dev)
        self.result_pool = collections.deque(
            torch.zeros((nmax, 8), dtype=torch.float32, pin_memory=True) for _ in range(8))
        self.pending: collections.deque = collections.deque()   # waiting for a frame slot
        self.landed: list = []                                   # copied in (or copying)
        self.inflight: collections.deque = collections.deque()
        self.logs = [SessionLog() for _ in range(sessions)]
        self.dropped = 0
        self.graphs = {}
        self._capture()

    # ------------------------------------------------------------------ device work
    def _device_step(self, k: int, stream):
        s = ctypes.c_void_p(stream.cuda_stream)
        rc = self.lib.fs_serve_roi_cut(_p(self.frames), self.fw, self.fh, self.roi, self.m,
                                       _p(self.desc), k, _p(self.state), _p(self.rois),
                                       _p(self.init), _p(self.origin), s)
        fitspots.check(rc, "fs_serve_roi_cut")
        n = k * self.m
        o = {key: v[:n] for key, v in self.fit_out.items()}
        fitspots.fit_uniform(self.rois[:n * self.roi * self.roi], self.roi, self.roi,
                             fitspots.MODEL_ISO, self.init[:n], out=o, workspace=self.ws,
                             stream=stream, **self.tol)
        rc = self.lib.fs_serve_update(_p(self.desc), k, self.m, _p(o["params"]), _p(o["alpha"]),
                                      _p(o["beta"]), _p(o["chi2"]), _p(o["state"]),
                                      _p(self.origin), _p(self.state), _p(self.results), s)
        fitspots.check(rc, "fs_serve_update")

    def _capture(self):
        """One graph per batch size; the batch's slots and sessions come from self.desc."""
        with torch.cuda.stream(self.compute):
            self.desc.zero_()
            for k in range(1, self.max_batch + 1):   # warm-up (lazy attribute set-up) outside capture
                self._device_step(k, self.compute)
            self.compute.synchronize()
            for k in range(1, self.max_batch + 1):
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=self.compute):
                    self._device_step(k, self.compute)
                self.graphs[k] = g
        self.compute.synchronize()

    # ------------------------------------------------------------------ API
    def set_markers(self, session: int, start: torch.Tensor) -> None:
        """Start state (x, y, sigma_x, sigma_y) of a session's markers, frame coordinates."""
        self.state[session].copy_(start.to(self.dev, torch.float32))
        torch.cuda.synchronize(self.dev)

    def snapshot(self, session: int) -> torch.Tensor:
        """Checkpoint of a session's marker state (host copy)."""
        torch.cuda.synchronize(self.dev)
        return self.state[session].cpu().clone()

    def restore(self, session: int, snap: torch.Tensor) -> None:
        self.set_markers(session, snap)

    def submit(self, session: int, index: int, host_frame: torch.Tensor, t_arrival: float) -> bool:
        """Offer a frame (pinned host uint16 [H, W]). False if it was rejected."""
        if len(self.pending) >= self.queue_limit:
            self.dropped += 1
            return False
        self.pending.append(FrameRecord(session, index, t_arrival, host_frame))
        return True

    def step(self) -> int:
        """Admit, launch and retire what is ready; returns the number of frames retired."""
        # 1. admission: free frame slots (the memory budget) take waiting frames
        while self.pending and self.free_slots:
            fr = self.pending.popleft()
            fr.slot = self.free_slots.popleft()
            with torch.cuda.stream(self.copy):
                self.frames[fr.slot].copy_(fr.host_frame, non_blocking=True)
                fr.copied = torch.cuda.Event()
                fr.copied.record(self.copy)
            self.landed.append(fr)
        # 2. launch: one frame per session, oldest first, among frames already on the device
        if self.landed and len(self.inflight) < self.max_inflight:
            chosen, seen = [], set()
            for fr in self.landed:
                if fr.session in seen or not fr.copied.query():
                    continue
                if any(f.session == fr.session for b in self.inflight for f in b.frames):
                    continue   # its previous frame is still on the device
                chosen.append(fr)
                seen.add(fr.session)
                if len(chosen) == self.max_batch:
                    break
            if chosen:
                for fr in chosen:
                    self.landed.remove(fr)
                self._launch(chosen)
        # 3. retire finished batches
        done = 0
        while self.inflight and self.inflight[0].done.query():
            b = self.inflight.popleft()
            t = time.perf_counter()
            res = b.results.numpy()
            for j, fr in enumerate(b.frames):
                log = self.logs[fr.session]
                log.results[fr.index] = res[j * self.m:(j + 1) * self.m].copy()
                log.latency[fr.index] = t - fr.t_arrival
                self.free_slots.append(fr.slot)
            self.result_pool.append(b.results)
            self.desc_pool.append(b.desc)
            done += len(b.frames)
        return done

    def _launch(self, frames: list) -> None:
        k = len(frames)
        desc = self.desc_pool.popleft()
        desc[0] = k
        for j, fr in enumerate(frames):
            desc[1 + 2 * j] = fr.slot
            desc[2 + 2 * j] = fr.session
        res = self.result_pool.popleft()
        with torch.cuda.stream(self.compute):
            for fr in frames:
                self.compute.wait_event(fr.copied)
            self.desc.copy_(desc, non_blocking=True)
            self.graphs[k].replay()
            res[:k * self.m].copy_(self.results[:k * self.m], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(self.compute)
        self.inflight.append(Batch(frames, ev, res, desc))

    def drain(self, timeout_s: float = 30.0) -> None:
        t_end = time.perf_counter() + timeout_s
        while (self.pending or self.landed or self.inflight) and time.perf_counter() < t_end:
            self.step()
        if self.pending or self.landed or self.inflight:
            raise TimeoutError("tracking server did not drain")


def run_stream(server: TrackingServer, session: int, host_frames: torch.Tensor, n_frames: int,
               fps: float, t0: float | None = None) -> None:
    """Feed frames of one session at ``fps`` (arrival = scheduled time) and serve them.
    Python's cyclic garbage collector is paused meanwhile: a collection of the loop's
    short-lived objects can stall the host for longer than the queue's 32 ms at 2000 fps."""
    t0 = time.perf_counter() if t0 is None else t0
    period = 1.0 / fps
    ring = host_frames.shape[0]
    k = 0
    was_enabled = gc.isenabled()
    gc.disable()
    try:
        while k < n_frames or server.pending or server.landed or server.inflight:
            now = time.perf_counter()
            while k < n_frames and t0 + k * period <= now:
                server.submit(session, k, host_frames[k % ring], t0 + k * period)
                k += 1
            server.step()
    finally:
        if was_enabled:
            gc.enable()


def latency_summary(lat: np.ndarray) -> dict:
    lat = np.asarray(lat) * 1e3
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "max_ms": float(lat.max()), "frames": int(lat.size)}
