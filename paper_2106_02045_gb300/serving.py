"""Real-time fiducial tracking with continuous batching: a thin binding of the library's
serving sessions (``fs_session_*`` in ``include/fitspots.h``; argument marshalling only).

The session (C++ in ``csrc/serving.cu``) owns the device frame slots, the admission queue,
the batching of frames of different camera streams, one captured CUDA graph per batch
size (ROI cut at the previous positions, warm-started fit, marker-state update) and the
latency stamps. This module keeps the host frames alive until their results are back,
collects the per-frame results and drives the session from a Python loop.
"""
from __future__ import annotations

import ctypes
import gc
from dataclasses import dataclass, field

import numpy as np
import torch

from . import fitspots

CONVERGED = fitspots.CONVERGED_STATES
RESULT_FLOATS = 16   # FS_SERVE_RESULT_FLOATS: x, y, sx, sy, alpha, beta, chi2, state, origin
                     # x, y, warm start (4, ROI coordinates), iterations, 0


class _Config(ctypes.Structure):
    _fields_ = [("frame_w", ctypes.c_int), ("frame_h", ctypes.c_int), ("roi", ctypes.c_int),
                ("markers", ctypes.c_int), ("streams", ctypes.c_int), ("max_batch", ctypes.c_int),
                ("frame_slots", ctypes.c_int), ("queue_limit", ctypes.c_int),
                ("max_inflight", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("min_delta", ctypes.c_double), ("min_step", ctypes.c_double)]


class _Done(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("index", ctypes.c_int64), ("t_arrival", ctypes.c_double),
                ("t_done", ctypes.c_double)]


def _bind():
    lib = fitspots.library()
    if not hasattr(lib, "_serve_bound"):
        vp, i, i64, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        lib.fs_serve_roi_cut.argtypes = [vp, i, i, i, i, vp, i, vp, vp, vp, vp, vp]
        lib.fs_serve_roi_cut.restype = i
        lib.fs_serve_update.argtypes = [vp, i, i, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        lib.fs_serve_update.restype = i
        lib.fs_session_clock.argtypes = []
        lib.fs_session_clock.restype = d
        lib.fs_session_create.argtypes = [ctypes.POINTER(_Config), ctypes.POINTER(vp)]
        lib.fs_session_create.restype = i
        lib.fs_session_destroy.argtypes = [vp]
        lib.fs_session_destroy.restype = i
        lib.fs_session_add_markers.argtypes = [vp, i, vp]
        lib.fs_session_add_markers.restype = i
        lib.fs_session_get_markers.argtypes = [vp, i, vp]
        lib.fs_session_get_markers.restype = i
        lib.fs_session_submit_frame.argtypes = [vp, i, i64, vp, d]
        lib.fs_session_submit_frame.restype = i
        lib.fs_session_poll.argtypes = [vp, vp, vp, i, ctypes.POINTER(i)]
        lib.fs_session_poll.restype = i
        lib.fs_session_pending.argtypes = [vp]
        lib.fs_session_pending.restype = i
        lib.fs_session_stats.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                         ctypes.POINTER(i64)]
        lib.fs_session_stats.restype = i
        lib._serve_bound = True
    return lib


def clock() -> float:
    """The sessions' monotonic clock (seconds): stamp frame arrivals with it."""
    return _bind().fs_session_clock()


@dataclass
class SessionLog:
    results: dict = field(default_factory=dict)   # frame index -> np.ndarray [markers, 16]
    latency: dict = field(default_factory=dict)   # frame index -> seconds


class TrackingServer:
    """A serving session for ``sessions`` camera streams of one frame size (fs_session_*)."""

    def __init__(self, frame_w: int, frame_h: int, markers: int = 64, roi: int = 21,
                 sessions: int = 1, max_batch: int = 8, frame_slots: int = 8,
                 queue_limit: int = 64, max_inflight: int = 2, device="cuda:0",
                 max_iter: int = 20, min_delta: float = 1e-6, min_step: float = 1e-4):
        self.dev = torch.device(device)
        self.lib = _bind()
        self.m = markers
        self.max_batch = min(max_batch, sessions)
        cfg = _Config(frame_w, frame_h, roi, markers, sessions, self.max_batch, frame_slots,
                      queue_limit, max_inflight, max_iter, min_delta, min_step)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.dev):
            fitspots.check(self.lib.fs_session_create(ctypes.byref(cfg), ctypes.byref(h)),
                           "fs_session_create")
        self.h = h
        cap = self.max_batch * max_inflight
        self._done = (_Done * cap)()
        self._res = np.zeros((cap, markers, RESULT_FLOATS), np.float32)
        self._n = ctypes.c_int()
        self._frames = {}          # (stream, index) -> host frame, alive until retired
        self.logs = [SessionLog() for _ in range(sessions)]

    def close(self) -> None:
        if self.h:
            self.lib.fs_session_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass

    # ------------------------------------------------------------------ state
    def set_markers(self, session: int, start: torch.Tensor) -> None:
        """Start state (x, y, sigma_x, sigma_y) of a stream's markers, frame coordinates."""
        a = np.ascontiguousarray(start.detach().cpu().numpy(), dtype=np.float32).reshape(self.m, 4)
        fitspots.check(self.lib.fs_session_add_markers(self.h, session, a.ctypes.data),
                       "fs_session_add_markers")

    def snapshot(self, session: int) -> torch.Tensor:
        """Checkpoint of a stream's marker state (host copy)."""
        a = np.zeros((self.m, 4), np.float32)
        fitspots.check(self.lib.fs_session_get_markers(self.h, session, a.ctypes.data),
                       "fs_session_get_markers")
        return torch.from_numpy(a)

    def restore(self, session: int, snap: torch.Tensor) -> None:
        self.set_markers(session, snap)

    # ------------------------------------------------------------------ serving
    def submit(self, session: int, index: int, host_frame: torch.Tensor, t_arrival: float) -> bool:
        """Offer a frame (host uint16 [H, W], pinned). False if it was rejected."""
        rc = self.lib.fs_session_submit_frame(self.h, session, index,
                                              ctypes.c_void_p(host_frame.data_ptr()), t_arrival)
        if rc == -9:
            return False
        fitspots.check(rc, "fs_session_submit_frame")
        self._frames[(session, index)] = host_frame
        return True

    def step(self) -> int:
        """Admit, launch and retire what is ready; returns the number of frames retired."""
        rc = self.lib.fs_session_poll(self.h, self._done, self._res.ctypes.data, len(self._done),
                                      ctypes.byref(self._n))
        fitspots.check(rc, "fs_session_poll")
        for j in range(self._n.value):
            d = self._done[j]
            log = self.logs[d.stream]
            log.results[d.index] = self._res[j].copy()
            log.latency[d.index] = d.t_done - d.t_arrival
            self._frames.pop((d.stream, d.index), None)
        return self._n.value

    def outstanding(self) -> int:
        """Frames submitted and not yet retired."""
        return int(self.lib.fs_session_pending(self.h))

    def stats(self) -> dict:
        dr, sv, bt = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        fitspots.check(self.lib.fs_session_stats(self.h, ctypes.byref(dr), ctypes.byref(sv),
                                                 ctypes.byref(bt)), "fs_session_stats")
        return {"dropped": dr.value, "served": sv.value, "batches": bt.value}

    @property
    def dropped(self) -> int:
        return self.stats()["dropped"]

    def drain(self, timeout_s: float = 30.0) -> None:
        t_end = clock() + timeout_s
        while self.outstanding() and clock() < t_end:
            self.step()
        if self.outstanding():
            raise TimeoutError("tracking server did not drain")


def run_stream(server: TrackingServer, session: int, host_frames: torch.Tensor, n_frames: int,
               fps: float, t0: float | None = None) -> None:
    """Feed frames of one stream at ``fps`` (arrival = scheduled time on the sessions' clock)
    and serve them. Python's cyclic garbage collector is paused meanwhile: a collection of
    the loop's short-lived objects can stall the host for longer than the queue lasts."""
    t0 = clock() if t0 is None else t0
    period = 1.0 / fps
    ring = host_frames.shape[0]
    k = 0
    was_enabled = gc.isenabled()
    gc.disable()
    try:
        while k < n_frames or server.outstanding():
            now = clock()
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
