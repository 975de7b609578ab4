"""The C-ABI library builds, loads and exports every declared symbol; host-side argument
checks reject bad calls before any GPU work (no GPU needed)."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def lib():
    from paper_2106_02045_gb300 import build, fitspots
    build.build()
    return fitspots.library()


def _declared():
    names = []
    for h in (ROOT / "include").glob("*.h"):
        text = re.sub(r"/\*.*?\*/", "", h.read_text(), flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b([A-Za-z_]\w*)\s*\(", text, flags=re.M):
            if m.group(1) not in ("defined",):
                names.append(m.group(1))
    return sorted(set(names))


def test_every_declared_function_is_exported(lib):
    names = _declared()
    assert "fit_spots" in names and "fit_spots_uniform" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_workspace_sizes(lib):
    assert lib.fit_spots_workspace(0) == 0
    assert lib.fit_spots_workspace(-5) == 0
    # the schedule header: counts, starts, cursors and fill cursors of the 17 size classes
    assert lib.fit_spots_workspace(1000) == 272 + 4 * 1000
    assert lib.fit_spots_uniform_workspace() == 272


def _call(lib, **over):
    """fit_spots with dummy (never dereferenced) pointers; only argument checks run."""
    fake = ctypes.c_void_p(0x1000)
    a = dict(images=fake, dtype=1, image_elems=100, offsets=fake, dims=fake, init=fake,
             model=fake, n=10, max_iter=20, max_error=0.0, min_delta=1e-6, min_step=1e-4,
             params=fake, alpha=fake, beta=fake, chi2=fake, state=fake, iters=fake,
             evals=None, ws=fake, ws_bytes=0, stream=None)
    a.update(over)
    return lib.fit_spots(a["images"], a["dtype"], a["image_elems"], a["offsets"], a["dims"],
                         a["init"], a["model"], a["n"], a["max_iter"], a["max_error"],
                         a["min_delta"], a["min_step"], a["params"], a["alpha"], a["beta"],
                         a["chi2"], a["state"], a["iters"], a["evals"], a["ws"], a["ws_bytes"],
                         a["stream"])


def test_argument_checks(lib):
    assert _call(lib, n=0) == 0                       # nothing to do, nothing enqueued
    assert _call(lib, n=-1) == -2
    assert _call(lib, n=2**31) == -2
    assert _call(lib, image_elems=-1) == -2
    assert _call(lib, dtype=7) == -3
    assert _call(lib, max_iter=0) == -4
    assert _call(lib, max_iter=1001) == -4
    assert _call(lib, min_delta=-1e-6) == -5
    assert _call(lib, min_delta=1.0) == -5
    assert _call(lib, min_step=float("nan")) == -5
    assert _call(lib, max_error=float("inf")) == -5
    assert _call(lib, images=None) == -1
    assert _call(lib, ws=None) == -1
    assert _call(lib, ws_bytes=10) == -6                # smaller than fit_spots_workspace(10)
    assert _call(lib, ws=ctypes.c_void_p(0x1004), ws_bytes=1 << 20) == -6   # misaligned
    for code in (0, -1, -2, -3, -4, -5, -6, -7, -8):
        assert lib.fit_spots_strerror(code)
    assert lib.fit_spots_last_cuda_error() == 0


def test_uniform_argument_checks(lib):
    fake = ctypes.c_void_p(0x1000)

    def call(W=32, H=32, model=1, n=10, ws=fake, ws_bytes=272, max_iter=20):
        return lib.fit_spots_uniform(fake, 0, W, H, model, fake, n, max_iter, 0.0, 1e-6, 1e-4,
                                     fake, fake, fake, fake, fake, fake, None, ws, ws_bytes, None)
    assert call(W=2) == -8 and call(H=3, W=342) == -8 and call(model=3) == -8
    assert call(W=33, H=32) == -8                       # 1056 pixels: above the 1024 bound
    assert call(W=64, H=16, n=0) == 0 and call(W=3, H=341, n=0) == 0   # elongated ROIs
    assert call(n=0) == 0
    assert call(ws_bytes=16) == -6
    assert call(ws=None) == -1
    assert call(max_iter=0) == -4


def test_host_call_argument_checks(lib):
    """fit_spots_uniform_host: sizes of its double-buffered device scratch, and the checks
    that run before any CUDA call."""
    one = lib.fit_spots_uniform_host_workspace(1000, 32, 32, 0)
    # per chunk buffer: images, start values, 7 outputs, schedule header; 256-byte aligned
    up = lambda v: (v + 255) // 256 * 256
    assert one == 2 * (up(1000 * 32 * 32 * 2) + 2 * up(16000) + 5 * up(4000) + up(4000) + up(272))
    assert lib.fit_spots_uniform_host_workspace(1000, 32, 32, 1) > one
    assert lib.fit_spots_uniform_host_workspace(0, 32, 32, 0) == 0
    assert lib.fit_spots_uniform_host_workspace(10, 33, 32, 0) == 0      # 1056 pixels
    assert lib.fit_spots_uniform_host_workspace(10, 64, 16, 0) > 0       # elongated
    assert lib.fit_spots_uniform_host_workspace(10, 32, 32, 5) == 0
    fake = ctypes.c_void_p(0x1000)

    def call(W=32, H=32, model=1, n=10, chunk=4, ws=ctypes.c_void_p(0x10000), ws_bytes=1 << 30,
             images=fake, max_iter=20):
        return lib.fit_spots_uniform_host(images, 0, W, H, model, fake, n, max_iter, 0.0, 1e-6,
                                          1e-4, fake, fake, fake, fake, fake, fake, None, chunk,
                                          ws, ws_bytes, None)
    assert call(chunk=0) == -8 and call(W=2) == -8 and call(model=2) == -8
    assert call(n=0) == 0
    assert call(images=None) == -1 and call(ws=None) == -1
    assert call(ws_bytes=1000) == -6                          # below two chunk buffers
    assert call(ws=ctypes.c_void_p(0x10010)) == -6            # not 256-byte aligned
    assert call(max_iter=0) == -4


def test_start_and_explicit_argument_checks(lib):
    """fit_spots_start and the one-warp comparison fits reject malformed calls
    before any CUDA work."""
    fake = ctypes.c_void_p(0x1000)

    def start(n=10, dtype=0, rule=0, elems=100, images=fake, out=fake):
        return lib.fit_spots_start(images, dtype, elems, fake, fake, n, rule, out, None)
    assert start(n=-1) == -2 and start(elems=-1) == -2 and start(dtype=4) == -3
    assert start(rule=2) == -8 and start(n=0) == 0
    assert start(images=None) == -1 and start(out=None) == -1

    for fn in (lib.fit_spots_explicit, lib.fit_spots_weighted, lib.fit_spots_poisson):
        def call(n=10, max_iter=20, min_delta=1e-6, images=fake, state=fake):
            return fn(images, 0, 100, fake, fake, fake, fake, n, max_iter, 0.0, min_delta, 1e-4,
                      fake, fake, fake, fake, state, fake, None, None)
        assert call(n=-1) == -2 and call(max_iter=0) == -4 and call(min_delta=1.0) == -5
        assert call(n=0) == 0 and call(images=None) == -1 and call(state=None) == -1


def test_background_argument_checks(lib):
    """fit_spots_subtract_background rejects malformed calls before any CUDA work."""
    fake = ctypes.c_void_p(0x1000)

    def call(n=10, dtype=0, elems=100, border=1, images=fake, out=fake, plane=fake):
        return lib.fit_spots_subtract_background(images, dtype, elems, fake, fake, n, border,
                                                 out, plane, None)
    assert call(n=-1) == -2 and call(elems=-1) == -2 and call(n=2**31 - 2**24 + 1) == -2
    assert call(dtype=2) == -3 and call(dtype=-1) == -3
    assert call(border=0) == -8 and call(border=9) == -8
    assert call(n=0) == 0
    assert call(images=None) == -1 and call(out=None) == -1


def test_backward_argument_checks(lib):
    """fit_spots_backward rejects malformed calls before any CUDA call; n = 0 is a no-op."""
    fake = ctypes.c_void_p(0x1000)

    def call(n=10, dtype=1, elems=2560, images=fake, state=fake, grad=fake):
        return lib.fit_spots_backward(images, dtype, elems, fake, fake, fake, n, fake, fake,
                                      fake, state, None, None, None, None, grad, None)
    assert call(n=-1) == -2 and call(n=2**31) == -2 and call(elems=-1) == -2
    assert call(dtype=2) == -3 and call(dtype=-1) == -3
    assert call(n=0) == 0
    assert call(images=None) == -1 and call(state=None) == -1 and call(grad=None) == -1


def test_serving_argument_checks(lib):
    """fs_serve_roi_cut and fs_serve_update reject NULL pointers and out-of-range sizes
    before launching anything."""
    from paper_2106_02045_gb300 import serving
    serving._bind()
    fake = ctypes.c_void_p(0x1000)

    def cut(roi=21, fw=2048, fh=2048, markers=64, batch=8, frames=fake):
        return lib.fs_serve_roi_cut(frames, fw, fh, roi, markers, fake, batch, fake, fake, fake,
                                    fake, None)
    assert cut(frames=None) == -1
    assert cut(roi=2) == -8 and cut(roi=33) == -8 and cut(fw=20) == -8 and cut(fh=20) == -8
    assert cut(markers=0) == -8 and cut(batch=0) == -8
    assert cut(markers=65536) == -8 and cut(batch=65536) == -8

    def upd(markers=64, batch=8, state=fake, iters=fake):
        return lib.fs_serve_update(fake, batch, markers, fake, fake, fake, fake, fake, iters,
                                   fake, fake, state, fake, None)
    assert upd(state=None) == -1 and upd(iters=None) == -1
    assert upd(markers=0) == -8 and upd(batch=0) == -8
    assert upd(markers=65536) == -8 and upd(batch=65536) == -8


def test_session_argument_checks(lib):
    """fs_session_create rejects a malformed configuration before any CUDA call; the other
    session calls reject a NULL session."""
    from paper_2106_02045_gb300 import serving
    serving._bind()
    good = dict(frame_w=2048, frame_h=2048, roi=21, markers=64, streams=2, max_batch=2,
                frame_slots=8, queue_limit=64, max_inflight=2, max_iter=20, min_delta=1e-6,
                min_step=1e-4)

    def create(**over):
        c = dict(good, **over)
        cfg = serving._Config(*(c[f] for f, _ in serving._Config._fields_))
        h = ctypes.c_void_p()
        return lib.fs_session_create(ctypes.byref(cfg), ctypes.byref(h))
    for bad in (dict(roi=2), dict(roi=33), dict(frame_w=20), dict(markers=0), dict(streams=0),
                dict(max_batch=3), dict(max_batch=0), dict(frame_slots=0), dict(queue_limit=-1),
                dict(max_inflight=0), dict(max_iter=0), dict(min_delta=1.0), dict(min_step=-1.0)):
        assert create(**bad) == -8, bad
    assert lib.fs_session_create(None, None) == -1
    n = ctypes.c_int()
    assert lib.fs_session_poll(None, None, None, 0, ctypes.byref(n)) == -1
    assert lib.fs_session_submit_frame(None, 0, 0, ctypes.c_void_p(0x1000), 0.0) == -1
    assert lib.fs_session_add_markers(None, 0, ctypes.c_void_p(0x1000)) == -1
    assert lib.fs_session_destroy(None) == -1 and lib.fs_session_pending(None) == -1
    t0 = lib.fs_session_clock()
    assert lib.fs_session_clock() >= t0 > 0
    assert lib.fit_spots_strerror(-9) == b"frame queue full, frame rejected"


def test_spot_count_limit(lib):
    """FS_MAX_SPOTS (2^31 - 2^24) leaves the kernels' 32-bit work counters headroom: the
    header's value is the binding's, and every C entry point that takes a spot count
    rejects one spot more before any CUDA work (checked in C, no Python guard on the way)."""
    from paper_2106_02045_gb300 import fitspots
    text = (ROOT / "include" / "fitspots.h").read_text()
    m = re.search(r"#define FS_MAX_SPOTS (\d+)LL", text)
    assert m and int(m.group(1)) == fitspots.MAX_SPOTS == 2**31 - 2**24
    top = fitspots.MAX_SPOTS
    over = top + 1
    fake = ctypes.c_void_p(0x1000)
    assert lib.fit_spots_start(fake, 0, 100, fake, fake, over, 0, fake, None) == -2
    for fn in (lib.fit_spots_explicit, lib.fit_spots_weighted, lib.fit_spots_poisson,
               lib.fit_spots_noalloc):
        assert fn(fake, 0, 100, fake, fake, fake, fake, over, 20, 0.0, 1e-6, 1e-4,
                  fake, fake, fake, fake, fake, fake, None, None) == -2
    # the workspace calls: one spot more is a size error, the limit itself gets as far as
    # the workspace check (dummy pointers, so nothing is ever enqueued)
    assert _call(lib, n=over) == -2
    assert _call(lib, n=top, ws_bytes=272) == -6
    uni = lambda n: lib.fit_spots_uniform(fake, 0, 32, 32, 1, fake, n, 20, 0.0, 1e-6, 1e-4,
                                         fake, fake, fake, fake, fake, fake, None, fake, 16, None)
    assert uni(over) == -2 and uni(top) == -6
    host = lambda n: lib.fit_spots_uniform_host(fake, 0, 32, 32, 1, fake, n, 20, 0.0, 1e-6,
                                                1e-4, fake, fake, fake, fake, fake, fake, None,
                                                1000, fake, 16, None)
    assert host(over) == -2 and host(top) == -6
    bwd = lambda n: lib.fit_spots_backward(fake, 1, 100, fake, fake, fake, n, fake, fake, fake,
                                           fake, None, None, None, None, fake, None)
    assert bwd(over) == -2
    with pytest.raises(fitspots.FitSpotsError, match="at most"):
        fitspots._check_count(over)
    fitspots._check_count(fitspots.MAX_SPOTS)


def test_size_classes_and_configs(lib):
    from paper_2106_02045_gb300 import fitspots
    assert lib.fit_spots_num_classes() == 17
    cfgs = fitspots.configs()
    assert len(cfgs) == lib.fit_spots_num_configs() == 58
    assert sum(c[3] for c in cfgs) == 22 and lib.fit_spots_config_batched(99) == -8
    generic, elong = 56, 57   # one column per lane, each ROI oriented; row blocks for class 16
    assert cfgs[generic] == (32, 1, 32, 1) and cfgs[elong] == (32, 1, 32, 1)
    assert fitspots.config_generic(generic) and fitspots.config_generic(elong)
    assert not fitspots.config_generic(55)
    for cls in range(16):
        wmax, hmax = (cls // 4 + 1) * 8, (cls % 4 + 1) * 8
        usable = [c for c in range(len(cfgs)) if fitspots.config_fits(cls, c)]
        assert usable, cls
        for c in usable:
            L, C, R, batched = cfgs[c]
            if c == generic:   # takes any ROI up to 32 x 32, oriented
                continue
            assert L * C >= wmax and L * C <= 32 and R == hmax and 32 % L == 0
        assert fitspots.get_config(cls) in usable and generic in usable and elong not in usable
    # the elongated class (a side above 32) runs the row-block configuration and nothing else
    assert [c for c in range(len(cfgs)) if fitspots.config_fits(16, c)] == [elong]
    assert fitspots.default_config(16) == elong
    assert lib.fit_spots_set_config(15, 0) == -8          # (4,2,8) cannot hold 32x32
    keep = fitspots.get_config(15)
    other = [c for c in range(len(cfgs)) if fitspots.config_fits(15, c) and c != keep][0]
    fitspots.set_config(15, other)
    assert fitspots.get_config(15) == other
    fitspots.set_config(15, keep)
    assert lib.fit_spots_get_config(17) == -8 and lib.fit_spots_config_info(99, None, None, None) == -8


def test_binding_refuses_cpu_tensors():
    import torch
    from paper_2106_02045_gb300 import fitspots
    x = torch.zeros(100)
    with pytest.raises(fitspots.FitSpotsError):
        fitspots.fit(x, torch.zeros(1, dtype=torch.int64), torch.zeros(1, 2, dtype=torch.int32),
                     torch.zeros(1, 4), torch.zeros(1, dtype=torch.uint8))


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No CPU fallback: with the compiled library absent every call raises."""
    from paper_2106_02045_gb300 import fitspots
    monkeypatch.setattr(fitspots, "LIB", tmp_path / "missing.so")
    monkeypatch.setattr(fitspots, "_lib", None)
    with pytest.raises(fitspots.FitSpotsError, match="missing"):
        fitspots.library()
    with pytest.raises(fitspots.FitSpotsError):
        fitspots.workspace_bytes(10)
