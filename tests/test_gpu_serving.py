"""Serving sessions (fs_session_*): device ROI cut + warm-started fit + resident marker state,
one CUDA graph per batch size, continuous batching across camera streams, admission by
memory, checkpoint / restore, oracle parity of the served fits, real-time latency."""
import numpy as np
import pytest
import torch

from paper_2106_02045_gb300 import serving, synth
from tests.parity import CONVERGED, REL_TOL, XY_TOL

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _stream(n_frames, markers, size, seed):
    cs = synth.make_camera_stream(n_frames, markers, size, size, seed=seed, device=DEV)
    host = torch.empty(cs.frames.shape, dtype=torch.uint16, pin_memory=True)
    host.copy_(cs.frames)
    return cs, host


def _serve_alone(cs, host, markers, size, n, **kw):
    srv = serving.TrackingServer(size, size, markers=markers, sessions=1, device=DEV, **kw)
    srv.set_markers(0, cs.start)
    for k in range(n):
        srv.submit(0, k, host[k], serving.clock())
        srv.drain()
    return srv


def test_tracker_follows_drifting_markers():
    markers, size, n = 32, 512, 40
    cs, host = _stream(n, markers, size, seed=101)
    srv = _serve_alone(cs, host, markers, size, n)
    log = srv.logs[0]
    assert sorted(log.results) == list(range(n))
    truth = cs.truth.cpu().numpy()
    err = np.array([np.hypot(*(log.results[k][:, :2] - truth[k]).T) for k in range(n)])
    states = np.array([log.results[k][:, 7] for k in range(n)])
    print(f"tracking error median {np.median(err):.4f} px, p99 {np.percentile(err, 99):.4f} px")
    assert np.isin(states, (1, 2, 3, 4)).mean() > 0.99
    assert np.median(err) < 0.03 and np.percentile(err, 99) < 0.15


def test_served_fits_match_the_oracle():
    """Every served marker fit, refitted by the FP64 oracle from the same ROI (cut on the host
    at the origin the session reports) and the same warm start: centre within 1e-3 px, sigma,
    alpha and beta within 1e-4 relative, the same convergence class."""
    import oracle
    markers, size, n, roi = 48, 640, 30, 21
    cs, host = _stream(n, markers, size, seed=150)
    srv = _serve_alone(cs, host, markers, size, n, roi=roi)
    frames = host.view(torch.int16).numpy().view(np.uint16)
    pix, init, res = [], [], []
    for k in range(n):
        r = srv.logs[0].results[k]                      # [markers, 16]
        for m in range(markers):
            ox, oy = int(r[m, 8]), int(r[m, 9])
            pix.append(frames[k, oy:oy + roi, ox:ox + roi].ravel())
            init.append(r[m, 10:14])
            res.append(r[m])
    res = np.array(res)
    N = len(pix)
    img = np.concatenate(pix).astype(np.uint16)
    ref = oracle.fit_spots(img, np.arange(N, dtype=np.int64) * roi * roi,
                           np.tile([roi, roi], (N, 1)), np.array(init, np.float32),
                           np.zeros(N, np.uint8))
    conv, rconv = np.isin(res[:, 7], CONVERGED), np.isin(ref["state"], CONVERGED)
    both = conv & rconv
    xy = np.abs(res[:, :2] - res[:, 8:10] - ref["params"][:, :2]).max(1)
    rel = lambda a, b: np.abs(a - b) / np.abs(b)
    ok = ((xy < XY_TOL) & (rel(res[:, 2], ref["params"][:, 2]) < REL_TOL) &
          (rel(res[:, 4], ref["alpha"]) < REL_TOL) & (rel(res[:, 5], ref["beta"]) < REL_TOL))
    print(f"served fits: {N}, class agreement {np.mean(conv == rconv):.5f}, "
          f"within the bar {ok[both].mean():.5f}")
    assert np.mean(conv == rconv) >= 0.999
    assert ok[both].mean() >= 0.999


def test_results_are_the_same_alone_and_in_the_mix():
    """Stream 0 served alone, then together with three other streams whose frames arrive
    staggered and are batched with its frames: identical results, bit for bit."""
    markers, size, n = 24, 384, 24
    streams = [_stream(n, markers, size, seed=200 + s) for s in range(4)]
    alone = _serve_alone(streams[0][0], streams[0][1], markers, size, n).logs[0].results

    srv = serving.TrackingServer(size, size, markers=markers, sessions=4, frame_slots=6,
                                 queue_limit=1024, device=DEV)
    for s in range(4):
        srv.set_markers(s, streams[s][0].start)
    # staggered arrivals: stream s starts s rounds late; each round brings the next frame
    # of every started stream while earlier batches may still be on the device
    for r in range(n + 4):
        for s in range(4):
            k = r - s
            if 0 <= k < n:
                srv.submit(s, k, streams[s][1][k], serving.clock())
        for _ in range(3):
            srv.step()
    srv.drain()
    st = srv.stats()
    assert st["batches"] < st["served"]       # frames of different streams shared batches
    assert st["dropped"] == 0 and st["served"] == 4 * n
    mixed = srv.logs[0].results
    for k in range(n):
        assert np.array_equal(alone[k].view(np.int32), mixed[k].view(np.int32)), k
    for s in range(1, 4):
        assert sorted(srv.logs[s].results) == list(range(n))


def test_admission_rejects_beyond_queue_and_checkpoint_restores():
    markers, size, n = 16, 256, 12
    cs, host = _stream(n, markers, size, seed=300)
    srv = serving.TrackingServer(size, size, markers=markers, sessions=1, frame_slots=2,
                                 queue_limit=3, device=DEV)
    srv.set_markers(0, cs.start)
    accepted = [srv.submit(0, k, host[k], serving.clock()) for k in range(n)]
    assert sum(accepted) == 3 and srv.dropped == n - 3
    srv.drain()
    assert len(srv.logs[0].results) == 3
    # checkpoint, serve two frames, restore, serve them again: same results
    snap = srv.snapshot(0)
    for k in (3, 4):
        srv.submit(0, k, host[k], serving.clock())
        srv.drain()
    first = {k: srv.logs[0].results[k].copy() for k in (3, 4)}
    srv.restore(0, snap)
    for k in (3, 4):
        srv.submit(0, k, host[k], serving.clock())
        srv.drain()
    for k in (3, 4):
        assert np.array_equal(first[k], srv.logs[0].results[k])


def _realtime_run(queue_limit: int = 1024) -> dict:
    """Serve the 2048 x 2048 / 2000 fps / 64-marker stream (1,000 warm-up frames, then
    20,000) and return the latency summary of the timed frames and the drop count."""
    markers, size, ring, warm, n = 64, 2048, 128, 1000, 20000
    cs, host = _stream(ring, markers, size, seed=400)
    srv = serving.TrackingServer(size, size, markers=markers, sessions=1,
                                 queue_limit=queue_limit, device=DEV)
    srv.set_markers(0, cs.start)
    serving.run_stream(srv, 0, host, warm + n, fps=2000.0)
    log = srv.logs[0]
    lat = np.array([log.latency[k] for k in range(warm, warm + n) if k in log.latency])
    summ = serving.latency_summary(lat)
    summ["dropped"] = int(srv.dropped)
    srv.close()
    return summ


def test_realtime_stream_latency_2048():
    """The camera workload: 2048 x 2048 uint16 frames at 2000 fps, 64 markers, 21 x 21 ROIs,
    20,000 frames after 1,000 warm-up frames: every frame served, the median latency (host
    arrival stamp -> results on the host) inside the 0.5 ms frame period and the 99th
    percentile within ten periods. The stream is served by a process of its own, as a
    deployment would run it: inside this long test process (after the other tests) the host
    loop was measured to stall for up to ~0.1 s at a time, which is the test process, not
    the session. The admission queue holds 1,024 frames (0.5 s of the stream; queued frames
    cost host pointers only)."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import json; from tests.test_gpu_serving import _realtime_run; "
            "print('RESULT ' + json.dumps(_realtime_run()))")
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    summ = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")][-1][7:])
    print("realtime 2048^2 at 2000 fps:", summ)
    assert summ["dropped"] == 0 and summ["frames"] == 20000
    assert summ["p50_ms"] < 0.5 and summ["p99_ms"] < 5.0
