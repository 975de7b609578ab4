"""The multi-rank bookkeeping of bench.py on CPU: two gloo ranks with different times and
work; the job value is all ranks' fits over the slowest rank's time (weak scaling)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, conv = bench.job_totals(10.0 + 5.0 * rank, 1000.0 * (rank + 1), world, "cpu")
    q.put((rank, ms, conv))
    dist.destroy_process_group()


def test_job_totals_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    for rank, ms, conv in got:
        assert ms == 15.0 and conv == 3000.0


def test_job_totals_single_rank_is_identity():
    import bench
    assert bench.job_totals(12.5, 42, 1, "cpu") == (12.5, 42.0)


def test_cpu_baseline_detail_small():
    """The oracle timings of the other workloads and of one core run on the host alone."""
    import bench
    out = bench._cpu_baseline_detail(detail=(("iso15", 200), ("iso16", 200), ("mixed", 300)),
                                      one_core_sample=100)
    assert set(out) == {"iso15", "iso16", "mixed", f"{bench.WORKLOAD}_one_core"}
    for v in out.values():
        assert v["value"] > 0 and v["unit"] == bench.UNIT and v["cores"] >= 1
    assert out[f"{bench.WORKLOAD}_one_core"]["cores"] == 1


def test_reference_arm_prints_one_json_line():
    """``bench.py --impl reference`` (the oracle on the host cores) on a tiny sample: one
    JSON line with the reference keys."""
    import json
    import subprocess
    import sys
    from pathlib import Path
    root = Path(__file__).resolve().parents[1]
    r = subprocess.run([sys.executable, str(root / "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1", "--ref-sample", "300"],
                       capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "fits/s"
    assert d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_paper_protocol_section_with_a_stub(monkeypatch):
    """The paper-protocol bench section's bookkeeping on the host, the library call replaced
    by a stub that checks its arguments and marks every fit converged."""
    import bench
    import torch
    from paper_2106_02045_gb300 import fitspots
    calls = []

    def fake_host(images, W, H, model, init, *, chunk, out, workspace, device, stream):
        n = init.shape[0]
        assert images.numel() == n * W * H and chunk == n and out["state"].shape[0] == n
        assert workspace.numel() >= 256 and model == 0 and W == H
        out["state"][:] = 1
        calls.append((W, n))
        return out

    def fake_alloc(n):
        return {k: torch.zeros(v, dtype=t) for k, (v, t) in dict(
            params=((n, 4), torch.float32), alpha=(n, torch.float32), beta=(n, torch.float32),
            chi2=(n, torch.float32), state=(n, torch.int32), iters=(n, torch.int32),
            evals=(n, torch.int32)).items()}

    class FakeStream:
        def synchronize(self):
            pass

    monkeypatch.setattr(fitspots, "fit_uniform_host", fake_host)
    monkeypatch.setattr(fitspots, "alloc_host_outputs", fake_alloc)
    monkeypatch.setattr(bench, "PAPER_BATCHES", ((10, 3), (100, 2)))
    monkeypatch.setattr(bench, "PAPER_SIZES", (9,))
    out = bench._extra_paper_protocol("cpu", FakeStream(), pin=False)["paper_protocol"]
    assert [(r["S"], r["batch"], r["calls"]) for r in out["rows"]] == [(9, 10, 3), (9, 100, 2)]
    assert all(r["converged_fraction"] == 1.0 and r["fits_per_s"] > 0 for r in out["rows"])
    assert calls == [(9, 10)] * 4 + [(9, 100)] * 3


def test_profile_key_ignores_comments_and_tracks_code(tmp_path):
    """The ncu summaries are tied to the CUDA source by a hash of its code without comments:
    editing a comment keeps the key (and the DRAM traffic the bench reports), changing code
    drops it."""
    import bench
    src = tmp_path / "k.cu"
    src.write_text("// header\nint f(int x) {  // doubled\n  return 2 * x;\n}\n")
    key = bench.code_hash(src)
    src.write_text("// another header\n\nint f(int x) {  // twice x\n  return 2 * x;\n}\n")
    assert bench.code_hash(src) == key
    prof = tmp_path / "p.md"
    prof.write_text(f"code_sha256_16: {key}\ntraffic_bytes_per_full_launch: 123 (x)\n")
    assert bench._traffic_from_profile(prof, src) == 123.0
    src.write_text("int f(int x) {\n  return 3 * x;\n}\n")
    assert bench.code_hash(src) != key
    assert bench._traffic_from_profile(prof, src) is None
