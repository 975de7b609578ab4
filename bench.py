"""Benchmark: converged 2-D Gaussian fits per second on the 32x32 workload.

One step = one batched fit of 1,000,000 spots (32x32 uint16 ROIs, elliptic model, seeded
synthetic camera data) through ``fit_spots_uniform``, inputs resident in HBM (2 GB, larger
than L2, so no flush is needed between steps). The JSON line reports:

* value        converged fits per second, kernel timed with CUDA events on its stream
* e2e          the same metric through the host-buffer call (fit_spots_uniform_host) from
               pinned host memory: the H2D copies of the step's pixels and start values and
               the D2H copies of all per-spot results are inside the timed region,
               overlapped with the fits chunk by chunk
* roofline     the fit kernel against the FP32 FMA rate measured in this run
               (fit_spots_probe_rates), counting the work of a per-pixel evaluation of the
               method: 12 FP32 operations per pixel per evaluated point and 26 more per pixel
               at each gradient point (elliptic model); `separable` repeats it with the 7
               operations per pixel per evaluated point that the separable kernel cannot
               avoid, `sfu` the exponentials against the measured MUFU rate
* paper_protocol  the paper's own throughput protocol (batches of 10..10,000 9x9 and 32x32
               fits per call, host data to host results) through the host-buffer call, as
               context for the paper's printed fits/s
* cpu_baseline the FP64 oracle on the host cores, timed on a bounded sample of spots;
               other_workloads adds the 15x15, 16x16 and mixed workloads (all cores) and
               the 32x32 workload on one core

``--impl reference`` times the oracle itself as the reference arm (host cores only).
Under torchrun every rank fits its own 1,000,000 spots (weak scaling, no collective on
the data path); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "converged fits/s at 32x32 ROI (frac of roofline); p50/p99 frame latency"
UNIT = "fits/s"
WORKLOAD = "ell32"
W = H = 32
N_SPOTS = 1_000_000
OPS_PER_PIXEL_EVAL = 7          # separable kernel: FP32 ops per pixel per evaluated point
C_V, C_D = 12, 26               # per-pixel evaluation (elliptic): per point, per gradient point
SMS, LANES_PER_SM = 152, 128
CONVERGED = (1, 2, 3, 4)
PROFILE = ROOT / "profiles" / "fit_kernel_ell32.md"
SOURCE = ROOT / "paper_2106_02045_gb300" / "csrc" / "fitspots.cu"
E2E_CHUNK = 125_000   # spots per chunk of the host-buffer call (8 chunks per 1,000,000)
BWD_SOURCE = ROOT / "paper_2106_02045_gb300" / "csrc" / "backward.cu"
BWD_PROFILE = ROOT / "profiles" / "backward_iso16.md"


def _dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _config(n_gpus: int, n_spots: int = N_SPOTS) -> dict:
    return {"workload": f"{WORKLOAD}: {n_spots:,} spots per GPU, {W}x{H} uint16 ROIs, elliptic "
                        "Gaussian, photons log-U(200,20000), background U(50,500)+100, "
                        "Poisson + 2 e- read noise, LM <= 20 iterations",
            "global_batch": n_spots * n_gpus, "roi": f"{W}x{H}", "model": "elliptic",
            "tolerances": {"max_error": 0.0, "min_delta": 1e-6, "min_step": 1e-4},
            "l2": "inputs (2 GB/GPU) larger than L2; no flush",
            "parallelism": f"dp{n_gpus}" if n_gpus > 1 else "single GPU"}


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        try:
            for line in open(self.path):
                f = [v.strip() for v in line.split(",")]
                if len(f) < 7:
                    continue
                try:
                    sm.append(float(f[0]))
                    mx.append(float(f[1]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[3:7]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        finally:
            os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _kernel_name(size_class: int) -> str:
    """The kernel a size class runs under the current configuration table."""
    from paper_2106_02045_gb300 import fitspots
    L, C, R, batched = fitspots.configs()[fitspots.get_config(size_class)]
    return f"fit_kernel{'_batched' if batched else ''}<{L},{C},{R}>"


def code_hash(source: Path) -> str:
    """First 16 hex digits of the SHA-256 of a CUDA source with its // comments and blank
    lines removed: the key that ties an ncu summary to the code it measured, so that edits
    of comments alone do not orphan a profile."""
    import re
    lines = (re.sub(r"//.*$", "", ln).rstrip() for ln in source.read_text().splitlines())
    return hashlib.sha256("\n".join(ln for ln in lines if ln).encode()).hexdigest()[:16]


def _traffic_from_profile(profile=None, source=None) -> float | None:
    """DRAM bytes per launch from the committed ncu summary, if it was taken on this source."""
    profile = PROFILE if profile is None else profile
    source = SOURCE if source is None else source
    if not profile.exists():
        return None
    sha = code_hash(source)
    per_launch, src = None, None
    for line in profile.read_text().splitlines():
        if line.startswith("traffic_bytes_per_full_launch:"):
            per_launch = float(line.split(":", 1)[1].split()[0])
        if line.startswith("code_sha256_16:"):
            src = line.split(":", 1)[1].strip()
    return per_launch if (src == sha and per_launch is not None) else None


def _cpu_baseline(batch_cpu, n_sample: int) -> dict:
    import oracle
    from paper_2106_02045_gb300 import synth
    import numpy as np
    sub = batch_cpu
    d = sub.numpy()
    img = synth.as_numpy_images(sub)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    ref = oracle.fit_spots(img, d["offsets"], d["dims"], d["init"], d["model"], nthreads=cores)
    dt = time.perf_counter() - t0
    conv = int(np.isin(ref["state"], CONVERGED).sum())
    return {"value": conv / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {n_sample:,} spots of the {WORKLOAD} workload, FP64 oracle, "
                      f"{dt:.1f} s"}


# the other workloads the oracle is timed on (all host cores), and the one-core sample
CPU_DETAIL = (("iso15", 10_000), ("iso16", 50_000), ("mixed", 50_000))
CPU_ONE_CORE_SAMPLE = 5_000


def _cpu_baseline_detail(detail=CPU_DETAIL, one_core_sample: int = CPU_ONE_CORE_SAMPLE) -> dict:
    """The FP64 oracle's converged fits/s on the other workloads (all host cores, each with
    the tolerances its GPU section uses) and on the 32x32 workload with one core."""
    import numpy as np
    import oracle
    from paper_2106_02045_gb300 import synth
    cores = os.cpu_count() or 1

    def timed(b, nthreads, **kw):
        d = b.numpy()
        img = synth.as_numpy_images(b)
        t0 = time.perf_counter()
        r = oracle.fit_spots(img, d["offsets"], d["dims"], d["init"], d["model"],
                             nthreads=nthreads, **kw)
        dt = time.perf_counter() - t0
        return int(np.isin(r["state"], CONVERGED).sum()) / dt, dt

    out = {}
    for name, n in detail:
        b = synth.make_workload(name, n, device="cpu")
        kw = dict(max_iter=50, min_delta=0.0, min_step=1e-6) if name == "iso16" else {}
        v, dt = timed(b, cores, **kw)
        out[name] = {"value": v, "unit": UNIT, "cores": cores,
                     "sample": f"{b.n:,} spots of the {name} workload, {dt:.2f} s"}
    b = synth.make_workload(WORKLOAD, one_core_sample, device="cpu")
    v, dt = timed(b, 1)
    out[f"{WORKLOAD}_one_core"] = {"value": v, "unit": UNIT, "cores": 1,
                                   "sample": f"{b.n:,} spots of the {WORKLOAD} workload, "
                                             f"{dt:.2f} s"}
    return out


def run_reference(args) -> None:
    """The reference arm: the FP64 oracle on the host cores, same workload and metric."""
    world, rank, _ = _dist_env()
    if rank != 0:
        return
    import numpy as np
    import oracle
    from paper_2106_02045_gb300 import synth
    n = args.ref_sample
    b = synth.make_workload(WORKLOAD, n, device="cpu")
    d = b.numpy()
    img = synth.as_numpy_images(b)
    cores = os.cpu_count() or 1
    oracle.build()
    for _ in range(args.warmup):
        oracle.fit_spots(img, d["offsets"], d["dims"], d["init"], d["model"], nthreads=cores)
    times, conv = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.fit_spots(img, d["offsets"], d["dims"], d["init"], d["model"], nthreads=cores)
        times.append(time.perf_counter() - t0)
        conv = int(np.isin(r["state"], CONVERGED).sum())
    tot = sum(times)
    value = conv * args.steps / tot
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference", "config": _config(world),
            "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": cores,
                             "sample": f"{n:,} spots of the {WORKLOAD} workload per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run(args) -> None:
    import numpy as np
    import torch
    import torch.distributed as dist

    world, rank, local = _dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_02045_gb300 import fitspots, synth

    # roofline denominators, measured on this GPU before the timed region
    rates = fitspots.probe_rates(dev)
    n_spots = args.spots
    b = synth.make_workload(WORKLOAD, n_spots, device=dev)
    if rank > 0:   # each rank its own draw of the workload
        b = synth.make_ell32(n_spots, seed=synth.SEED_BASE + 2 + 1000 * rank, device=dev)
    out = fitspots.alloc_outputs(n_spots, dev)
    ws = torch.empty(max(int(fitspots.library().fit_spots_uniform_workspace()), 16),
                     dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        fitspots.fit_uniform(b.images, W, H, synth.MODEL_ELLIPTIC, b.init, out=out,
                             workspace=ws, stream=stream)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(max(args.warmup, 3)):
        step()
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with ClockSampler(dev.index) as clk:
        barrier()
        t_all0 = torch.cuda.Event(enable_timing=True)
        t_all1 = torch.cuda.Event(enable_timing=True)
        t_all0.record(stream)
        for e0, e1 in ev:
            e0.record(stream)
            step()
            e1.record(stream)
        t_all1.record(stream)
        barrier()
    clocks = clk.summary()
    ms_total = t_all0.elapsed_time(t_all1)
    kernel_ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    state = out["state"]
    conv = int(torch.isin(state, torch.tensor(CONVERGED, device=dev, dtype=torch.int32)).sum())
    evals = int(out["evals"].sum())
    iters = int(out["iters"].sum())
    launches = args.steps  # one fit kernel per step (plus one workspace memset)

    ms_job, conv_job = job_totals(ms_total, conv, world, dev)
    value = conv_job * args.steps / (ms_job * 1e-3)

    # ---------------------------------------------------------------- end to end
    e2e = _e2e(args, b, out, ws, stream, barrier, world, dev) if not args.no_e2e else None

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    # ---------------------------------------------------------------- roofline
    kernel_s = statistics.mean(kernel_ms) * 1e-3
    peak = rates["ffma"]
    ops_direct = float(evals * C_V + iters * C_D) * W * H
    ops_sep = float(evals) * W * H * OPS_PER_PIXEL_EVAL
    exps_sep = float(evals) * (W + H)
    traffic = _traffic_from_profile()
    if traffic is not None:
        traffic *= n_spots / N_SPOTS
    roofline = {"bound": "alu", "achieved": ops_direct / kernel_s / 1e12, "peak": peak / 1e12,
                "unit": "T lane-op/s", "frac": ops_direct / kernel_s / peak, "traffic": traffic,
                "ops_definition": f"{C_V} FP32 ops (FMA = 1) per pixel per evaluated point + "
                                  f"{C_D} per pixel per gradient point (one per LM iteration): "
                                  "the work of a per-pixel evaluation of the method, elliptic",
                "ops_per_launch": ops_direct, "evals_per_spot": evals / n_spots,
                "iters_per_spot": iters / n_spots,
                "peak_source": "measured in this run: FP32 FMA chains on every SM "
                               "(fit_spots_probe_rates), 'of measured'",
                "separable": {"frac": ops_sep / kernel_s / peak,
                              "achieved": ops_sep / kernel_s / 1e12,
                              "ops_definition": f"{OPS_PER_PIXEL_EVAL} FP32 ops per pixel per "
                                                "evaluated point: the separable evaluation's "
                                                "unavoidable work"},
                "sfu": {"frac": exps_sep / kernel_s / rates["ex2"],
                        "achieved": exps_sep / kernel_s / 1e12, "peak": rates["ex2"] / 1e12,
                        "ops_definition": "W + H exponentials per evaluated point (separable)"},
                "fp64_peak": rates["dfma"] / 1e12,
                "kernel": _kernel_name(15)}
    cpu = None
    if not args.no_cpu_baseline:
        bcpu = b.head(args.cpu_sample).to("cpu")
        cpu = _cpu_baseline(bcpu, args.cpu_sample)
        cpu["other_workloads"] = _cpu_baseline_detail()
    extras = {} if args.no_extras else _extras(args, dev, set(args.extras.split(",")))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms_job / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": _config(world, n_spots), "clocks": clocks,
            "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu,
            "fits_per_step": n_spots * world, "converged_fraction": conv / n_spots}
    line.update(extras)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def job_totals(ms: float, converged: float, world: int, device) -> tuple[float, float]:
    """Whole-job time and work: the slowest rank's time (MAX) and all ranks' converged
    fits (SUM). No collective touches the fit data; the ranks' spots are independent."""
    if world <= 1:
        return float(ms), float(converged)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    c = torch.tensor([float(converged)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), float(c.item())


def _timed(fn, steps, stream):
    """Mean CUDA-event time (ms) of fn() over `steps` runs on `stream`, after 3 warm-ups."""
    import torch
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _extras(args, dev, which=("mixed", "backward", "serving", "start")) -> dict:
    """The other hot-path rows on their workloads: mixed sizes, backward, serving, start
    values."""
    import torch
    stream = torch.cuda.current_stream(dev)
    out = {}
    hbm = 6691.8
    try:
        hbm = float(json.loads((ROOT / "MEASURED_PEAKS.json").read_text())["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        pass
    if "mixed" in which:
        out.update(_extra_mixed(args, dev, stream))
    if "backward" in which:
        out.update(_extra_backward(dev, stream, hbm))
    if "serving" in which:
        out.update(_extra_serving(args, dev))
    if "start" in which:
        out.update(_extra_start(dev, stream, hbm))
    if "table1" in which:
        out.update(_extra_table1(dev, stream))
    if "explicit" in which:
        out.update(_extra_explicit(dev, stream))
    if "weighted" in which:
        out.update(_extra_weighted(dev, stream))
    if "background" in which:
        out.update(_extra_background(dev, stream, hbm))
    if "paper_protocol" in which:
        # last, and guarded: a failure of this context section must not cost the line
        try:
            out.update(_extra_paper_protocol(dev, stream))
        except Exception as e:  # noqa: BLE001
            out["paper_protocol"] = {"error": f"{type(e).__name__}: {e}"}
    return out


# the paper's throughput protocol (Results): batch sizes and how many calls each gets
PAPER_BATCHES = ((10, 200), (100, 20), (1_000, 10), (10_000, 1))
PAPER_SIZES = (9, 32)


def _extra_paper_protocol(dev, stream, pin: bool = True) -> dict:
    """The paper's throughput protocol (Results section): batches of 10 / 100 / 1,000 / 10,000
    fits of S x S spots (400 signal, 40 background counts), called 200 / 20 / 10 / 1 times,
    each call timed from host data to host results. Here through the public host-buffer
    call (one chunk per call: upload, fit, download), host wall clock per call including
    the binding's Python overhead, median over the calls after one warm-up call."""
    import numpy as np
    import torch
    from paper_2106_02045_gb300 import fitspots, synth
    nmax = max(b for b, _ in PAPER_BATCHES)
    rows = []
    for S in PAPER_SIZES:
        b = synth.make_paper(nmax, S, 400.0, 40.0, seed=synth.SEED_BASE + 40 + S)
        h_img = torch.empty(b.images.shape, dtype=b.images.dtype, pin_memory=pin)
        h_img.copy_(b.images)
        h_init = torch.empty(b.init.shape, dtype=b.init.dtype, pin_memory=pin)
        h_init.copy_(b.init)
        h_out = fitspots.alloc_host_outputs(nmax)
        ws = torch.empty(max(fitspots.host_workspace_bytes(nmax, S, S, fitspots.F32), 256),
                         dtype=torch.uint8, device=dev)
        for batch, calls in PAPER_BATCHES:
            o = {k: v[:batch] for k, v in h_out.items()}
            times = []
            for _ in range(calls + 1):
                t0 = time.perf_counter()
                fitspots.fit_uniform_host(h_img[:batch * S * S], S, S, synth.MODEL_ISO,
                                          h_init[:batch], chunk=batch, out=o, workspace=ws,
                                          device=dev, stream=stream)
                stream.synchronize()
                times.append(time.perf_counter() - t0)
            t = statistics.median(times[1:])
            conv = int(np.isin(o["state"].numpy(), CONVERGED).sum())
            rows.append({"S": S, "batch": batch, "calls": calls, "ms_per_call": t * 1e3,
                         "fits_per_s": batch / t, "converged_fraction": conv / batch})
    return {"paper_protocol": {
        "what": "batches of 10..10,000 S x S fits (400:40 counts) per call, host data to host "
                "results, fit_spots_uniform_host, median host wall clock per call",
        "rows": rows,
        "paper_context": "Quadro P600 under MATLAB: about 1e5 fits/s at batch 100 and 4e5 at "
                         "1,000 or more for 7-12 px ROIs; about 0.5 ms per call for small "
                         "batches (other hardware; context, not a target)"}}


def _extra_weighted(dev, stream) -> dict:
    """Unweighted, variance-weighted and Poisson-likelihood implicit fits of the same 100,000
    iso15 spots (peak 1000, background 100): time, and centre and width errors in units of
    the true sigma."""
    import numpy as np
    from paper_2106_02045_gb300 import fitspots, synth
    b = synth.make_iso(100_000, 15, 7.0, synth.SEED_BASE + 51, device=dev, name="iso15")
    t = b.truth["params"].cpu().numpy()
    res = {}
    o = fitspots.alloc_outputs(b.n, dev)
    ws = _fit_workspace(b.n, dev)
    for name, run in (("unweighted", lambda: fitspots.fit_batch(b, out=o, workspace=ws,
                                                                  stream=stream)),
                      ("weighted", lambda: fitspots.fit_weighted(b.images, b.offsets, b.dims,
                                                                 b.init, b.model, out=o,
                                                                 stream=stream)),
                      ("poisson", lambda: fitspots.fit_poisson(b.images, b.offsets, b.dims,
                                                               b.init, b.model, out=o,
                                                               stream=stream))):
        ms = _timed(run, 3, stream)
        p = o["params"].cpu().numpy().astype(np.float64)
        c = np.isin(o["state"].cpu().numpy(), CONVERGED)
        res[name] = {"ms": ms, "converged": float(c.mean()),
                     "x_err_rms": float(np.sqrt(np.mean(((p[c, 0] - t[c, 0]) / t[c, 2]) ** 2))),
                     "sigma_err_rms": float(np.sqrt(np.mean(((p[c, 2] - t[c, 2]) / t[c, 2]) ** 2)))}
    return {"weighted": {"workload": "iso15-like: 100,000 spots of 15x15, peak 1000, background "
                                     "100, Poisson", **res}}


def _extra_explicit(dev, stream) -> dict:
    """Implicit against explicit amplitudes on the same 262,144 ell32 spots: time, LM
    iterations and evaluated points per spot, share stopped by the iteration budget."""
    import torch
    from paper_2106_02045_gb300 import fitspots, synth
    b = synth.make_workload("ell32", 262_144, device=dev)
    conv = torch.tensor(CONVERGED, device=dev, dtype=torch.int32)
    res = {}
    oi = fitspots.alloc_outputs(b.n, dev)
    ws = _fit_workspace(b.n, dev)
    ms = _timed(lambda: fitspots.fit_batch(b, out=oi, workspace=ws, stream=stream), 3, stream)
    oe = fitspots.alloc_outputs(b.n, dev)
    mse = _timed(lambda: fitspots.fit_explicit(b.images, b.offsets, b.dims, b.init, b.model,
                                               out=oe, stream=stream), 3, stream)
    for name, o, t in (("implicit", oi, ms), ("explicit", oe, mse)):
        c = torch.isin(o["state"], conv)
        res[name] = {"ms": t, "converged": float(c.float().mean()),
                     "iters_per_spot": float(o["iters"].float().mean()),
                     "evals_per_spot": float(o["evals"].float().mean()),
                     "at_iteration_budget": float((o["state"] == 0).float().mean())}
    return {"explicit": {"workload": "ell32: 262,144 spots, the same start values, damping and "
                                     "stop tests for both methods", **res}}


def _extra_table1(dev, stream) -> dict:
    """The paper's accuracy protocol (Results section, Table 1): 100,000 fits of 9x9 spots
    per row, timed, with the absolute centre and width errors in units of the true sigma."""
    import numpy as np
    from paper_2106_02045_gb300 import fitspots, synth
    golden = ROOT / "tests" / "golden" / "table1_fit2dgaussian.txt"
    rows = [[float(v) for v in line.split()] for line in golden.read_text().splitlines()
            if line.strip() and not line.startswith("#")]
    res = []
    for k, (sig, bg, *ref) in enumerate(rows):
        b = synth.make_paper(100_000, 9, sig, bg, seed=synth.SEED_BASE + 10 + k, device=dev)
        out = fitspots.alloc_outputs(b.n, dev)
        ws = _fit_workspace(b.n, dev)
        ms = _timed(lambda: fitspots.fit_batch(b, out=out, workspace=ws, stream=stream), 3, stream)
        p = out["params"].cpu().numpy().astype(np.float64)
        t = b.truth["params"].cpu().numpy()
        st = t[:, 2]
        ex = np.concatenate([np.abs(p[:, 0] - t[:, 0]), np.abs(p[:, 1] - t[:, 1])])
        ex /= np.concatenate([st, st])
        es = np.abs(np.abs(p[:, 2]) - st) / st
        it = out["iters"].cpu().numpy()
        res.append({"signal": sig, "background": bg, "ms": ms, "fits_per_s": b.n / (ms * 1e-3),
                    "x_err_median_mean_std": [float(np.median(ex)), float(ex.mean()), float(ex.std())],
                    "sigma_err_median_mean_std": [float(np.median(es)), float(es.mean()), float(es.std())],
                    "paper_x": ref[:3], "paper_sigma": ref[3:],
                    "iters_4_or_5": float(np.mean((it == 4) | (it == 5)))})
    return {"table1": {"workload": "paper protocol: 100,000 fits of 9x9 isotropic spots per row",
                       "rows": res}}


def _fit_workspace(n, dev):
    import torch
    from paper_2106_02045_gb300 import fitspots
    return torch.empty(fitspots.workspace_bytes(n), dtype=torch.uint8, device=dev)


def _extra_start(dev, stream, hbm) -> dict:
    import torch
    from paper_2106_02045_gb300 import fitspots, synth
    # start values on the device for the 1,000,000 ell32 ROIs (uint16), both rules
    b = synth.make_workload("ell32", None, device=dev)
    init = torch.empty((b.n, 4), dtype=torch.float32, device=dev)
    res = {}
    nbytes = b.n * (32 * 32 * 2 + 16 + 12)
    for rule, name in ((fitspots.START_CENTROID, "centroid"), (fitspots.START_PAPER, "paper")):
        ms = _timed(lambda: fitspots.start_values(b.images, b.offsets, b.dims, rule, out=init,
                                                  stream=stream), 5, stream)
        res[name] = {"ms_per_step": ms, "value": b.n / (ms * 1e-3), "unit": "spots/s",
                     "roofline": {"bound": "hbm", "achieved": nbytes / (ms * 1e-3) / 1e9,
                                  "peak": hbm, "unit": "GB/s",
                                  "frac": nbytes / (ms * 1e-3) / 1e9 / hbm,
                                  "bytes_per_spot": 32 * 32 * 2 + 16 + 12}}
    del b, init
    return {"start": {"workload": "ell32: 1,000,000 ROIs of 32x32 uint16, start values on the "
                                  "device (fit_spots_start)", **res}}


def _extra_background(dev, stream, hbm) -> dict:
    """Local background pre-subtraction on the tilted workload (1,000,000 ROIs of 21 x 21
    uint16 on tilted planes): the subtraction pass against HBM, then the fit of the
    subtracted float32 spots, and the centre errors with and without the subtraction."""
    import numpy as np
    import torch
    from paper_2106_02045_gb300 import fitspots, synth
    b = synth.make_workload("tilted", None, device=dev)
    N = 21 * 21
    sub = torch.zeros(b.images.numel(), dtype=torch.float32, device=dev)
    plane = torch.empty((b.n, 3), dtype=torch.float32, device=dev)
    per_spot = N * (2 + 4) + 16 + 12       # pixels in and out, offset + dims, plane
    ms = _timed(lambda: fitspots.subtract_background(b.images, b.offsets, b.dims, out=sub,
                                                     plane=plane, stream=stream), 5, stream)
    gbs = b.n * per_spot / (ms * 1e-3) / 1e9
    res = {"subtract": {"ms_per_step": ms, "value": b.n / (ms * 1e-3), "unit": "ROIs/s",
                        "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm,
                                     "unit": "GB/s", "frac": gbs / hbm,
                                     "bytes_per_roi": per_spot}}}
    t = b.truth["params"].cpu().numpy()
    tilt = b.truth["tilt"].cpu().numpy()
    o = fitspots.alloc_outputs(b.n, dev)
    ws = _fit_workspace(b.n, dev)
    for name, imgs in (("fit_subtracted", sub), ("fit_raw", b.images)):
        ms_f = _timed(lambda: fitspots.fit(imgs, b.offsets, b.dims, b.init, b.model, out=o,
                                           workspace=ws, stream=stream), 3, stream)
        p = o["params"].cpu().numpy().astype(np.float64)
        c = np.isin(o["state"].cpu().numpy(), CONVERGED)
        e = p[c, :2] - t[c, :2]
        res[name] = {"ms_per_step": ms_f, "converged": float(c.mean()),
                     "x_err_rms_px": float(np.sqrt(np.mean(e[:, 0] ** 2))),
                     "x_err_slope_corr": float(np.corrcoef(e[:, 0], tilt[c, 0])[0, 1])}
    del b, sub, plane, o, ws
    return {"background": {"workload": "tilted: 1,000,000 ROIs of 21x21 uint16, peak 800 on "
                                       "background planes U(150, 400) + U(-6, 6) counts/px "
                                       "slopes, Poisson noise; border ring width 1", **res}}


def _extra_mixed(args, dev, stream) -> dict:
    import torch
    from paper_2106_02045_gb300 import fitspots, synth
    from paper_2106_02045_gb300.autotune import class_of as autotune_class
    out = {}
    # mixed sizes 5..32, both models, 2,000,000 spots (fit_spots with the size-class prepass)
    mb = synth.make_workload("mixed", args.mixed_spots, device=dev)
    mo = fitspots.alloc_outputs(mb.n, dev)
    mws = torch.empty(fitspots.workspace_bytes(mb.n), dtype=torch.uint8, device=dev)
    ms = _timed(lambda: fitspots.fit_batch(mb, out=mo, workspace=mws, stream=stream), 3, stream)
    conv = int(torch.isin(mo["state"], torch.tensor(CONVERGED, device=dev, dtype=torch.int32)).sum())
    out["mixed"] = {"workload": f"mixed: {mb.n:,} spots, W,H ~ U{{5..32}}, models 50/50, FP32",
                    "value": conv / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                    "fit_launches_per_step": 1,
                    "launches_per_step": "memset + 3 prepass kernels + one persistent fit launch "
                                         "for all size classes"}
    # the plain form: the same prepass, then one persistent launch per size class in use
    pcs = _timed(lambda: fitspots.fit_batch(mb, out=mo, workspace=mws, stream=stream,
                                            per_class=True), 3, stream)
    used = int(torch.unique(torch.tensor([autotune_class(int(w), int(h)) for w, h in
                                          torch.unique(mb.dims, dim=0).tolist()])).numel())
    out["mixed"]["one_launch_per_class"] = {
        "ms_per_step": pcs, "fit_launches_per_step": used, "single_launch_speedup": pcs / ms,
        "what": "fit_spots_per_class: the same prepass and kernels, one persistent launch per "
                "size class in use"}
    # the plain form: per-spot kernels (every lane group runs its own spot's LM step, no
    # slots), one launch per size class, each class on the per-spot twin of its batched
    # configuration (same lanes x columns x rows)
    keep = [fitspots.get_config(c) for c in range(16)]
    cfgs = fitspots.configs()
    try:
        for c in range(16):
            L, C, R, _ = cfgs[keep[c]]
            twin = [i for i, (l, cc, r, bt) in enumerate(cfgs)
                    if (l, cc, r) == (L, C, R) and not bt and fitspots.config_fits(c, i)]
            if twin:
                fitspots.set_config(c, twin[0])
        plain = _timed(lambda: fitspots.fit_batch(mb, out=mo, workspace=mws, stream=stream,
                                                  per_class=True), 3, stream)
    finally:
        for c, k in enumerate(keep):
            fitspots.set_config(c, k)
    out["mixed"]["plain_per_class"] = {
        "ms_per_step": plain, "fit_launches_per_step": used, "single_launch_speedup": plain / ms,
        "what": "per-spot kernels (LM step run by every lane group for its own spot, no "
                "slots), one launch per size class, same geometry as the batched defaults"}
    # elongated ROIs (a side above 32, at most 1024 pixels) through the same single launch
    eb = synth.make_workload("elongated", None, device=dev)
    eo = fitspots.alloc_outputs(eb.n, dev)
    ews = torch.empty(fitspots.workspace_bytes(eb.n), dtype=torch.uint8, device=dev)
    ems = _timed(lambda: fitspots.fit_batch(eb, out=eo, workspace=ews, stream=stream), 3, stream)
    econv = int(torch.isin(eo["state"], torch.tensor(CONVERGED, device=dev, dtype=torch.int32)).sum())
    out["elongated"] = {"workload": f"elongated: {eb.n:,} spots, 64x16 .. 341x3 and transposes, "
                                    "both models, FP32", "value": econv / (ems * 1e-3),
                        "unit": UNIT, "ms_per_step": ems,
                        "converged_fraction": econv / eb.n}
    del eb, eo, ews
    # autotuned: every usable configuration timed per size class on a 131,072-spot sample;
    # the table drives the per-class launches (the single launch always runs the generic
    # kernel), so the tuned table is timed through fit_spots_per_class
    from paper_2106_02045_gb300 import autotune
    t0 = time.perf_counter()
    tuned = autotune.autotune(n=131072, reps=2, dtype=fitspots.F32, device=dev)
    tune_s = time.perf_counter() - t0
    ams = _timed(lambda: fitspots.fit_batch(mb, out=mo, workspace=mws, stream=stream,
                                            per_class=True), 3, stream)
    aconv = int(torch.isin(mo["state"], torch.tensor(CONVERGED, device=dev, dtype=torch.int32)).sum())
    out["mixed"]["autotuned"] = {"value": aconv / (ams * 1e-3), "ms_per_step": ams,
                                 "tuning_s": tune_s, "call": "fit_spots_per_class",
                                 "configs": {c: fitspots.configs()[r["config"]]
                                             for c, r in tuned.items()}}
    autotune.defaults()
    del mb, mo, mws
    return out


def _extra_backward(dev, stream, hbm) -> dict:
    import torch
    from paper_2106_02045_gb300 import fitspots, synth
    # backward: 262,144 spots of 16x16, implicit-function-theorem VJP
    bb = synth.make_workload("iso16", None, device=dev)
    fo = fitspots.fit_batch(bb, max_iter=50, min_delta=0.0, min_step=1e-6)
    gen = torch.Generator(device=dev).manual_seed(7)
    up = [torch.randn(bb.n, 4, generator=gen, device=dev)] + \
         [torch.randn(bb.n, generator=gen, device=dev) for _ in range(3)]
    gimg = torch.zeros(bb.images.numel(), dtype=torch.float32, device=dev)
    bms = _timed(lambda: fitspots.backward(bb.images, bb.offsets, bb.dims, bb.model, fo, *up,
                                           grad_images=gimg, stream=stream), 10, stream)
    nbytes = bb.n * (256 * 8 + 73)
    out_b = {"workload": f"iso16: {bb.n:,} spots, 16x16 FP32, isotropic, VJP of all "
                                   "outputs w.r.t. all pixels",
                       "value": bb.n / (bms * 1e-3), "unit": "spots/s", "ms_per_step": bms,
                       "roofline": {"bound": "hbm", "achieved": nbytes / (bms * 1e-3) / 1e9,
                                    "peak": hbm, "unit": "GB/s",
                                    "frac": nbytes / (bms * 1e-3) / 1e9 / hbm,
                                    "bytes_per_spot": 256 * 8 + 73,
                                    "traffic": _traffic_from_profile(BWD_PROFILE, BWD_SOURCE),
                                    "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"}}
    # the backward workload as configured: the gradient of (x0, y0, sigma, alpha, beta), no
    # upstream for the normalised chi^2, so the second pixel pass writes without reading
    bms2 = _timed(lambda: fitspots.backward(bb.images, bb.offsets, bb.dims, bb.model, fo, up[0],
                                            up[1], up[2], None, grad_images=gimg, stream=stream),
                  10, stream)
    nb2 = bb.n * (256 * 8 + 69)
    out_b["params_alpha_beta_only"] = {
        "what": "VJP of (x0, y0, sigma, alpha, beta) only (no chi^2 upstream)",
        "value": bb.n / (bms2 * 1e-3), "unit": "spots/s", "ms_per_step": bms2,
        "roofline": {"bound": "hbm", "achieved": nb2 / (bms2 * 1e-3) / 1e9, "peak": hbm,
                     "unit": "GB/s", "frac": nb2 / (bms2 * 1e-3) / 1e9 / hbm,
                     "bytes_per_spot": 256 * 8 + 69}}
    return {"backward": out_b}


def _extra_serving(args, dev) -> dict:
    import numpy as np
    import torch
    from paper_2106_02045_gb300 import serving, synth
    out = {}
    # serving: 2048x2048 uint16 frames at 2000 fps, 64 markers, 21x21 ROIs cut on device
    cs = synth.make_camera_stream(args.serving_ring, 64, 2048, 2048, device=dev)
    host = torch.empty(cs.frames.shape, dtype=torch.uint16, pin_memory=True)
    host.copy_(cs.frames)
    srv = serving.TrackingServer(2048, 2048, markers=64, sessions=1, device=dev)
    srv.set_markers(0, cs.start)
    warm = args.serving_warmup
    nfr = warm + args.serving_frames
    t0 = time.perf_counter()
    serving.run_stream(srv, 0, host, nfr, fps=2000.0)
    wall = time.perf_counter() - t0
    lat = np.array([srv.logs[0].latency[k] for k in range(warm, nfr) if k in srv.logs[0].latency])
    summ = serving.latency_summary(lat)
    truth = cs.truth.cpu().numpy()
    err = np.concatenate([np.hypot(*(srv.logs[0].results[k][:, :2] - truth[k % args.serving_ring]).T)
                          for k in range(warm, nfr) if k in srv.logs[0].results])
    out["serving"] = {"workload": "2048x2048 uint16 camera at 2000 fps, 64 fiducials, 21x21 ROIs "
                                  "cut on device, warm-started isotropic fits, drift 0.05 px/frame",
                      "p50_ms": summ["p50_ms"], "p99_ms": summ["p99_ms"], "max_ms": summ["max_ms"],
                      "frames": summ["frames"], "warmup_frames": warm, "dropped": srv.dropped,
                      "sustained_fps": nfr / wall, "tracking_error_px_median": float(np.median(err)),
                      "latency": "host arrival stamp -> results on host; one CUDA graph per frame"}
    return out


def _e2e(args, b, out, ws, stream, barrier, world, dev):
    """The metric through the public host-buffer call (fit_spots_uniform_host): pinned host
    images and start values in, host results out, copies overlapped with the fits chunk by
    chunk, all inside the timed region."""
    import numpy as np
    import torch
    from paper_2106_02045_gb300 import fitspots, synth
    h_img = torch.empty(b.images.shape, dtype=b.images.dtype, pin_memory=True)
    h_img.copy_(b.images)
    h_init = torch.empty(b.init.shape, dtype=b.init.dtype, pin_memory=True)
    h_init.copy_(b.init)
    h_out = fitspots.alloc_host_outputs(b.n)
    chunk = args.e2e_chunk
    dtype = fitspots.U16 if b.images.dtype == torch.uint16 else fitspots.F32
    d_ws = torch.empty(fitspots.host_workspace_bytes(min(chunk, b.n), W, H, dtype),
                       dtype=torch.uint8, device=dev)

    def e2e_step():
        fitspots.fit_uniform_host(h_img, W, H, synth.MODEL_ELLIPTIC, h_init, chunk=chunk,
                                  out=h_out, workspace=d_ws, device=dev, stream=stream)

    # one event before every call and one after the last: the mean over the steps is the
    # value, the per-call times show the spread (the host link of some boxes stalls for tens
    # of ms now and then, plain pinned copies included; see link_copy_ms)
    e2e_steps = max(5, args.steps)
    e2e_step()
    barrier()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(e2e_steps + 1)]
    evs[0].record(stream)
    for k in range(e2e_steps):
        e2e_step()
        evs[k + 1].record(stream)
    barrier()
    per_call = [evs[k].elapsed_time(evs[k + 1]) for k in range(e2e_steps)]
    e2e_ms = sum(per_call) / e2e_steps
    conv_e2e = int(np.isin(h_out["state"].numpy(), CONVERGED).sum())
    h2d = h_img.numel() * h_img.element_size() + h_init.numel() * h_init.element_size()
    d2h = sum(v.numel() * v.element_size() for v in h_out.values())
    ms_max, conv_sum = job_totals(e2e_ms, conv_e2e, world, dev)
    e2e_value = conv_sum / (ms_max * 1e-3)

    # the host link alone: one plain pinned host -> device copy of the same bytes, so that
    # the line shows whether the end-to-end number is bound by the link or by the fits
    d_img = torch.empty_like(b.images)
    copies = []
    with torch.cuda.stream(stream):
        d_img.copy_(h_img, non_blocking=True)
        for _ in range(e2e_steps):
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            d_img.copy_(h_img, non_blocking=True)
            c1.record(stream)
            copies.append((c0, c1))
    torch.cuda.synchronize(dev)
    copy_times = [c0.elapsed_time(c1) for c0, c1 in copies]
    copy_ms = statistics.median(copy_times)
    del d_img
    img_bytes = h_img.numel() * h_img.element_size()
    # the link split sits at the top level of the e2e object: the whole call's time, the
    # images' copy alone, and their ratio (near 1 = bound by the host link, not the fits)
    med = statistics.median(per_call)
    return {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "e2e_ms": e2e_ms, "e2e_median_ms": med, "e2e_max_ms": max(per_call),
            "steps": e2e_steps, "image_copy_ms": copy_ms, "image_copy_max_ms": max(copy_times),
            "link_h2d_gbs": img_bytes / (copy_ms * 1e-3) / 1e9,
            "frac_of_link": copy_ms / med, "chunk_spots": chunk,
            "call": "fit_spots_uniform_host (copies overlapped with fits; even and odd chunks "
                    "fitted on two streams)",
            "link_note": "image_copy_ms: median of as many pinned host-to-device copies of the "
                         "step's images alone, timed with CUDA events after the e2e steps; "
                         "frac_of_link = image_copy_ms / e2e_median_ms"}


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--cpu-sample", type=int, default=200_000)
    ap.add_argument("--ref-sample", type=int, default=100_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-chunk", type=int, default=E2E_CHUNK,
                    help="spots per chunk of the host-buffer call in the end-to-end leg")
    ap.add_argument("--no-extras", action="store_true", help="skip mixed/backward/serving")
    ap.add_argument("--extras",
                    default="mixed,backward,serving,start,table1,explicit,weighted,background,"
                            "paper_protocol",
                    help="comma-separated subset of mixed,backward,serving,start,table1,"
                         "explicit,weighted,background,paper_protocol")
    ap.add_argument("--mixed-spots", type=int, default=2_000_000)
    ap.add_argument("--serving-frames", type=int, default=20000)
    ap.add_argument("--serving-warmup", type=int, default=1000)
    ap.add_argument("--serving-ring", type=int, default=128)
    ap.add_argument("--spots", type=int, default=N_SPOTS, help="spots per GPU (profiling runs)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run(args)


if __name__ == "__main__":
    main()
