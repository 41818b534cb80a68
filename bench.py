#!/usr/bin/env python
"""Benchmark of the MGVI sampling hot path on the 2-D correlated field.

Workload (one step): 2-D 512x512 periodic correlated field with the
power-spectrum model, exponential response and Poisson counts (rate 10 exp(cf)),
FP32 vectors with FP64 CG reductions, a batch of B=32 MGVI sample systems
linearised at one expansion point: the MGVI right-hand side
b = xi' + J^T sqrt(w) eta, then 100 CG iterations of M_p = J^T N^-1 J + 1 on all
B systems.  Unit: metric-vector products/s (B * 100 per step).  Inputs are
larger than L2 (the CG working set is ~0.3 GB) and L2 is also flushed between
timed steps (outside the per-step CUDA events).

--impl reference times the FP64 CPU oracle (numpy) on a bounded sample of the
same workload.  Multi-GPU runs are independent replicas (the path has no
exchange step): every rank runs the same workload and value = all ranks'
products / the slowest rank's time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "metric-vector products/s & HBM roofline frac; serve p50/p99 vs plain at 1e-5 rel"
UNIT = "metric-vector products/s"
GRID = (512, 512)
BATCH = 32
CG_ITERS = 100
WORKLOAD = "cf2d_512x512_power_poisson_mgvi_cg100"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=BATCH)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--no-metric-grids", action="store_true",
                    help="skip the metric-product roofline leg on 2-D 1024^2 and 3-D 256^3")
    ap.add_argument("--metric-batch", type=int, default=8)
    ap.add_argument("--icr-batch", type=int, default=32)
    ap.add_argument("--cg3d-maxiter", type=int, default=2000,
                    help="iteration cap of the 3-D masked batched CG solve in the metric leg")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests of the serving stream (0: skip the serving leg)")
    ap.add_argument("--serve-budget-gb", type=float, default=2.0,
                    help="HBM budget of the second FP32 server run (0: skip it)")
    ap.add_argument("--serve-budget-requests", type=int, default=500,
                    help="requests of the stream's start that the budgeted run serves")
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-sustained-requests", type=int, default=300,
                    help="requests of the slower stream served by the FP32 server alone (0: skip)")
    ap.add_argument("--serve-sustained-rate", type=float, default=10.0)
    ap.add_argument("--serve-plain-cap-s", type=float, default=90.0,
                    help="stop the sequential FP64 arm after this many seconds")
    ap.add_argument("--serve-timeout-s", type=float, default=900.0,
                    help="limit of the serving leg's child process")
    ap.add_argument("--serve-only", action="store_true", help="run only the serving leg")
    ap.add_argument("--icr-only", action="store_true", help="run only the ICR leg")
    ap.add_argument("--next-only", action="store_true", help="run only the KL / geoVI / 3-D ICR leg")
    ap.add_argument("--no-next-rows", action="store_true", help="skip the KL / geoVI / 3-D ICR leg")
    ap.add_argument("--icr3-only", action="store_true", help="run only the 3-D ICR part of that leg")
    return ap.parse_args()


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum, ncu,
# one capture, caches flushed before each launch) of the kernels that can be
# the dominant one, keyed by (kernel tag, batch), averaged over the launch
# variants the tag covers, with the digest of the sources that define those
# kernels at capture time (kernel_src_digest); an entry whose digest differs
# from the current sources is stale and reported as null.
# row_sweep_f32_2d at batch 32: the traced (unsplit) launches take the whole
# batch; the capture ran the half-batch launches of the split product (16
# samples): 18.18 MB (prologue sweep) and 34.84 MB (epilogue sweep) read,
# 0.01 MB written, scaled by two (traffic grows with the samples; the shared
# bin and expansion-point tables, 1.5 MB, are then counted twice) and
# averaged over the two variants (profiles/traffic_f32_2d_512x512_b32.md).
DRAM_TRAFFIC = {("row_sweep_f32_2d", 32): (53.02e6, "ncu dram__bytes_read.sum + dram__bytes_write.sum, "
                                                    "half-batch launches x 2, mean of the two row sweeps",
                                           "7a55a704d9d23b42")}

# The sources that define the row sweeps' device code (the digest of
# DRAM_TRAFFIC), the bulk-copy helpers of their row staging included; the C
# header does not enter it.
SWEEP_SOURCES = ["common.cuh", "cf_internal.cuh", "fft.cuh", "regfft.cuh", "tma.cuh", "sweeps_reg.cuh",
                 "sweeps_launch.cuh", "sweeps_inst.cu"]


def kernel_src_digest(files=SWEEP_SOURCES):
    """sha256 (first 16 hex digits) of the given library sources."""
    import hashlib
    d = os.path.join(ROOT, "paper_2402_16683_gb300", "csrc")
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read())
    return h.hexdigest()[:16]


def config(batch):
    return {"workload": WORKLOAD, "grid": list(GRID), "batch": batch, "cg_iters": CG_ITERS,
            "amplitude": "power-spectrum model, 256 log-|k| bins", "likelihood": "poisson, rate 10 exp(cf)",
            "l2": "inputs larger than L2 (CG working set ~0.3 GB) and L2 flushed between timed steps"}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ----------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------- oracle leg
def oracle_setup():
    from oracle import amplitude as oamp
    from oracle.cf import CFModel
    from oracle.likelihood import poisson_weight
    pr = oamp.AmpPrior(**synth.AMP_PRIOR)
    om = CFModel(GRID, tuple(1.0 / s for s in GRID), prior=pr)
    xi_p = synth.normal(synth.SEED_POS, om.latent_size)
    w = poisson_weight(om.forward(xi_p), 10.0)
    return om, xi_p, w


def oracle_step(om, xi_p, w, seed, iters):
    """One bounded sample of the workload on the CPU: one system's MGVI
    right-hand side and `iters` CG iterations (one metric product each)."""
    from oracle.cg import cg
    from oracle.metric import metric_apply, mgvi_rhs
    g = np.random.default_rng(seed)
    b = mgvi_rhs(om, xi_p, w, g.standard_normal(om.latent_size), g.standard_normal(om.n_field))
    cg(lambda p: metric_apply(om, xi_p, w, p), b, rtol=0.0, maxiter=iters)
    return iters


def _oracle_worker(args):
    """One host process of the CPU baseline: systems seed0, seed0 + stride, ...
    until `seconds` have passed; returns (products, seconds)."""
    seed0, stride, seconds, iters = args
    om, xi_p, w = oracle_setup()
    t0 = time.perf_counter()
    n, k = 0, 0
    while time.perf_counter() - t0 < seconds:
        n += oracle_step(om, xi_p, w, seed0 + stride * k, iters)
        k += 1
    return n, time.perf_counter() - t0, k


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                low = line.lower()
                if low.startswith("model name") or low.startswith("cpu part") or low.startswith("hardware"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_on_cores(ncores, seconds, iters=20, seed0=1000):
    """The oracle on `ncores` host processes (one thread each, started with
    spawn), each solving its own systems for `seconds`: products/s of all."""
    if ncores <= 1:
        n, dt, k = _oracle_worker((seed0, 1, seconds, iters))
        return n / dt, k
    import multiprocessing as mp
    env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(ncores) as pool:
            res = pool.map(_oracle_worker, [(seed0 + c, ncores, seconds, iters) for c in range(ncores)])
    finally:
        for k, v in env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return sum(r[0] for r in res) / max(r[1] for r in res), sum(r[2] for r in res)


def cpu_baseline(target_s=12.0):
    """The FP64 oracle on every host core (one process per core), and on one."""
    nc = cpu_cores()
    v_all, k_all = oracle_on_cores(nc, target_s)
    v_one, k_one = oracle_on_cores(1, target_s)
    return {"value": v_all, "unit": UNIT, "cores": nc, "kind": "oracle",
            "sample": f"{k_all} systems x (MGVI rhs + 20 CG iterations) of the 512x512 Poisson metric, "
                      f"FP64 numpy oracle, one process per core on {nc} cores ({cpu_model()}), "
                      f"{target_s:.0f} s",
            "single_core": {"value": v_one, "cores": 1,
                            "sample": f"{k_one} systems, one process, {target_s:.0f} s"}}


def _oracle_systems(args):
    """`count` systems of the reference arm from seed0 (one host process)."""
    seed0, count, iters = args
    om, xi_p, w = oracle_setup()
    for k in range(count):
        oracle_step(om, xi_p, w, seed0 + k, iters)
    return count * iters


def run_reference(args, rank, world):
    """The oracle as it stands on the host cores: each step solves one system
    per core (MGVI rhs + 20 CG iterations), one process per core."""
    if rank != 0:
        return
    import multiprocessing as mp
    iters = 20
    nc = cpu_cores()
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    with mp.get_context("spawn").Pool(nc) as pool:
        pool.map(_oracle_systems, [(2000 + c, 1, iters) for c in range(nc)] * max(1, args.warmup))
        times = []
        for i in range(args.steps):
            t0 = time.perf_counter()
            pool.map(_oracle_systems, [(3000 + 100 * i + c, 1, iters) for c in range(nc)])
            times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = args.steps * nc * iters / tot
    cb = {"value": value, "unit": UNIT, "cores": nc, "kind": "oracle",
          "sample": f"each step: {nc} systems (one per core, {cpu_model()}), each the MGVI rhs + {iters} "
                    f"CG iterations of the 512x512 Poisson metric, FP64 numpy oracle"}
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
                      "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
                      "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config(1),
                      "cpu_baseline": cb,
                      "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
          flush=True)


# ----------------------------------------------------------------- GPU leg
def max_over_ranks(t, world, device):
    """The slowest rank's time (replicas run the same work): all-reduce MAX over
    the process group when world > 1."""
    if world <= 1:
        return t
    import torch
    v = torch.tensor([t], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(v, op=torch.distributed.ReduceOp.MAX)
    return float(v.item())


def replica_throughput(units_per_rank, world, t_max):
    """Whole-job throughput of `world` replicas: all ranks' units over the
    slowest rank's time."""
    return world * units_per_rank / t_max


def run_ours(args, rank, world):
    import ctypes as C

    import torch

    import paper_2402_16683_gb300 as nre
    from paper_2402_16683_gb300 import _lib

    if args.serve_only:
        if rank == 0:
            try:
                serve = run_serve(args)
            except Exception as e:
                serve = {"error": f"{type(e).__name__}: {e}"[:500]}
            print(json.dumps({"serve": serve}), flush=True)
        return
    if args.icr_only:
        lib0 = _lib.load()
        dev0 = torch.device("cuda", torch.cuda.current_device())
        fl = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev0)
        if rank == 0:
            print(json.dumps({"icr": run_icr(args, lib0, fl, torch.cuda.current_stream(), peaks()[0])}), flush=True)
        return
    if args.next_only or args.icr3_only:
        lib0 = _lib.load()
        dev0 = torch.device("cuda", torch.cuda.current_device())
        fl = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev0)
        if rank == 0:
            print(json.dumps({"next_rows": run_next_rows(args, lib0, fl, torch.cuda.current_stream(), peaks()[0],
                                                          icr3_only=args.icr3_only)}), flush=True)
        return
    lib = _lib.load()
    lib.nre_launch_count.restype = C.c_ulonglong
    lib.nre_launch_count.argtypes = []
    lib.nre_prof_enable.argtypes = [C.c_int]
    lib.nre_prof_report.argtypes = [C.c_char_p, C.c_size_t]

    dev = torch.device("cuda", torch.cuda.current_device())
    B = args.batch
    plan = nre.CorrelatedField(GRID, tuple(1.0 / s for s in GRID), amplitude="power",
                               prior=dict(synth.AMP_PRIOR), dtype=torch.float32)
    lik = nre.Likelihood("poisson", scale=10.0)
    xi_p = torch.tensor(synth.normal(synth.SEED_POS, plan.latent_size), dtype=torch.float32, device=dev)
    M = nre.Metric(plan, lik, plan.pad(xi_p[None])[0], max_batch=B)
    g = np.random.default_rng(synth.SEED_RHS + 100 * rank)
    xi_prime = plan.pad(torch.tensor(g.standard_normal((B, plan.latent_size)), dtype=torch.float32, device=dev))
    eta = torch.tensor(g.standard_normal((B, plan.n_field)), dtype=torch.float32, device=dev)
    b = torch.zeros_like(xi_prime)
    x = torch.zeros_like(xi_prime)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        M.mgvi_rhs(xi_prime, eta, out=b)
        _, its, rel, st = M.cg(b, rtol=0.0, maxiter=CG_ITERS, x=x)
        return its

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def timed(n):
        ev = []
        for _ in range(n):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            its = step()
            e1.record(stream)
            ev.append((e0, e1))
        barrier()
        return sum(a.elapsed_time(b_) for a, b_ in ev), its

    clocks = Clocks(torch.cuda.current_device())
    barrier()
    clocks.start()
    n0 = lib.nre_launch_count()
    ms, its = timed(args.steps)
    launches = lib.nre_launch_count() - n0
    clk = clocks.stop()
    # per-kernel device times from a separate traced pass (the events that
    # bracket every launch are kept out of the timed steps above)
    lib.nre_prof_enable(1)
    timed(max(1, min(args.steps, 5)))
    lib.nre_prof_enable(0)
    buf = C.create_string_buffer(1 << 16)
    _lib.check(lib.nre_prof_report(buf, len(buf)))
    kern = json.loads(buf.value.decode())
    t_max = max_over_ranks(ms / 1e3, world, dev)
    value = replica_throughput(args.steps * B * CG_ITERS, world, t_max)

    # dominant kernel: largest total device time in the timed region
    name, (cnt, kms, kbytes) = max(kern.items(), key=lambda kv: kv[1][1])
    peak, peak_kind = peaks()
    achieved = kbytes / (kms / 1e3) / 1e9
    traffic = DRAM_TRAFFIC.get((name, B))
    if traffic and traffic[2] != kernel_src_digest():
        traffic = None  # captured from other kernel sources: stale
    roofline = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind,
                "traffic": traffic[0] if traffic else None,
                "traffic_source": traffic[1] if traffic else None,
                "launches": int(cnt), "avg_launch_us": 1e3 * kms / cnt,
                "algorithmic_bytes_per_launch": kbytes / cnt}
    kernels = {k: {"launches": int(v[0]), "ms": v[1], "share": v[1] / sum(u[1] for u in kern.values()),
                   "GBps": (v[2] / (v[1] / 1e3) / 1e9) if v[1] > 0 else None} for k, v in kern.items()}

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, M, plan, xi_prime, eta, b, x, flush, stream, world, barrier)
    grids = None
    if not args.no_metric_grids:
        grids = run_metric_grids(args, lib)
    nxt = None
    if not args.no_next_rows and rank == 0:
        try:
            nxt = run_next_rows(args, lib, flush, stream, peaks()[0])
        except Exception as e:  # keep the line: the leg's failure is part of the result
            nxt = {"error": f"{type(e).__name__}: {e}"[:500]}
    serve = None
    if args.serve_requests > 0 and world == 1:
        serve = run_serve_child(args)
    if rank != 0:
        return
    cb = None
    if world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline()
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": config(B), "roofline": roofline, "cpu_baseline": cb, "e2e": e2e,
           "gpu_launches": int(launches), "clocks": clk, "kernels": kernels,
           "cg_iterations": its[:1]}
    if grids is not None:
        out["metric_grids"] = grids
    if nxt is not None:
        out["next_rows"] = nxt
    if serve is not None:
        out["serve"] = serve
    print(json.dumps(out), flush=True)


def run_e2e(args, M, plan, xi_prime, eta, b, x, flush, stream, world, barrier):
    """The same step through the public API with pinned host buffers: every
    step's excitations are copied in and its samples copied out inside the
    timed region.  The copies run on a copy stream, pipelined with the compute
    (the next step's inputs go in while this step solves, this step's samples
    come out while the next one solves; device buffers alternate between two
    steps), the way a caller streams batches through the API."""
    import torch
    B = xi_prime.shape[0]
    dev = xi_prime.device
    h_xi = torch.empty_like(xi_prime, device="cpu").pin_memory()
    h_eta = torch.empty_like(eta, device="cpu").pin_memory()
    h_x = [torch.empty_like(x, device="cpu").pin_memory() for _ in range(2)]
    h_xi.copy_(xi_prime)
    h_eta.copy_(eta)
    d_xi = [torch.empty_like(xi_prime) for _ in range(2)]
    d_eta = [torch.empty_like(eta) for _ in range(2)]
    d_x = [x, torch.empty_like(x)]
    cs = torch.cuda.Stream(device=dev)

    def run(n, e0=None):
        """n pipelined steps on `stream` (compute) and `cs` (copies)."""
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_done = [torch.cuda.Event() for _ in range(2)]
        ev_out = torch.cuda.Event()

        def put(k):  # inputs of step k into buffer k % 2 (after step k - 2 used it)
            j = k % 2
            with torch.cuda.stream(cs):
                if k >= 2:
                    cs.wait_event(ev_done[j])
                d_xi[j].copy_(h_xi, non_blocking=True)
                d_eta[j].copy_(h_eta, non_blocking=True)
                ev_in[j].record(cs)

        if e0 is not None:
            cs.wait_event(e0)
        put(0)
        for k in range(n):
            j = k % 2
            if k + 1 < n:
                put(k + 1)
            stream.wait_event(ev_in[j])
            M.mgvi_rhs(d_xi[j], d_eta[j], out=b)
            M.cg(b, rtol=0.0, maxiter=CG_ITERS, x=d_x[j])
            ev_done[j].record(stream)
            with torch.cuda.stream(cs):
                cs.wait_event(ev_done[j])
                h_x[j].copy_(d_x[j], non_blocking=True)
        ev_out.record(cs)
        stream.wait_event(ev_out)

    run(2)
    barrier()
    e_steps = max(2, min(args.steps, 5))
    flush.zero_()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    run(e_steps, e0)
    e1.record(stream)
    barrier()
    e_ms = e0.elapsed_time(e1)
    e_t = max_over_ranks(e_ms / 1e3, world, dev)
    return {"value": replica_throughput(e_steps * B * CG_ITERS, world, e_t), "unit": UNIT,
            "h2d_bytes_per_step": int(h_xi.numel() * 4 + h_eta.numel() * 4),
            "d2h_bytes_per_step": int(h_x[0].numel() * 4),
            "pipelined": "copies on a second stream, overlapped with the neighbouring steps' solves"}


# ----------------------------------------------------------------- metric roofline leg
METRIC_GRIDS = [((1024, 1024), "poisson"), ((256, 256, 256), "gauss_mask10")]


def run_metric_grids(args, lib):
    """Metric-vector products alone (no CG) at B=8 on the 2-D 1024^2 Poisson
    and the 3-D 256^3 Gaussian (sigma 0.05, 10% mask) fields: products/s and
    the HBM roofline of the whole product (algorithmic bytes of all its
    kernels over the untraced time of a product) and of each kernel (over its
    own device time in a traced pass)."""
    import ctypes as C

    import torch

    import paper_2402_16683_gb300 as nre
    from paper_2402_16683_gb300 import _lib

    peak, _ = peaks()
    dev = torch.device("cuda", torch.cuda.current_device())
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    B = args.metric_batch
    out = {}
    for shape, kind in METRIC_GRIDS:
        plan = nre.CorrelatedField(shape, amplitude="power", prior=dict(synth.AMP_PRIOR), dtype=torch.float32)
        if kind == "poisson":
            lik = nre.Likelihood("poisson", scale=10.0)
        else:
            # the Gaussian likelihood observes the field itself (identity response)
            lik = nre.Likelihood("gauss", sigma=0.05, mask=synth.mask_fraction(synth.SEED_MASK, plan.n_field),
                                 n_data=plan.n_field, response="identity")
        xi_p = torch.tensor(synth.normal(synth.SEED_POS, plan.latent_size), dtype=torch.float32, device=dev)
        M = nre.Metric(plan, lik, plan.pad(xi_p[None])[0], max_batch=B)
        g = np.random.default_rng(synth.SEED_TANGENT)
        v = plan.pad(torch.tensor(g.standard_normal((B, plan.latent_size)), dtype=torch.float32, device=dev))
        o = torch.empty_like(v)
        for _ in range(3):
            M.apply(v, out=o)
        torch.cuda.synchronize()

        def timed(n):
            ev = []
            for _ in range(n):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                M.apply(v, out=o)
                e1.record(stream)
                ev.append((e0, e1))
            torch.cuda.synchronize()
            return sum(a.elapsed_time(b_) for a, b_ in ev) / n

        n = max(5, args.steps)
        ms = timed(n)
        lib.nre_prof_enable(1)
        timed(n)
        lib.nre_prof_enable(0)
        buf = C.create_string_buffer(1 << 16)
        _lib.check(lib.nre_prof_report(buf, len(buf)))
        kern = json.loads(buf.value.decode())
        kms = sum(x[1] for x in kern.values())
        kbytes = sum(x[2] for x in kern.values())
        name = "x".join(str(d) for d in shape)
        out[f"{len(shape)}d_{name}"] = {
            "likelihood": kind, "batch": B, "products_per_s": B / (ms / 1e3), "ms_per_apply": ms,
            "bytes_per_apply": kbytes / n,
            # whole product: its algorithmic bytes over the untraced time of a product
            "achieved_GBps": kbytes / n / (ms / 1e3) / 1e9, "frac": kbytes / n / (ms / 1e3) / 1e9 / peak,
            # the same over the summed device times of its kernels, traced one by one
            # (launches serialised: the split product's two streams run one after the other)
            "frac_traced_kernels": kbytes / (kms / 1e3) / 1e9 / peak,
            "kernels": {k: {"us_per_launch": 1e3 * x[1] / x[0], "GBps": x[2] / (x[1] / 1e3) / 1e9 if x[1] else None,
                            "frac": (x[2] / (x[1] / 1e3) / 1e9 / peak) if x[1] else None}
                        for k, x in kern.items()}}
        if len(shape) == 3:
            # the 3-D masked workload's batched sample solve: FP32 CG with the
            # harmonic preconditioner on the MGVI right-hand sides to a
            # recursive 1e-5 (timed), the FP64 true residual ||b - M x|| / ||b||
            # of each solution from an FP64 metric at the same expansion point,
            # then the same systems with FP64 residual correction around the
            # FP32 PCG to a true 1e-5
            eta = torch.tensor(np.random.default_rng(synth.SEED_RHS).standard_normal((B, plan.n_field)),
                               dtype=torch.float32, device=dev)
            M.mgvi_rhs(v, eta, out=o)
            M.set_precond("harmonic")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            x3, its, rel, st_ = M.cg(o, rtol=1e-5, maxiter=args.cg3d_maxiter)
            torch.cuda.synchronize()
            secs = time.perf_counter() - t0
            p64 = nre.CorrelatedField(shape, amplitude="power", prior=dict(synth.AMP_PRIOR), dtype=torch.float64)
            M64 = nre.Metric(p64, lik, p64.pad(xi_p.double()[None])[0], max_batch=B)
            o64 = o.double()
            r64 = o64 - M64.apply(x3.double())
            true = [float(p64.unpad(r64)[i].norm() / p64.unpad(o64)[i].norm()) for i in range(B)]
            del r64
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, its_r, true_r, passes, st_r = M.cg_refined(M64, o64, rtol=1e-5, max_outer=8, inner_rtol=1e-3,
                                                          inner_maxiter=args.cg3d_maxiter)
            torch.cuda.synchronize()
            secs_r = time.perf_counter() - t0
            del M64, p64, o64
            out[f"{len(shape)}d_{name}"]["cg_to_1e-5"] = {
                "maxiter": args.cg3d_maxiter, "precond": "harmonic",
                "likelihood": "gauss sigma 0.05 on the field (identity response), 10 % mask",
                "fp32_pcg": {"iterations": [int(i) for i in its], "relres": [float(r) for r in rel],
                             "true_relres_fp64": true, "converged_recursive": st_ == 0, "seconds": secs},
                "refined": {"passes": passes, "inner_iterations": [int(i) for i in its_r],
                            "true_relres_fp64": [float(r) for r in true_r], "converged": st_r == 0,
                            "seconds": secs_r}}
        del M, v, o
        torch.cuda.empty_cache()
    out["icr_8_to_1024"] = run_icr(args, lib, flush, stream, peak)
    return out


def run_icr(args, lib, flush, stream, peak):
    """ICR on the log-radial chart refined 8^2 -> 1024^2 (7 levels), Matern-3/2
    (length scale 0.1, unit variance), FP32, batch 32: forward (= JVP, the
    model is linear in xi) and the hand-written VJP; fields/s and the HBM
    fraction of a whole call (its kernels' algorithmic bytes over its untraced
    time) and of its kernels traced one by one."""
    import ctypes as C

    import torch

    import paper_2402_16683_gb300 as nre
    from paper_2402_16683_gb300 import _lib

    dev = torch.device("cuda", torch.cuda.current_device())
    B = args.icr_batch
    icr = nre.ICR(n0=8, n_levels=7, rho=0.1, var=1.0, dtype=torch.float32)
    g = np.random.default_rng(synth.SEED_POS)
    xi = icr.pad(torch.tensor(g.standard_normal((B, icr.latent_size)), dtype=torch.float32, device=dev))
    ct = torch.tensor(g.standard_normal((B, icr.n_out)), dtype=torch.float32, device=dev)
    res = {"batch": B, "levels": 7, "grid": [1024, 1024]}
    for name, fn in (("forward", lambda: icr.forward(xi)), ("vjp", lambda: icr.vjp(xi, ct))):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()

        def timed(n):
            ev = []
            for _ in range(n):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                ev.append((e0, e1))
            torch.cuda.synchronize()
            return sum(a.elapsed_time(b_) for a, b_ in ev) / n

        n = max(5, args.steps)
        ms = timed(n)
        lib.nre_prof_enable(1)
        timed(n)
        lib.nre_prof_enable(0)
        buf = C.create_string_buffer(1 << 16)
        _lib.check(lib.nre_prof_report(buf, len(buf)))
        kern = json.loads(buf.value.decode())
        kms = sum(x[1] for x in kern.values())
        kbytes = sum(x[2] for x in kern.values())
        res[name] = {"fields_per_s": B / (ms / 1e3), "ms": ms, "bytes": kbytes / n,
                     # all bytes of a call over its untraced time; and over the summed
                     # device times of its kernels traced one by one
                     "achieved_GBps": kbytes / n / (ms / 1e3) / 1e9, "frac": kbytes / n / (ms / 1e3) / 1e9 / peak,
                     "frac_traced_kernels": kbytes / (kms / 1e3) / 1e9 / peak,
                     "kernels": {k: {"launches_per_call": x[0] / n, "us_per_call": 1e3 * x[1] / n,
                                     "GBps": x[2] / (x[1] / 1e3) / 1e9 if x[1] else None}
                                 for k, x in kern.items()}}
    return res


# ----------------------------------------------------------------- KL / geoVI / 3-D ICR leg
def _timed_traced(lib, fn, n, flush, stream):
    """Mean untraced time (ms) of fn over n calls, L2 flushed before each, and
    the per-kernel (launches, ms, algorithmic bytes) of n traced calls."""
    import ctypes as C

    import torch

    from paper_2402_16683_gb300 import _lib

    def timed():
        ev = []
        for _ in range(n):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            ev.append((e0, e1))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b_) for a, b_ in ev) / n

    ms = timed()
    lib.nre_prof_enable(1)
    timed()
    lib.nre_prof_enable(0)
    buf = C.create_string_buffer(1 << 16)
    _lib.check(lib.nre_prof_report(buf, len(buf)))
    return ms, json.loads(buf.value.decode())


def _leg_stats(ms, kern, n, peak, units, unit_name):
    """units per second, and the HBM fraction of the whole call (its kernels'
    algorithmic bytes over its untraced time) and of its kernels traced one by
    one (over their summed device time)."""
    kms = sum(x[1] for x in kern.values())
    kbytes = sum(x[2] for x in kern.values())
    top = max(kern.items(), key=lambda kv: kv[1][1])[0] if kern else None
    return {unit_name: units / (ms / 1e3), "ms": ms, "bytes": kbytes / n,
            "achieved_GBps": kbytes / n / (ms / 1e3) / 1e9, "frac": kbytes / n / (ms / 1e3) / 1e9 / peak,
            "frac_traced_kernels": (kbytes / (kms / 1e3) / 1e9 / peak) if kms else None,
            "kernel_launches_per_call": sum(x[0] for x in kern.values()) / n, "top_kernel": top,
            "kernels": {k: {"us_per_call": 1e3 * x[1] / n, "share": x[1] / kms if kms else None,
                            "GBps": x[2] / (x[1] / 1e3) / 1e9 if x[1] else None} for k, x in kern.items()}}


def run_next_rows(args, lib, flush, stream, peak, icr3_only=False):
    """The rows after sampling, FP32 on the 2-D 512^2 Poisson workload (rate
    10 exp(cf), power-spectrum model) and the 3-D chart:

    * KL (MGVI): four residual samples (two antithetic pairs of linear draws,
      CG to 1e-3 on the MGVI right-hand sides at xi_bar); energy and gradient,
      the sample-averaged metric product, one Newton-CG step (CG to 1e-3);
    * geoVI: the nonlinear update of 8 linear draws (5 Newton iterations at
      most, inner CG to 1e-3);
    * ICR on the spherical log-radial chart refined 4^3 -> 256^3 (6 levels),
      Matern-3/2 (length scale 0.1), batch 4: forward and VJP.
    Counts drawn from the model at a N(0, 1) truth (seed SEED_TRUTH)."""
    import torch

    import paper_2402_16683_gb300 as nre

    dev = torch.device("cuda", torch.cuda.current_device())
    n = max(5, args.steps)
    out = {}
    if icr3_only:
        out["icr3_4_to_256"] = run_icr3(args, lib, flush, stream, peak, n, dev)
        return out
    shape = (512, 512)
    plan = nre.CorrelatedField(shape, amplitude="power", prior=dict(synth.AMP_PRIOR), dtype=torch.float32)
    lik = nre.Likelihood("poisson", scale=10.0)
    truth = torch.tensor(synth.normal(synth.SEED_TRUTH, plan.latent_size), dtype=torch.float32, device=dev)
    cf = plan.forward(plan.pad(truth[None]))[0].double().cpu().numpy()
    data = synth.rng(synth.SEED_TRUTH + 100).poisson(10.0 * np.exp(cf)).astype(np.float64)
    xbar = plan.pad(torch.tensor(0.1 * synth.normal(synth.SEED_POS, plan.latent_size), dtype=torch.float32,
                                 device=dev)[None])[0]

    # ---- MGVI: linear draws at xi_bar, the KL of their antithetic samples
    M = nre.Metric(plan, lik, xbar, max_batch=8)
    g = np.random.default_rng(synth.SEED_RHS)
    xi_prime = plan.pad(torch.tensor(g.standard_normal((8, plan.latent_size)), dtype=torch.float32, device=dev))
    eta = torch.tensor(g.standard_normal((8, plan.n_field)), dtype=torch.float32, device=dev)
    rhs = M.mgvi_rhs(xi_prime, eta)
    draws, _, _, _ = M.cg(rhs, rtol=1e-3, maxiter=500)
    deltas = torch.cat([draws[:2], -draws[:2]])
    kl = nre.KL(plan, lik, data, deltas.contiguous())
    kl.set_position(xbar)
    res = {"samples": 4, "grid": list(shape)}
    # energy and gradient at a position: S forward models, the likelihood
    # terms and S adjoints (set_position evaluates both; energy_gradient
    # returns them)
    ms, kern = _timed_traced(lib, lambda: kl.set_position(xbar), n, flush, stream)
    res["energy_and_gradient"] = _leg_stats(ms, kern, n, peak, 1, "per_s")
    KM = kl.metric()
    v = plan.pad(torch.tensor(g.standard_normal((1, plan.latent_size)), dtype=torch.float32, device=dev))
    o = torch.empty_like(v)
    ms, kern = _timed_traced(lib, lambda: KM.apply(v, out=o), n, flush, stream)
    res["metric_product"] = _leg_stats(ms, kern, n, peak, 1, "products_per_s")
    e0 = kl.energy_gradient()[0]
    steps = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, e, its = kl.newton_step(cg_rtol=1e-3, cg_maxiter=200)
        torch.cuda.synchronize()
        steps.append({"ms": 1e3 * (time.perf_counter() - t0), "cg_iterations": its, "mean_abs_step": st,
                      "energy": e})
    res["newton_steps"] = steps
    res["energy_start"] = e0
    out["kl_2d_512x512_poisson_S4"] = res
    del KM, kl

    # ---- geoVI: nonlinear update of the 8 linear draws at xi_bar
    d0 = draws.clone()
    d = torch.empty_like(d0)
    info = {}

    def gv():
        d.copy_(d0)
        its, stp = M.geovi_update(rhs, d, xtol=0.0, maxiter=5, cg_rtol=1e-3, cg_maxiter=500)
        info["its"], info["steps"] = its, stp

    gv()
    ms, kern = _timed_traced(lib, gv, max(3, n // 2), flush, stream)
    r = _leg_stats(ms, kern, max(3, n // 2), peak, 8, "samples_per_s")
    r.update({"samples": 8, "newton_iterations": [int(i) for i in info["its"]],
              "last_mean_abs_step": [float(s) for s in info["steps"]]})
    out["geovi_2d_512x512_poisson_B8"] = r
    del M, draws, d0, d, rhs
    torch.cuda.empty_cache()

    out["icr3_4_to_256"] = run_icr3(args, lib, flush, stream, peak, n, dev)
    return out


def run_icr3(args, lib, flush, stream, peak, n, dev):
    """ICR on the spherical log-radial chart refined 4^3 -> 256^3 (6 levels),
    Matern-3/2 (length scale 0.1), FP32, batch 4: forward and VJP."""
    import torch

    import paper_2402_16683_gb300 as nre

    B = 4
    icr = nre.ICR(n0=4, n_levels=6, rho=0.1, var=1.0, dtype=torch.float32, ndim=3)
    xi = icr.pad(torch.tensor(synth.rng(synth.SEED_POS).standard_normal((B, icr.latent_size)), dtype=torch.float32,
                              device=dev))
    ct = torch.tensor(synth.rng(synth.SEED_TANGENT).standard_normal((B, icr.n_out)), dtype=torch.float32, device=dev)
    res = {"batch": B, "levels": 6, "grid": [256, 256, 256]}
    for name, fn in (("forward", lambda: icr.forward(xi)), ("vjp", lambda: icr.vjp(xi, ct))):
        fn()
        ms, kern = _timed_traced(lib, fn, n, flush, stream)
        res[name] = _leg_stats(ms, kern, n, peak, B, "fields_per_s")
    del icr, xi, ct
    torch.cuda.empty_cache()
    return res


# ----------------------------------------------------------------- serving leg
def run_serve_child(args):
    """The serving leg in a child process (this script with --serve-only), so
    that its failure, whatever it is, leaves the rest of the line intact."""
    cmd = [sys.executable, os.path.abspath(__file__), "--serve-only",
           "--serve-requests", str(args.serve_requests), "--serve-budget-gb", str(args.serve_budget_gb),
           "--serve-budget-requests", str(args.serve_budget_requests), "--serve-slots", str(args.serve_slots),
           "--serve-plain-cap-s", str(args.serve_plain_cap_s),
           "--serve-sustained-requests", str(args.serve_sustained_requests),
           "--serve-sustained-rate", str(args.serve_sustained_rate)]
    try:
        p = subprocess.run(cmd, capture_output=True, text=True, timeout=args.serve_timeout_s)
    except subprocess.TimeoutExpired:
        return {"error": f"serving leg exceeded {args.serve_timeout_s:.0f} s"}
    for line in reversed(p.stdout.splitlines()):
        if line.startswith('{"serve"'):
            return json.loads(line)["serve"]
    return {"error": f"serving leg exited with {p.returncode}: {p.stderr[-400:]}"}


SERVE_SAMPLES = 8
SERVE_RTOL = 1e-5
SERVE_MAXITER = 2000
# residual-correction passes of the FP32 server's requests: its solutions are
# FP64 and meet SERVE_RTOL on the true residual
SERVE_REFINE = 4
# Gaussian requests observe the field itself (sigma 0.1, every pixel); Poisson
# requests count at rate 10 exp(cf)
SERVE_RESPONSE = {"gauss": "identity", "poisson": "exp"}


def _pctl(v, q):
    return float(np.percentile(np.asarray(v), q)) if v else None


def run_serve(args):
    """The request stream (Poisson arrivals at 50/s, grids drawn uniformly from
    1-D 4096, 2-D 256^2, 2-D 1024^2, 3-D 128^3, Gaussian (sigma 0.1 on cf,
    every pixel) / Poisson (rate 10 exp(cf)) 50/50, 8 sample systems per
    request to 1e-5 relative residual) through

    * the FP32 server: continuous batching, one stream per admitted request,
      CG chunks replayed as CUDA graphs, admission by HBM footprint, FP32
      solves with FP64 residual correction to the true 1e-5 (FP64 solutions);
      run once with the whole device and once under an HBM budget;
    * the plain sequential FP64 path: requests first in first out, one
      system at a time (batch 1), through Metric / cg, nothing overlapped.

    Both use the harmonic preconditioner and the same inputs (a pool of two
    input sets per grid, reused round-robin; expansion points with N(0, 1)
    field and offset excitations and the power-spectrum excitations at the
    prior median).  Latency = result in host memory
    minus arrival.  One request per grid is served first, untimed, so that plans
    (and the server's slot objects) exist before the stream starts."""
    import torch

    import paper_2402_16683_gb300 as nre

    reqs = synth.request_stream(synth.SEED_STREAM, n=args.serve_requests, rate=50.0)
    pool = 2
    inputs = {}
    for si, shape in enumerate(synth.SERVE_SHAPES):
        N = int(np.prod(shape))
        lat = N + 4 + 2 * 255
        sets = []
        for k in range(pool):
            g = np.random.default_rng(9000 + 10 * si + k)
            xv = g.standard_normal(lat)
            xv[N:] = 0.0  # power-spectrum excitations at the prior median
            xi = torch.tensor(xv, dtype=torch.float32).pin_memory()
            b = torch.tensor(g.standard_normal((SERVE_SAMPLES, lat)), dtype=torch.float32).pin_memory()
            sets.append((xi, b))
        inputs[shape] = sets
    free = {shape: [] for shape in synth.SERVE_SHAPES}
    lock = threading.Lock()

    def take_out(shape):
        with lock:
            if free[shape]:
                return free[shape].pop()
        return torch.empty(inputs[shape][0][1].shape, dtype=torch.float64).pin_memory()

    def serve_fp32(budget_bytes, reqs):
        """The stream through one FP32 server; returns its statistics and one
        solution per (grid, likelihood) class for the true-residual check."""
        srv = nre.Server(hbm_budget_bytes=budget_bytes, max_slots=args.serve_slots, dtype=torch.float32,
                         chunk_iters=8, use_graphs=True)
        try:
            return _serve_fp32(srv, reqs)
        finally:
            srv.close()

    def _serve_fp32(srv, reqs):
        for shape in synth.SERVE_SHAPES:
            for lik in ("gauss", "poisson"):
                xi, b = inputs[shape][0]
                out = take_out(shape)
                srv.poll(srv.submit(shape, xi, b, None, lik=lik, rtol=SERVE_RTOL, maxiter=SERVE_MAXITER,
                                    response=SERVE_RESPONSE[lik], refine=SERVE_REFINE, x64_out=out), -1)
                free[shape].append(out)
        results = [None] * len(reqs)
        ids = [None] * len(reqs)
        kept = {}
        ready = threading.Semaphore(0)

        def poller():
            for i in range(len(reqs)):
                ready.acquire()
                r = srv.poll(ids[i][0], 600000)
                if r is None:  # not done after 10 minutes: count it as failed
                    r = {"status": -1, "error": "no result within 600 s", "t_done": time.monotonic(),
                         "iters": [0] * SERVE_SAMPLES, "relres": [float("inf")] * SERVE_SAMPLES}
                results[i] = r
                key = (reqs[i][1], reqs[i][2])
                if key not in kept and r["status"] == 0:
                    kept[key] = (i % pool, ids[i][1].clone())
                with lock:
                    free[reqs[i][1]].append(ids[i][1])

        th = threading.Thread(target=poller, daemon=True)
        th.start()
        t0 = time.monotonic()
        for i, (ta, shape, lik) in enumerate(reqs):
            dt = t0 + ta - time.monotonic()
            if dt > 0:
                time.sleep(dt)
            xi, b = inputs[shape][i % pool]
            out = take_out(shape)
            ids[i] = (srv.submit(shape, xi, b, None, lik=lik, rtol=SERVE_RTOL, maxiter=SERVE_MAXITER,
                                 response=SERVE_RESPONSE[lik], refine=SERVE_REFINE, x64_out=out), out)
            ready.release()
        th.join()
        st = srv.stats()
        lat32 = [1e3 * (r["t_done"] - (t0 + reqs[i][0])) for i, r in enumerate(results)]
        errors = []
        for r in results:
            if r["status"] != 0 and r["error"] not in errors and len(errors) < 5:
                errors.append(r["error"])
        ok32 = sum(1 for r in results if r["status"] == 0)
        end32 = max(r["t_done"] for r in results)
        its32 = [max(r["iters"][:SERVE_SAMPLES]) for r in results]
        by_class = {}
        for i, r in enumerate(results):
            key = "x".join(str(d) for d in reqs[i][1]) + "_" + reqs[i][2]
            c = by_class.setdefault(key, {"n": 0, "converged": 0, "iters": [], "lat": []})
            c["n"] += 1
            c["converged"] += int(r["status"] == 0)
            c["iters"].append(max(r["iters"][:SERVE_SAMPLES]))
            c["lat"].append(lat32[i])
        by_class = {k: {"n": v["n"], "converged": v["converged"], "mean_iters": float(np.mean(v["iters"])),
                        "p50_ms": _pctl(v["lat"], 50), "p99_ms": _pctl(v["lat"], 99)}
                    for k, v in sorted(by_class.items())}
        res = {"p50_ms": _pctl(lat32, 50), "p99_ms": _pctl(lat32, 99), "mean_ms": float(np.mean(lat32)),
               "solves_per_s": SERVE_SAMPLES * len(reqs) / (end32 - t0), "converged": ok32,
               "mean_iters": float(np.mean(its32)),
               "max_true_relres": max(max(r["relres"][:SERVE_SAMPLES]) for r in results),
               "refine_passes_max": SERVE_REFINE,
               "slots": args.serve_slots, "graph_replays": st["graph_replays"], "chunks": st["chunks"],
               "slot_objects_created": st["created"], "reused": st["reused"], "evicted": st["evicted"],
               "peak_reserved_gb": st["peak_reserved"] / 1e9, "budget_gb": st["budget"] / 1e9,
               "failed": len(results) - ok32, "errors": errors, "by_class": by_class,
               # the time the server needed for the stream against the span of its arrivals
               "busy_s": end32 - t0, "arrival_span_s": reqs[-1][0]}
        return res, kept

    fp32, kept32 = serve_fp32(0, reqs)
    fp32_budget = None
    if args.serve_budget_gb > 0:
        fp32_budget, _ = serve_fp32(int(args.serve_budget_gb * 1e9), reqs[:args.serve_budget_requests])
        fp32_budget["requests"] = min(len(reqs), args.serve_budget_requests)
    # a slower stream of the same mix that one server keeps up with: latency
    # without the queueing of the 50/s stream
    fp32_sustained = None
    if args.serve_sustained_requests > 0:
        reqs_s = synth.request_stream(synth.SEED_STREAM + 1, n=args.serve_sustained_requests,
                                      rate=args.serve_sustained_rate)
        fp32_sustained, _ = serve_fp32(0, reqs_s)
        fp32_sustained.update({"requests": len(reqs_s), "rate_hz": args.serve_sustained_rate})

    # ---- plain sequential FP64 path
    plans = {shape: nre.CorrelatedField(shape, amplitude="power", prior=dict(synth.AMP_PRIOR),
                                        dtype=torch.float64) for shape in synth.SERVE_SHAPES}
    liks = {"gauss": nre.Likelihood("gauss", sigma=0.1, response=SERVE_RESPONSE["gauss"]),
            "poisson": nre.Likelihood("poisson", scale=10.0)}
    dev = torch.device("cuda", torch.cuda.current_device())
    inp64 = {shape: [(xi.double().pin_memory(), b.double().pin_memory()) for (xi, b) in sets]
             for shape, sets in inputs.items()}

    def plain(shape, lik, k):
        plan = plans[shape]
        xi, b = inp64[shape][k]
        xp = torch.zeros(plan.stride, dtype=torch.float64, device=dev)
        xp[:plan.latent_size].copy_(xi, non_blocking=True)
        M = nre.Metric(plan, liks[lik], xp, max_batch=1)
        M.set_precond("harmonic")
        bd = torch.zeros(1, plan.stride, dtype=torch.float64, device=dev)
        xd = torch.zeros_like(bd)
        out = torch.empty_like(b).pin_memory()
        its, rels, sts = [], [], []
        for s_ in range(SERVE_SAMPLES):
            bd[0, :plan.latent_size].copy_(b[s_], non_blocking=True)
            _, it, rel, st_ = M.cg(bd, rtol=SERVE_RTOL, maxiter=SERVE_MAXITER, x=xd)
            out[s_].copy_(xd[0, :plan.latent_size])
            its.append(it[0])
            rels.append(rel[0])
            sts.append(st_)
        torch.cuda.synchronize()
        return max(its), max(rels), all(v == 0 for v in sts), out

    def true_relres(shape, lik, k, x):
        """FP64 ||b - M x|| / ||b|| of the 8 solutions x (host) of input set k."""
        plan = plans[shape]
        xi, b = inp64[shape][k]
        xp = torch.zeros(plan.stride, dtype=torch.float64, device=dev)
        xp[:plan.latent_size].copy_(xi)
        M = nre.Metric(plan, liks[lik], xp, max_batch=SERVE_SAMPLES)
        xd = plan.pad(x.to(dev).double())
        bd = plan.pad(b.to(dev))
        r = plan.unpad(bd - M.apply(xd))
        return float((r.norm(dim=1) / plan.unpad(bd).norm(dim=1)).max())

    true32 = {"x".join(str(d) for d in sh) + "_" + lik: true_relres(sh, lik, k, x)
              for (sh, lik), (k, x) in sorted(kept32.items())}
    fp32["true_relres_fp64_by_class"] = true32
    fp32["max_true_relres_sampled"] = max(true32.values()) if true32 else None

    for shape in synth.SERVE_SHAPES:
        plain(shape, "gauss", 0)
    lat64, its64, ok64, rel64 = [], [], 0, 0.0
    kept64 = {}
    t0 = time.monotonic()
    truncated = False
    for i, (ta, shape, lik) in enumerate(reqs):
        dt = t0 + ta - time.monotonic()
        if dt > 0:
            time.sleep(dt)
        it, rel, ok, x64 = plain(shape, lik, i % pool)
        if (shape, lik) not in kept64:
            kept64[(shape, lik)] = (i % pool, x64.clone())
        lat64.append(1e3 * (time.monotonic() - (t0 + ta)))
        its64.append(it)
        rel64 = max(rel64, rel)
        ok64 += int(ok)
        if time.monotonic() - t0 > args.serve_plain_cap_s:
            truncated = i + 1 < len(reqs)
            break
    end64 = time.monotonic()
    n64 = len(lat64)
    true64 = {"x".join(str(d) for d in sh) + "_" + lik: true_relres(sh, lik, k, x)
              for (sh, lik), (k, x) in sorted(kept64.items())}
    fp64 = {"true_relres_fp64_by_class": true64, "max_true_relres_sampled": max(true64.values()) if true64 else None,
            "p50_ms": _pctl(lat64, 50), "p99_ms": _pctl(lat64, 99), "mean_ms": float(np.mean(lat64)),
            "solves_per_s": SERVE_SAMPLES * n64 / (end64 - t0), "converged": ok64, "requests_served": n64,
            "mean_iters": float(np.mean(its64)), "max_relres": rel64,
            "truncated_at_s": args.serve_plain_cap_s if truncated else None}
    return {"requests": len(reqs), "rate_hz": 50.0, "samples_per_request": SERVE_SAMPLES, "rtol": SERVE_RTOL,
            "grids": [list(s) for s in synth.SERVE_SHAPES], "precond": "harmonic",
            "likelihoods": {"gauss": "sigma 0.1, identity response", "poisson": "rate 10 exp(cf)"},
            "fp32_batched": fp32, "fp32_batched_budget": fp32_budget, "fp32_batched_sustained": fp32_sustained,
            "fp64_sequential": fp64,
            "p50_speedup": fp64["p50_ms"] / fp32["p50_ms"], "p99_speedup": fp64["p99_ms"] / fp32["p99_ms"],
            "throughput_ratio": fp32["solves_per_s"] / fp64["solves_per_s"]}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    try:
        run_ours(args, rank, world)
    finally:
        if world > 1:
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
