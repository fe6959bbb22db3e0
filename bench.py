"""Benchmark: MIS-2 + aggregation (+ coarse graph) throughput on GB300.

Default workload (N=1): the 100^3 27-point grid (1,000,000 vertices,
25,463,592 directed entries, int32 CSR), one full coarsening level per step:
MIS-2 (Algorithm 1), aggregation (Algorithm 3) and the coarse graph.  The
metric is edges/s = input entries per step / step time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload 27pt|small|rmat|serve|ablation|setup|timeline]

- value: device-resident input, CUDA events around each step, L2 flushed
  (256 MiB write) before every step, outside the timed interval.
- e2e: the same metric through the host-buffer C entry point
  (mis2_coarsen_level_host): host->device copy of the CSR and device->host
  copy of every output inside the timed interval.
- roofline: the dominant kernel's algorithmic bytes (the per-round byte model
  applied to the worklist trace the library reports) over its CUDA-event time,
  the timed steps bracketing that kernel's launches alone
  (MIS2_TIMING_LOOP); the per-class breakdown (kernel_ms_per_step) comes from
  3 steps after the timed ones with every class bracketed.
- cpu_baseline: the CPU oracle on a bounded sample of the same workload.
- batched_vs_plain: 512 mixed graphs coarsened recursively, batched engine
  (autotuned) against per-graph plain launches (host and device loops).
- other_configs: the 100x100 5-point grid and R-MAT scale 22 levels, and the
  serving comparison (Poisson requests; serial, slots, merged launches), on
  the same line (--no-extra-configs skips them).
- N > 1 (torchrun): independent replicas, one per GPU (the method does not
  shard); value = all ranks' edges / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MIS-2+aggregation edges/sec and % HBM roofline on 1 GB300; batched vs plain graphs/sec"
NOMINAL_HBM_GBS = 8000.0


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _workload(name):
    from paper_2204_02934_gb300 import graphgen as gg

    if name == "27pt":
        return gg.workload_27pt(100), ("27-point 3D grid 100^3 (1,000,000 vertices, 25,463,592 directed entries, "
                                       "int32 CSR): MIS-2 + aggregation (Alg. 3) + coarse graph, seed 0")
    if name == "small":
        return gg.workload_small(), ("5-point 2D grid 100x100 (10,000 vertices, 39,600 directed entries): MIS-2 + "
                                     "aggregation (Alg. 3) + coarse graph, seed 0")
    if name == "rmat":
        g = gg.workload_rmat(22)
        return g, (f"R-MAT scale 22 (0.57,0.19,0.19,0.05), 8n pairs symmetrised: {g.n} vertices, {g.nnz} entries, "
                   "int64 rowptr: MIS-2 + aggregation (Alg. 3) + coarse graph, seed 0")
    raise SystemExit(f"unknown workload {name}")


# ------------------------------------------------------------------ byte model
def mis2_bytes(trace, n, s):
    """Algorithmic bytes of the MIS-2 rounds from the per-round worklist
    trace (W1, W2, D1, D2): row refresh 8*W1; column step (8+s)*W2 + 4*D2 +
    4*min(n, D2+W2); decide (8+s)*W1 + 4*D1 + 4*min(n, D1+W1); worklist
    compaction 12*(W1+W2)."""
    total = 0
    for w1, w2, d1, d2 in np.asarray(trace, dtype=np.int64).tolist():
        total += 8 * w1
        total += (8 + s) * w2 + 4 * d2 + 4 * min(n, d2 + w2)
        total += (8 + s) * w1 + 4 * d1 + 4 * min(n, d1 + w1)
        total += 12 * (w1 + w2)
    return total


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ dist
def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_model():
    """The host CPU as /proc/cpuinfo names it (x86: "model name"; Arm: the
    implementer / part codes), else the machine type."""
    try:
        info = open("/proc/cpuinfo").read().splitlines()
    except OSError:
        return platform.machine()
    for key in ("model name", "Model name"):
        for ln in info:
            if ln.startswith(key) and ":" in ln:
                return ln.split(":", 1)[1].strip()
    impl = next((ln.split(":", 1)[1].strip() for ln in info if ln.startswith("CPU implementer")), None)
    part = next((ln.split(":", 1)[1].strip() for ln in info if ln.startswith("CPU part")), None)
    if impl or part:
        return f"{platform.machine()} (CPU implementer {impl}, part {part})"
    return platform.machine()


def _cpu_baseline(g, budget_s=12.0):
    """The oracle, as it stands, on the same graph: repeat full levels until
    about budget_s of CPU time is spent (at least one)."""
    import oracle

    oracle.build()
    t0 = time.perf_counter()
    reps = 0
    while True:
        oracle.coarsen_level(g, seed=0)
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or el / reps * (reps + 1) > budget_s * 1.5:
            break
    return {"value": g.nnz * reps / el, "unit": "edges/s", "cores": 1, "kind": "oracle",
            "sample": f"{reps} full coarsening level(s) of the same graph, single-threaded C oracle, "
                      f"{el:.1f} s on {cpu_model()} ({os.cpu_count()} cores present)"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    g, desc = _workload(args.workload)
    import oracle

    oracle.build()
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.coarsen_level(g, seed=0)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    tot = sum(times)
    val = g.nnz * len(times) / tot
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "edges/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": {"workload": desc, "n": g.n, "nnz": g.nnz},
            "cpu_baseline": {"value": val, "unit": "edges/s", "cores": 1, "kind": "oracle",
                             "sample": f"{len(times)} full levels of the workload graph, single-threaded C oracle "
                                       f"on {cpu_model()}"},
            "e2e": {"value": val, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def max_over_ranks(x, ws, device=None):
    """The largest of every rank's x (torch.distributed MAX all-reduce; the
    backend's device: cuda for NCCL, cpu for gloo)."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(units_per_rank, local_seconds, ws, device=None):
    """Whole-job throughput of ws independent replicas (the method does not
    shard): every rank's units over the slowest rank's time."""
    return ws * units_per_rank / max_over_ranks(local_seconds, ws, device)


def run_ours(args):
    import torch

    from paper_2204_02934_gb300 import _build, mis2

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    _build.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    g, desc = _workload(args.workload)
    s_bytes = 8 if g.rowptr.dtype == np.int64 else 4
    loop = mis2.MIS2_LOOP_DEVICE if args.loop == "device" else mis2.MIS2_LOOP_HOST
    # timed steps: only the device-loop MIS-2 launches are bracketed by
    # events (the roofline's kernel time); the per-class breakdown comes from
    # separate fully instrumented steps after the timed region
    ctx = mis2.Context(g.n, g.nnz, loop=loop, timing=mis2.MIS2_TIMING_LOOP)
    dg = mis2.DeviceGraph.from_host(g, dev)
    n = g.n
    in_set = torch.empty(n, dtype=torch.uint8, device=dev)
    roots = torch.empty(n, dtype=torch.int32, device=dev)
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    c_rowptr = torch.empty(n + 1, dtype=torch.int32, device=dev)
    c_colind = torch.empty(g.nnz, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        return mis2.mis2_coarsen_level(ctx.handle, dg.csr, 0, in_set, roots, labels, c_rowptr, c_colind, g.nnz,
                                       stream)

    for _ in range(max(args.warmup, 3)):
        flush.fill_(1)
        step()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ms_total = 0.0
    kernel_ms = np.zeros(mis2.MIS2_NUM_KERNEL_CLASSES)
    kernel_launch = np.zeros(mis2.MIS2_NUM_KERNEL_CLASSES, dtype=np.int64)
    launches = 0
    loop_bytes = 0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    for _ in range(args.steps):
        flush.fill_(1)
        ev0.record(stream)
        nr, na, cn = step()
        ev1.record(stream)
        ev1.synchronize()
        ms_total += ev0.elapsed_time(ev1)
        st = ctx.stats()
        kernel_ms += np.array(st.kernel_ms[:])
        kernel_launch += np.array(st.kernel_launches[:], dtype=np.int64)
        launches += st.launches
        tr = np.array(st.trace, dtype=np.int64)[:min(st.rounds, mis2.MIS2_TRACE_CAP)]
        tr2 = np.array(st.trace2, dtype=np.int64)[:min(st.rounds2, mis2.MIS2_TRACE_CAP)]
        loop_bytes += mis2_bytes(tr, n, s_bytes) + mis2_bytes(tr2, n, s_bytes)
    torch.cuda.synchronize()
    ck = clocks.stop()
    value = replica_value(g.nnz * args.steps, ms_total / 1e3, ws, dev)
    # per-class breakdown: every class bracketed, kernels launched serially
    ctx.configure(timing=mis2.MIS2_TIMING_ALL)
    class_ms, class_steps = np.zeros(mis2.MIS2_NUM_KERNEL_CLASSES), 3
    for _ in range(class_steps):
        flush.fill_(1)
        step()
        class_ms += np.array(ctx.stats().kernel_ms[:])
    ctx.configure(timing=mis2.MIS2_TIMING_OFF)

    # ---- end to end through the host-buffer entry point
    rp_h = torch.from_numpy(np.ascontiguousarray(g.rowptr)).pin_memory()
    ci_h = torch.from_numpy(np.ascontiguousarray(g.colind)).pin_memory()
    o_in = torch.empty(n, dtype=torch.uint8).pin_memory()
    o_roots = torch.empty(n, dtype=torch.int32).pin_memory()
    o_labels = torch.empty(n, dtype=torch.int32).pin_memory()
    o_crp = torch.empty(n + 1, dtype=torch.int32).pin_memory()
    o_cci = torch.empty(g.nnz, dtype=torch.int32).pin_memory()
    hcsr = mis2.mis2_csr(n, g.nnz, 1 if s_bytes == 8 else 0, 0, rp_h.data_ptr(), ci_h.data_ptr())
    e2e_times, d2h = [], 0

    def e2e_step():
        return mis2.mis2_coarsen_level_host(ctx.handle, hcsr, 0, o_in, o_roots, o_labels, o_crp, o_cci, g.nnz,
                                            stream)

    for _ in range(2):
        e2e_step()
    for _ in range(max(2, min(args.steps, 5))):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nr, na, cn = e2e_step()
        e2e_times.append(time.perf_counter() - t0)
        d2h = n + 4 * nr + 4 * n + 4 * (na + 1) + 4 * cn
    h2d = rp_h.numel() * rp_h.element_size() + ci_h.numel() * 4
    e2e_val = replica_value(g.nnz * len(e2e_times), sum(e2e_times), ws, dev)

    if rank != 0:
        if ws > 1:
            dist.barrier()
            dist.destroy_process_group()
        return 0
    # ---- roofline of the dominant kernel class (the device loop: its
    # launches are the only ones the timed steps bracket)
    peak, peak_kind = _peaks()
    names = mis2.KERNEL_CLASSES
    dom = int(np.argmax(class_ms))
    dom_ms = kernel_ms[dom]
    roofline = None
    if names[dom] == "device_loop" and dom_ms > 0:
        achieved = loop_bytes / (dom_ms / 1e3) / 1e9
        roofline = {"bound": "hbm", "kernel": "k_mis_loop (MIS-2 rounds, device loop)",
                    "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "peak_kind": peak_kind, "frac_of_nominal_8tbs": achieved / NOMINAL_HBM_GBS,
                    "traffic": _traffic_from_profile("k_mis_loop", args.workload),
                    "bytes_per_step": loop_bytes / args.steps,
                    "kernel_ms_per_step": dom_ms / args.steps,
                    "launches_per_step": int(kernel_launch[dom] // args.steps)}
    breakdown = {names[k]: round(class_ms[k] / class_steps, 4) for k in range(len(names)) if class_ms[k] > 0}
    line = {"metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": ws, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": desc, "n": g.n, "nnz": g.nnz, "loop": args.loop,
                       "l2": "flushed (256 MiB write) before every timed step", "parallelism":
                       "replicas only" if ws > 1 else "single GPU"},
            "e2e": {"value": e2e_val, "unit": "edges/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches),
            "roofline": roofline,
            "kernel_ms_per_step": breakdown,
            "kernel_ms_note": "per kernel class, from 3 steps after the timed ones with every class bracketed by "
                              "CUDA events and the kernels launched serially",
            "clocks": ck,
            "mis2": {"n_roots": int(nr), "n_aggs": int(na), "c_nnz": int(cn)}}
    if not args.no_batch:
        line["batched_vs_plain"] = run_batch_compare()
    if not args.no_extra_configs and args.workload == "27pt":
        # the other single-graph configurations and serving, on the same line
        line["other_configs"] = {
            "small_5pt_100x100": level_config("small", steps=20, warmup=3, loop=args.loop),
            "rmat_scale22": level_config("rmat", steps=5, warmup=3, loop=args.loop),
            "serving_poisson": serve_compare(requests=4000, rate=2000.0, slots=4, batch_max=16, sat_requests=2000,
                                             below_requests=1000, loop=args.serve_loop),
        }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = _cpu_baseline(g, args.cpu_budget)
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def level_config(name, steps=10, warmup=3, loop="device"):
    """One more coarsening-level configuration for the bench line: the
    workload's graph (generated here, off the clock), levels through
    mis2_coarsen_level with input resident and L2 flushed before each, CUDA
    events around each level; the same through mis2_coarsen_level_host (host
    CSR in, every output out) for e2e."""
    import torch

    from paper_2204_02934_gb300 import mis2

    t_gen = time.perf_counter()
    g, desc = _workload(name)
    t_gen = time.perf_counter() - t_gen
    dev = torch.device("cuda", torch.cuda.current_device())
    lp = mis2.MIS2_LOOP_DEVICE if loop == "device" else mis2.MIS2_LOOP_HOST
    ctx = mis2.Context(g.n, g.nnz, loop=lp)
    dg = mis2.DeviceGraph.from_host(g, dev)
    n = g.n
    bufs = [torch.empty(n, dtype=torch.uint8, device=dev), torch.empty(n, dtype=torch.int32, device=dev),
            torch.empty(n, dtype=torch.int32, device=dev), torch.empty(n + 1, dtype=torch.int32, device=dev),
            torch.empty(g.nnz, dtype=torch.int32, device=dev)]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step = lambda: mis2.mis2_coarsen_level(ctx.handle, dg.csr, 0, *bufs, g.nnz, stream)
    for _ in range(max(warmup, 3)):
        flush.fill_(1)
        step()
    torch.cuda.synchronize()
    ms, launches = [], 0
    for _ in range(steps):
        flush.fill_(1)
        ev0.record(stream)
        nr, na, cn = step()
        ev1.record(stream)
        ev1.synchronize()
        ms.append(ev0.elapsed_time(ev1))
        st = ctx.stats()
        launches += st.launches
    rounds, rounds2 = int(st.rounds), int(st.rounds2)
    # per-class breakdown from 3 more levels, every class bracketed by events
    ctx.configure(timing=mis2.MIS2_TIMING_ALL)
    kernel_ms = np.zeros(mis2.MIS2_NUM_KERNEL_CLASSES)
    for _ in range(3):
        flush.fill_(1)
        step()
        kernel_ms += np.array(ctx.stats().kernel_ms[:]) / 3
    ctx.configure(timing=mis2.MIS2_TIMING_OFF)
    # e2e through the host-buffer entry point
    rp_h = torch.from_numpy(np.ascontiguousarray(g.rowptr)).pin_memory()
    ci_h = torch.from_numpy(np.ascontiguousarray(g.colind)).pin_memory()
    outs = [torch.empty(n, dtype=torch.uint8).pin_memory(), torch.empty(n, dtype=torch.int32).pin_memory(),
            torch.empty(n, dtype=torch.int32).pin_memory(), torch.empty(n + 1, dtype=torch.int32).pin_memory(),
            torch.empty(g.nnz, dtype=torch.int32).pin_memory()]
    hcsr = mis2.mis2_csr(n, g.nnz, 1 if g.rowptr.dtype == np.int64 else 0, 0, rp_h.data_ptr(), ci_h.data_ptr())
    e2e_step = lambda: mis2.mis2_coarsen_level_host(ctx.handle, hcsr, 0, *outs, g.nnz, stream)
    for _ in range(2):
        e2e_step()
    e2e = []
    for _ in range(max(2, min(steps, 5))):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step()
        e2e.append(time.perf_counter() - t0)
    ctx.close()
    tot = sum(ms) / 1e3
    names = mis2.KERNEL_CLASSES
    return {"workload": desc, "n": g.n, "nnz": g.nnz, "value": g.nnz * len(ms) / tot, "unit": "edges/s",
            "ms_per_level": 1e3 * tot / len(ms), "steps": len(ms),
            "kernel_ms_per_level": {names[k]: round(kernel_ms[k], 4) for k in range(len(names))
                                    if kernel_ms[k] > 0},
            "gpu_launches_per_level": launches // len(ms), "rounds": rounds, "rounds_phase2": rounds2,
            "mis2": {"n_roots": int(nr), "n_aggs": int(na), "c_nnz": int(cn)},
            "e2e": {"value": g.nnz * len(e2e) / sum(e2e), "unit": "edges/s"},
            "generation_s": round(t_gen, 1), "l2": "flushed (256 MiB write) before every timed level"}


def run_batch_compare(steps=3, warmup=2, n_graphs=512, seed=7, min_n=1000):
    """Batched hierarchies vs per-graph plain launches on the mixed-size batch
    (2D 5-pt / 3D 7-pt / 2D RGG, 1k-200k vertices, log-uniform), each graph
    coarsened recursively until it has fewer than min_n vertices.

    The batched arm runs with the configuration the autotuner picks for this
    batch (autotune.tune_batch: lanes per low-degree row and resident blocks
    of the persistent loop, each candidate checked element by element against
    the default configuration's output).  Two plain arms: one
    mis2_coarsen_level call per graph and level, with the host-driven round
    loop and with the persistent device loop.  Every arm is timed the same
    way: CUDA events around the whole pass, L2 flushed before it.  Returns a
    dict with graphs/s of every arm and the identity checks."""
    import torch

    from paper_2204_02934_gb300 import autotune, graphgen as gg, mis2

    graphs = gg.mixed_batch(n_graphs, seed=seed)
    tot_n, tot_nnz = sum(g.n for g in graphs), sum(g.nnz for g in graphs)
    dgs = [mis2.DeviceGraph.from_host(g) for g in graphs]
    tuned, tuned_ms, table = autotune.tune_batch(graphs, seed=0, min_n=min_n, reps=2)
    b = mis2.Batch(n_graphs, tot_n, tot_nnz, cfg=autotune._config(tuned))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        t, out = 0.0, None
        for _ in range(reps):
            flush.fill_(1)
            ev0.record()
            out = fn()
            ev1.record()
            ev1.synchronize()
            t += ev0.elapsed_time(ev1) / 1e3
        return t / reps, out

    for _ in range(max(warmup, 1)):
        nlev = b.coarsen(dgs, min_n=min_n)
    launches = 0
    t_b = 0.0
    for _ in range(steps):
        dt, nlev = timed(lambda: b.coarsen(dgs, min_n=min_n), 1)
        t_b += dt
        launches += b.stats().launches
    t_b /= steps
    batched = n_graphs / t_b

    maxn = max(g.n for g in graphs)
    maxnnz = max(g.nnz for g in graphs)

    def plain_pass(ctx, record=False):
        out = []
        for dg in dgs:
            cur, levels = dg, []
            while cur.n >= min_n and len(levels) < 32:
                r = ctx.coarsen_level(cur, 0)
                levels.append(r["labels"] if record else None)
                if r["n_aggs"] >= cur.n:
                    break
                cur = mis2.DeviceGraph(r["n_aggs"], int(r["c_colind"].numel()), r["c_rowptr"],
                                       r["c_colind"] if r["c_colind"].numel() else torch.zeros(4, dtype=torch.int32,
                                                                                             device="cuda"))
            out.append(levels)
        return out

    arms = {}
    for name, loop in (("plain_host_loop", mis2.MIS2_LOOP_HOST), ("plain_device_loop", mis2.MIS2_LOOP_DEVICE)):
        ctx = mis2.Context(maxn, maxnnz, loop=loop)
        ref = plain_pass(ctx, record=True)
        torch.cuda.synchronize()
        dt, _ = timed(lambda: plain_pass(ctx), 1)
        same = True
        for gi in range(n_graphs):
            for L, lab in enumerate(ref[gi]):
                if not torch.equal(b.labels(L, gi), lab):
                    same = False
                    break
            if not same:
                break
        arms[name] = {"graphs_per_s": n_graphs / dt, "ms": 1e3 * dt, "identical_output": same}
        ctx.close()
    fastest_plain = max(a["graphs_per_s"] for a in arms.values())
    return {"workload": f"{n_graphs} mixed graphs (2D 5-pt, 3D 7-pt, 2D RGG; 1k-200k vertices, log-uniform, "
                        f"{tot_n} vertices, {tot_nnz} entries), recursive coarsening until < {min_n} vertices",
            "unit": "graphs/s", "batched": batched, "batched_ms": 1e3 * t_b, "levels": nlev,
            "batched_config": {k: int(v) for k, v in tuned.items()},
            "autotune_candidates": [{"config": {k: int(v) for k, v in r["config"].items()},
                                     "ms": round(r["ms"], 3), "identical": r["identical"]} for r in table],
            "plain": fastest_plain, "plain_arms": arms, "speedup": batched / fastest_plain,
            "speedup_vs_host_loop_plain": batched / arms["plain_host_loop"]["graphs_per_s"],
            "identical_output": all(a["identical_output"] for a in arms.values()),
            "timing": "CUDA events around each whole pass, L2 flushed before it",
            "batched_gpu_launches_per_step": launches // steps}


def serve_compare(requests=20000, rate=2000.0, slots=4, batch_max=16, sat_requests=4000, below_requests=4000,
                  loop="auto"):
    """Serving: a Poisson stream of one-level requests (H2D of the CSR, MIS-2,
    aggregation, coarse graph, D2H of every output) drawn from a pool of 64
    pinned-host graphs (3D 7-pt grids of side 20-160 and R-MAT graphs of scale
    14-20, average degree 16).  Three servers: serial plain launches (one
    slot, one request at a time), `slots` slots of one request each, and
    merged launches (two slots, each running up to `batch_max` queued
    requests as one union through the batched engine).  Per server: p50/p99
    latency at the offered rate, throughput with every request queued at once
    (saturation), and p50/p99 at 50 % and 80 % of the merged server's
    saturation rate (below saturation, so latency is service time plus short
    queueing); each request's result fingerprint must be the same in every
    server.  loop "auto": each server on the round loop that suits it, the
    device loop for the single slot and the host-driven loop for several
    slots (device-loop kernels of different slots run one at a time, their
    per-round kernels interleave); "device" or "host": every server on it."""
    from paper_2204_02934_gb300 import graphgen as gg

    t_gen = time.perf_counter()
    pool = gg.serving_pool(64, processes=max(1, min(16, os.cpu_count() or 1)))
    t_gen = time.perf_counter() - t_gen
    import torch

    from paper_2204_02934_gb300 import _build, mis2

    _build.build()
    torch.cuda.init()
    pins, host = [], []
    for g in pool:
        rp = torch.from_numpy(np.ascontiguousarray(g.rowptr)).pin_memory()
        ci = torch.from_numpy(np.ascontiguousarray(g.colind)).pin_memory()
        pins.append((rp, ci))
        host.append(mis2.mis2_csr(g.n, g.nnz, 1 if rp.dtype == torch.int64 else 0, 0, rp.data_ptr(),
                                  ci.data_ptr() if g.nnz else None))
    max_n, max_nnz = max(g.n for g in pool), max(g.nnz for g in pool)
    arrivals = gg.poisson_arrivals(requests, rate, seed=13)
    idx = np.minimum((gg.uniform01(np.arange(requests, dtype=np.uint64), 17) * len(pool)).astype(np.int32),
                     len(pool) - 1)
    n_sat = min(requests, sat_requests)
    n_below = min(requests, below_requests)

    def summarize(res, t_first):
        lat = np.array([r.t_done - r.t_arrive for r in res])
        svc = np.array([r.t_done - r.t_start for r in res])
        span = max(r.t_done for r in res) - t_first
        return {"graphs_per_s": len(res) / span, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                "p99_ms": 1e3 * float(np.percentile(lat, 99)), "mean_ms": 1e3 * float(lat.mean()),
                "service_mean_ms": 1e3 * float(svc.mean())}

    servers = (("serial", 1, 0, max_n, max_nnz), ("slots", slots, 0, max_n, max_nnz),
               ("merged", 2, batch_max, max(4 * max_n, 1 << 22), max(4 * max_nnz, 1 << 26)))
    out, sums, handles = {}, {}, {}
    loops = {}
    for name, sl, bm, sn, snnz in servers:
        lp = loop if loop != "auto" else ("device" if sl == 1 else "host")
        loops[name] = lp
        srv = mis2.Server(slots=sl, slot_max_n=sn, slot_max_nnz=snnz, mem_budget=96 << 30, batch_max=bm,
                          loop=mis2.MIS2_LOOP_DEVICE if lp == "device" else mis2.MIS2_LOOP_HOST)
        srv.replay(host, np.zeros(len(pool)), np.arange(len(pool), dtype=np.int32), seed=0)  # warm-up
        res, mif = srv.replay(host, arrivals, idx, seed=0)
        if any(r.status != 0 for r in res):
            raise SystemExit(f"serving: a request failed ({name})")
        open_loop = summarize(res, min(r.t_arrive for r in res))
        open_loop["max_in_flight"] = mif
        sums[name] = [r.checksum for r in res]
        res2, mif2 = srv.replay(host, np.zeros(n_sat), idx[:n_sat], seed=0)
        sat = summarize(res2, min(r.t_arrive for r in res2))
        sat["max_in_flight"] = mif2
        sums[name + "_sat"] = [r.checksum for r in res2]
        out[name] = {"slots": sl, "batch_max": bm, "open_loop": open_loop, "saturation": sat}
        handles[name] = srv
    sat_rate = out["merged"]["saturation"]["graphs_per_s"]
    for name, srv in handles.items():
        below = {}
        for frac in (0.5, 0.8):
            arr = gg.poisson_arrivals(n_below, frac * sat_rate, seed=29)
            res3, mif3 = srv.replay(host, arr, idx[:n_below], seed=0)
            sm = summarize(res3, min(r.t_arrive for r in res3))
            sm.update(offered_req_per_s=round(frac * sat_rate, 1), max_in_flight=mif3)
            below[f"{int(frac * 100)}pct_of_merged_saturation"] = sm
            sums.setdefault(name + "_below", []).extend(r.checksum for r in res3)
        out[name]["below_saturation"] = below
        srv.close()
    same = all(sums[k] == sums["serial" + k[len(k.split("_")[0]):]] for k in sums)
    per_graph = {}
    for i, h in zip(idx, sums["serial"]):
        per_graph.setdefault(int(i), set()).add(h)
    same = same and all(len(v) == 1 for v in per_graph.values())
    return {
        "workload": f"{requests} requests, Poisson arrivals at {rate:g} req/s (seed 13), drawn uniformly from 64 "
                    f"pinned-host graphs (3D 7-pt side log-uniform 20-160 / R-MAT scale 14-20, avg degree 16, seed "
                    f"11; {sum(g.nnz for g in pool)} entries in the pool); saturation: {n_sat} requests queued at "
                    f"t=0; below saturation: {n_below} requests at 50 % and 80 % of the merged server's saturation",
        "unit": "graphs/s", "loop": loops,
        "serial": out["serial"], "slots": out["slots"], "merged": out["merged"],
        "speedup_vs_serial_at_saturation": {k: out[k]["saturation"]["graphs_per_s"] /
                                            out["serial"]["saturation"]["graphs_per_s"] for k in ("slots", "merged")},
        "identical_output": bool(same), "pool_generation_s": round(t_gen, 1),
    }


def run_serve(args):
    """--workload serve: serve_compare at the command line's sizes, one JSON line."""
    sc = serve_compare(args.requests, args.rate, args.slots, args.batch_max, args.saturation_requests,
                       args.below_requests, args.serve_loop)
    line = {"metric": "serving graphs/s at saturation and p50/p99 latency (one coarsening level per request, "
                      "H2D + compute + D2H)",
            "value": round(sc["merged"]["saturation"]["graphs_per_s"], 1), "unit": "graphs/s",
            "higher_is_better": True, "n_gpus": 1, "dtype": "int32", "data": "synthetic",
            "config": {"workload": sc["workload"], "slots": args.slots, "batch_max": args.batch_max,
                       "loop": sc["loop"]},
            **{k: v for k, v in sc.items() if k not in ("workload",)}}
    print(json.dumps(line), flush=True)
    return 0


def run_ablation(args):
    """Fig. 2 / Table I on GB300: MIS-2 (Algorithm 1) alone on the regenerated
    Laplace3D_100 (7-point 100^3) and Elasticity3D_60 (27-point x 3 dof
    60^3), with each optimisation switched off in turn: worklists, random
    (xorshift*) priorities -> fixed priorities or plain xorshift, and the
    packed tuple: the plain tuple engine with packed and with unpacked
    tuples (the packing's gain is their ratio).  Device loop, input
    resident, L2 flushed before each timed run."""
    import torch

    from paper_2204_02934_gb300 import _build, graphgen as gg, mis2

    _build.build()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    variants = [("all optimisations", {}),
                ("no worklists", {"ablation": mis2.MIS2_ABLATE_NO_WORKLISTS}),
                ("fixed priorities (no random tie-break per round)", {"hash_variant": mis2.MIS2_HASH_FIXED}),
                ("xorshift instead of xorshift*", {"hash_variant": mis2.MIS2_HASH_XORSHIFT}),
                ("packed tuples, plain engine", {"ablation": mis2.MIS2_ABLATE_TUPLE_ENGINE}),
                ("unpacked 3-tuples, plain engine", {"ablation": mis2.MIS2_ABLATE_UNPACKED_TUPLES})]
    graphs = [("Laplace3D_100 (7-point 100^3)", gg.grid3d_7pt(100, 100, 100)),
              ("Elasticity3D_60 (27-point x 3 dof, 60^3)", gg.elasticity3d(60, 60, 60))]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rows = []
    for gname, g in graphs:
        dg = mis2.DeviceGraph.from_host(g)
        ref = None
        for vname, over in variants:
            ctx = mis2.Context(g.n, g.nnz, loop=mis2.MIS2_LOOP_DEVICE if args.loop == "device" else
                               mis2.MIS2_LOOP_HOST, **over)
            for _ in range(max(args.warmup, 3)):
                in_set, roots, rounds = ctx.run(dg, 0)
            times = []
            for _ in range(args.steps):
                flush.fill_(1)
                ev0.record()
                in_set, roots, rounds = ctx.run(dg, 0)
                ev1.record()
                ev1.synchronize()
                times.append(ev0.elapsed_time(ev1))
            if ref is None:
                ref = in_set.clone()
            same = bool(torch.equal(in_set, ref)) if ("worklists" in vname or "packed tuples" in vname) else None
            rows.append({"graph": gname, "n": g.n, "nnz": g.nnz, "variant": vname, "rounds": int(rounds),
                         "mis2_size": int(roots.numel()), "ms": round(float(np.median(times)), 4),
                         "same_result_as_all": same})
            ctx.close()
    base = {r["graph"]: r["ms"] for r in rows if r["variant"] == "all optimisations"}
    plain = {r["graph"]: r["ms"] for r in rows if r["variant"] == "packed tuples, plain engine"}
    for r in rows:
        r["slowdown_vs_all"] = round(r["ms"] / base[r["graph"]], 3)
        if r["variant"] == "unpacked 3-tuples, plain engine":
            r["slowdown_vs_packed_plain_engine"] = round(r["ms"] / plain[r["graph"]], 3)
    line = {"metric": "MIS-2 time per variant (Fig. 2 ablation, Table I rounds) on GB300", "unit": "ms",
            "higher_is_better": False, "n_gpus": 1, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "Laplace3D_100 and Elasticity3D_60 regenerated from their definitions, seed 0",
                       "loop": args.loop, "steps": args.steps},
            "rows": rows}
    print(json.dumps(line), flush=True)
    return 0


def run_setup(args):
    """The steps that follow the coarse graph in a multilevel method, on
    GB300: the coarse edge weights and the tentative prolongator (Section
    III-B), the colour sets (on the coarse graph) and cluster lists of
    cluster multicolor Gauss-Seidel (Algorithm 4's setup), and distance-k MIS
    for k = 1, 2, 3 (Algorithm 1 generalised; host-driven rounds over every
    vertex).  Inputs resident; L2 flushed before each timed call; CUDA events
    around each call (each synchronises).  Algorithmic bytes of the
    bandwidth-bound steps: weights 4(n+1) + 8n + 8nnz + 8c_nnz (rowptr,
    labels of u, colind and the labels it gathers, the coarse row searched
    and its weights written); prolongator 28n + 4 (two reads of labels, the
    size gather, rowptr/colind/value writes); cluster lists 4n (key
    histogram) + per 8-bit radix pass 8n of key reads, 4n of value writes,
    4n of value reads after the first pass and 4n of key writes before the
    last.  cpu_baseline of each row: the oracle's restatement of the same
    step on the same input (single-threaded C, or numpy for the grouping),
    timed once on the host cores (skipped with --no-cpu-baseline)."""
    import time

    import torch

    from paper_2204_02934_gb300 import _build, graphgen as gg, mis2

    _build.build()
    peak, peak_kind = _peaks()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    graphs = [("27-point 100^3 grid", gg.workload_27pt(100)),
              ("R-MAT scale 20, 8 pairs per vertex", gg.rmat(20, 8, seed=42))]

    def timed(fn):
        for _ in range(max(args.warmup, 3)):
            out = fn()
        ts = []
        for _ in range(args.steps):
            flush.fill_(1)
            ev0.record()
            out = fn()
            ev1.record()
            ev1.synchronize()
            ts.append(ev0.elapsed_time(ev1))
        return float(np.median(ts)), out

    rows = []
    for gname, g in graphs:
        dg = mis2.DeviceGraph.from_host(g)
        ctx = mis2.Context(g.n, g.nnz, loop=mis2.MIS2_LOOP_DEVICE if args.loop == "device" else
                           mis2.MIS2_LOOP_HOST)
        lv = ctx.coarsen_level(dg, 0)
        labels, na = lv["labels"], int(lv["n_aggs"])
        crp, cci = lv["c_rowptr"], lv["c_colind"]
        cg = mis2.DeviceGraph(na, int(cci.numel()), crp, cci if cci.numel() else torch.zeros(4, dtype=torch.int32,
                                                                                                device="cuda"))
        c_nnz = int(cci.numel())
        w = torch.empty(max(c_nnz, 1), dtype=torch.int32, device="cuda")
        prp = torch.empty(g.n + 1, dtype=torch.int32, device="cuda")
        pci = torch.empty(g.n, dtype=torch.int32, device="cuda")
        pvl = torch.empty(g.n, dtype=torch.float64, device="cuda")
        colors = torch.empty(max(na, 1), dtype=torch.int32, device="cuda")
        cptr = torch.empty(na + 1, dtype=torch.int32, device="cuda")
        clist = torch.empty(max(na, 1), dtype=torch.int32, device="cuda")
        kptr = torch.empty(na + 1, dtype=torch.int32, device="cuda")
        kmem = torch.empty(g.n, dtype=torch.int32, device="cuda")
        in_set = torch.empty(g.n, dtype=torch.uint8, device="cuda")
        roots = torch.empty(g.n, dtype=torch.int32, device="cuda")
        base = {"graph": gname, "n": g.n, "nnz": g.nnz, "n_aggs": na, "c_nnz": c_nnz}

        h_labels = labels.cpu().numpy()
        h_crp, h_cci = crp.cpu().numpy(), cci.cpu().numpy()
        h_cg = gg.CSRGraph(na, h_crp.astype(np.int32), h_cci)

        def cpu_time(fn):
            if args.no_cpu_baseline:
                return None
            import oracle

            t0 = time.perf_counter()
            fn(oracle)
            return {"ms": round((time.perf_counter() - t0) * 1e3, 2), "cores": 1, "kind": "oracle",
                    "sample": "the same call on the same input, once"}

        def add(step, ms, items, item_unit, bytes_=None, cpu=None, **extra):
            r = dict(base, step=step, ms=round(ms, 4), throughput=items / (ms * 1e-3), throughput_unit=item_unit,
                     **extra)
            if cpu is not None:
                r["cpu_baseline"] = cpu
            if bytes_ is not None:
                gbs = bytes_ / (ms * 1e-3) / 1e9
                r["roofline"] = {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                                 "frac": round(gbs / peak, 3), "algorithmic_bytes": int(bytes_),
                                 "peak_kind": peak_kind}
            rows.append(r)

        ms, _ = timed(lambda: mis2.mis2_coarse_weights(ctx.handle, dg.csr, labels, na, crp, cci, w))
        add("coarse edge weights", ms, g.nnz, "fine entries/s", 4 * (g.n + 1) + 8 * g.n + 8 * g.nnz + 8 * c_nnz,
            cpu_time(lambda o: o.coarse_weights(g, h_labels, na, h_crp, h_cci)) if "R-MAT" not in gname else
            {"skipped": "the oracle scans each coarse row linearly; on the R-MAT hubs that is about 30 s"})
        ms, _ = timed(lambda: mis2.mis2_tentative_prolongator(ctx.handle, labels, g.n, na, 1, prp, pci, pvl))
        add("tentative prolongator", ms, g.n, "fine rows/s", 28 * g.n + 4,
            cpu_time(lambda o: o.prolongator(h_labels, na)))
        ms, (nc, rounds) = timed(lambda: mis2.mis2_color(ctx.handle, cg.csr, 0, colors, cptr, clist))
        add("colour sets of the coarse graph", ms, na, "coarse vertices/s", None,
            cpu_time(lambda o: o.color_sets(*o.color_greedy(h_cg, 0))), n_colors=nc, rounds=rounds)
        passes = max(1, (max(1, (na - 1).bit_length()) + 7) // 8)
        cl_bytes = 4 * g.n + sum(8 * g.n + 4 * g.n + (4 * g.n if p > 0 else 0) + (4 * g.n if p < passes - 1 else 0)
                                 for p in range(passes))
        ms, _ = timed(lambda: mis2.mis2_cluster_lists(ctx.handle, labels, g.n, na, kptr, kmem))
        add("cluster lists", ms, g.n, "fine rows/s", cl_bytes, cpu_time(lambda o: o.cluster_lists(h_labels, na)),
            radix_passes=passes)
        for k in (1, 2, 3):
            ms, (nr, rounds) = timed(lambda: mis2.mis2_run_k(ctx.handle, dg.csr, k, 0, in_set, roots))
            add(f"distance-{k} MIS", ms, g.nnz, "edges/s", None, cpu_time(lambda o: o.misk(g, k, 0)), set_size=nr,
                rounds=rounds)
        ctx.close()
    line = {"metric": "setup steps after the coarse graph on GB300 (time per call)", "unit": "ms",
            "higher_is_better": False, "n_gpus": 1, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "27-point 100^3 grid and R-MAT scale 20 (seed 42), level-0 aggregation, seed 0",
                       "loop": args.loop, "steps": args.steps,
                       "l2": "flushed (256 MiB write) before each timed call"},
            "rows": rows}
    print(json.dumps(line), flush=True)
    return 0


def _traffic_from_profile(kernel, workload):
    """dram bytes per launch recorded by an ncu capture of this kernel on this
    workload, when the recorded source digest still matches the library
    sources (None otherwise)."""
    p = os.path.join(ROOT, "profiles", f"{kernel}_traffic.txt")
    if not os.path.exists(p):
        return None
    vals = {}
    for ln in open(p):
        if ":" in ln:
            k, v = ln.split(":", 1)
            vals[k.strip()] = v.strip()
    try:
        from paper_2204_02934_gb300 import _build

        files = vals["source_files"].split() if "source_files" in vals else None
        if vals.get("workload_key") != workload or vals.get("source_digest") != _build.source_digest(files):
            return None
        return float(vals["dram_bytes_per_launch"])
    except Exception:
        return None


def run_timeline(args):
    """--workload timeline: GPU activity trace (CUPTI) of one coarsening level
    of --graph (27pt, small or rmat), with the short kernels launched with
    programmatic dependent launch (the default) and serially; per case the
    level's span, the time covered by at least one operation, the idle time
    between operations and every operation in order.  Not a bench value (the
    trace itself costs a little per operation)."""
    import torch

    from paper_2204_02934_gb300 import mis2, trace

    g, desc = _workload(args.graph)
    dev = torch.device("cuda", 0)
    dg = mis2.DeviceGraph.from_host(g, dev)
    n = g.n
    bufs = [torch.empty(n, dtype=torch.uint8, device=dev), torch.empty(n, dtype=torch.int32, device=dev),
            torch.empty(n, dtype=torch.int32, device=dev), torch.empty(n + 1, dtype=torch.int32, device=dev),
            torch.empty(g.nnz, dtype=torch.int32, device=dev)]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    cases = {}
    for label, serial in (("overlapped", 0), ("serial", 1)):
        ctx = mis2.Context(g.n, g.nnz, loop=mis2.MIS2_LOOP_DEVICE, serial_launches=serial)
        step = lambda: mis2.mis2_coarsen_level(ctx.handle, dg.csr, 0, *bufs, g.nnz, stream)
        for _ in range(max(args.warmup, 3)):
            flush.fill_(1)
            step()
        flush.fill_(1)
        with trace.GpuTrace() as t:
            step()
        ctx.close()
        t0 = t.records[0]["start_ns"] if t.records else 0
        cases[label] = dict(trace.summary(t.records), timeline=[
            [round((r["start_ns"] - t0) / 1e3, 1), round((r["end_ns"] - r["start_ns"]) / 1e3, 1),
             trace.short_name(r["name"]) if r["kind"] == "kernel" else r["name"]] for r in t.records])
    print(json.dumps({"workload": desc, "timeline": cases,
                      "note": "one level after 3 warm-up levels, L2 flushed before it; start and duration in us"}),
          flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="27pt", choices=["27pt", "small", "rmat", "serve", "ablation",
                                                                    "setup", "timeline"])
    ap.add_argument("--graph", default="27pt", choices=["27pt", "small", "rmat"], help="timeline: the level's graph")
    ap.add_argument("--loop", default="device", choices=["device", "host"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-vs-plain comparison")
    ap.add_argument("--no-extra-configs", action="store_true",
                    help="skip the 100x100 5-point grid, R-MAT scale 22 and serving entries of the default line")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--requests", type=int, default=20000, help="serve: requests in the Poisson stream")
    ap.add_argument("--rate", type=float, default=2000.0, help="serve: offered requests/s")
    ap.add_argument("--slots", type=int, default=4, help="serve: continuous-batching slots")
    ap.add_argument("--saturation-requests", type=int, default=4000)
    ap.add_argument("--below-requests", type=int, default=4000, help="serve: requests per below-saturation rate")
    ap.add_argument("--batch-max", type=int, default=16, help="serve: requests per merged launch")
    ap.add_argument("--serve-loop", default="auto", choices=["auto", "device", "host"],
                    help="serving round loop: auto = device loop for the single slot, host loop for several")
    args = ap.parse_args()
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "ablation":
        return run_ablation(args)
    if args.workload == "setup":
        return run_setup(args)
    if args.workload == "timeline":
        return run_timeline(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
