"""Benchmark of the fused three-lattice MRT-LB step on GB300.

One bench step = one pass of the whole hot path over the cavity: 100 time
steps of the fused collide-stream kernel (pull streaming with wall rules,
macroscopic fields, porous force, D2Q9 + 2 x D2Q5 MRT collisions) plus the
FP64 Nu/Sh wall reduction and the steady-state residual.  Workload: the
4096 x 4096 opposing-buoyancy porous cavity (Ra = 1e5, Da = 1e-3, eps = 0.4,
Pr = 1, Le = 5, N = -1) in FP32 shifted storage, two-buffer pull layout.
The state (2.8 GB) is far larger than L2 (129 MB), so no flush is needed.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "3-lattice GLUPS & %HBM peak; served solves/s, p99 vs plain at Nu/Sh err≤1e-3"
STEPS_PER_BENCH_STEP = 100
# algorithmic bytes per node update: 19 distributions + 4 history values, read and written
BYTES_PER_NODE = {"f64": 2 * (19 * 8 + 4 * 8), "f32": 2 * (19 * 4 + 4 * 4),
                  "bf16": 2 * (19 * 2 + 4 * 4), "f16": 2 * (19 * 2 + 4 * 4)}
BYTES_PER_NODE_19 = {"f64": 2 * 19 * 8, "f32": 2 * 19 * 4, "bf16": 2 * 19 * 2, "f16": 2 * 19 * 2}
KERNEL_SOURCES = ["paper_1708_07525_gb300/csrc/lbm_kernels.cuh",
                  "paper_1708_07525_gb300/csrc/lbm_device.cuh",
                  "paper_1708_07525_gb300/csrc/lbm_launchers.cuh"]


def kernel_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def profiled_traffic(name: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel sources (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            d = json.load(f)
        e = d.get(name)
        if e and e.get("kernel_hash") == kernel_hash():
            return float(e["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x: float, device=None) -> float:
    """Largest value of x over all ranks (the timing rule: the job is as slow as its
    slowest rank); x itself on a single process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(units_per_rank: float, seconds: float, world: int) -> float:
    """Whole-job throughput: units processed by all ranks / the slowest rank's time."""
    return world * units_per_rank / seconds


def dist_setup(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def cpu_baseline(nx, ny, spec, budget_s=12.0):
    """The FP64 oracle as it stands, all host cores, on the same cavity for as many
    whole time steps as fit in about `budget_s` seconds (at least one)."""
    from oracle import oracle as O
    threads = os.cpu_count() or 1
    O.set_threads(threads)
    p = O.derive(*spec.args())
    o = O.Oracle(p, seed=spec.seed, noise=spec.noise)
    t0 = time.perf_counter()
    o.step(1)
    dt1 = time.perf_counter() - t0
    more = max(0, int(budget_s / max(dt1, 1e-9)) - 1)
    more = min(more, 50)
    t0 = time.perf_counter()
    if more:
        o.step(more)
    dt = time.perf_counter() - t0
    steps, secs = (more, dt) if more else (1, dt1)
    glups = nx * ny * steps / secs / 1e9
    return {"value": glups, "unit": "GLUPS", "cores": O.get_threads(), "kind": "oracle",
            "sample": f"{nx}x{ny} cavity, {steps} time step(s) of the FP64 oracle after 1 warm-up "
                      f"step, {secs:.1f} s"}


def run_reference(args):
    rank, world, _ = dist_setup(args.gpus)
    if rank != 0:
        return 0
    from paper_1708_07525_gb300.workloads import throughput_cavity
    from oracle import oracle as O
    n = args.size
    spec = throughput_cavity(n)
    threads = os.cpu_count() or 1
    O.set_threads(threads)
    o = O.Oracle(O.derive(*spec.args()), seed=spec.seed, noise=spec.noise)
    per_step = max(1, int(args.ref_steps))
    for _ in range(args.warmup):
        o.step(per_step)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(per_step)
    secs = time.perf_counter() - t0
    value = n * n * per_step * args.steps / secs / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": secs / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"porous cavity {n}x{n}, Ra=1e5 Da=1e-3 eps=0.4 Pr=1 Le=5 N=-1",
                   "nx": n, "ny": n, "bench_step": f"{per_step} time step(s) of the CPU oracle"},
        "cpu_baseline": {"value": value, "unit": "GLUPS", "cores": O.get_threads(), "kind": "oracle",
                         "sample": f"{n}x{n} cavity, {per_step} time step(s) per bench step"},
        "e2e": {"value": value, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def step_launches(args, k):
    """Kernels launched by k time steps of one cavity: one fused kernel per step, except
    where the step is split into an inner-node kernel and a ring kernel (wall nodes; the
    two-buffer layout with FP64 or 16-bit storage; the odd steps of the in-place layout)."""
    if args.layout == "aa":
        return k + k // 2
    if args.walls == "nee" or args.precision != "f32":
        return 2 * k
    return k


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_setup(args.gpus)
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    from paper_1708_07525_gb300 import lbm
    from paper_1708_07525_gb300.workloads import throughput_cavity

    n = args.size
    spec = throughput_cavity(n)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    if args.walls == "nee":
        # the paper's own walls (Sec. 3.3): nodes on the walls, L = n - 1
        p = lbm.lbm_derive_params_nee(n, n, spec.Ra, spec.Da, spec.eps, spec.Pr, spec.Le, spec.N,
                                      spec.J, spec.sigma, 0.0, spec.varpi)
        cav = lbm.Cavity(params=p, precision=args.precision, layout=args.layout,
                         seed=spec.seed + rank, noise=spec.noise, stream=stream.cuda_stream,
                         block=(args.bx, args.by))
    else:
        cav = lbm.Cavity(*spec.args(), precision=args.precision, layout=args.layout,
                         seed=spec.seed + rank, noise=spec.noise, stream=stream.cuda_stream,
                         block=(args.bx, args.by))
    k = STEPS_PER_BENCH_STEP

    def bench_step(ev_pair=None):
        if ev_pair is not None:
            ev_pair[0].record(stream)
        cav.step(k)
        if ev_pair is not None:
            ev_pair[1].record(stream)
        nush = cav.nusselt_sherwood()
        r = cav.residual()
        return nush, r

    for _ in range(args.warmup):
        bench_step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    with ClockSampler(dev) as clk:
        start.record(stream)
        for s in range(args.steps):
            nush, r = bench_step(evs[s])
        stop.record(stream)
        torch.cuda.synchronize()
    barrier()
    total_ms = start.elapsed_time(stop)
    kernel_ms = sum(a.elapsed_time(b) for a, b in evs) / (args.steps * k)
    total_ms = max_over_ranks(total_ms, device="cuda")
    nodes = n * n
    value = aggregate_value(nodes * k * args.steps, total_ms / 1e3, world) / 1e9

    # end to end through the public API with host buffers: each step re-initialises the
    # cavity from pinned host T/C fields (H2D), runs the 100 time steps, and reads the
    # Nu/Sh result back (D2H).
    Th = torch.empty((n, n), dtype=torch.float64).pin_memory()
    Ch = torch.empty((n, n), dtype=torch.float64).pin_memory()
    rng = np.random.default_rng(10 + rank)
    Th.numpy()[:] = 0.5 + spec.noise * rng.uniform(-1, 1, (n, n))
    Ch.numpy()[:] = 0.5 + spec.noise * rng.uniform(-1, 1, (n, n))

    def e2e_step():
        cav.reset(T_ptr=Th.data_ptr(), C_ptr=Ch.data_ptr())
        cav.step(k)
        return cav.nusselt_sherwood()

    e2e_step()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, device="cuda")
    e2e_value = aggregate_value(nodes * k * args.steps, e2e_s, world) / 1e9

    peak, peak_kind = measured_peaks()
    bpn = BYTES_PER_NODE[args.precision]
    achieved = nodes * bpn / (kernel_ms / 1e3) / 1e9
    kname = f"step_{args.layout}_{args.precision}_{n}" + ("_nee" if args.walls == "nee" else "")
    traffic = profiled_traffic(kname)
    line = {
        "metric": METRIC, "value": value, "unit": "GLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": {
            "workload": f"porous cavity {n}x{n}, Ra=1e5 Da=1e-3 eps=0.4 Pr=1 Le=5 N=-1, "
                        f"{args.precision} {'two-buffer pull' if args.layout == 'ab' else 'in-place AA'}"
                        + (", wall nodes (Sec. 3.3)" if args.walls == "nee" else ", halfway walls"),
            "nx": n, "ny": n, "time_steps_per_bench_step": k,
            "bench_step": f"{k} fused time steps + FP64 Nu/Sh reduction + residual",
            "l2": "state larger than L2 (no flush needed)" if nodes * bpn / 2 > 129e6
                  else "state fits in L2 (cache-resident figure)",
            "parallelism": f"replicas x{world}",
        },
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_source": f"{peak_kind} hbm_gbs",
                     "kernel": (f"step_ab_kernel<{args.precision}> (inner nodes) + nee_ring_kernel"
                                if args.walls == "nee"
                                else f"step_{args.layout}_kernel<{args.precision}>"),
                     "kernel_us_per_launch": kernel_ms * 1e3,
                     "algorithmic_bytes_per_node": bpn,
                     "frac_19_distribution_convention":
                         nodes * BYTES_PER_NODE_19[args.precision] / (kernel_ms / 1e3) / 1e9 / peak},
        "e2e": {"value": e2e_value, "unit": "GLUPS",
                "h2d_bytes_per_step": 2 * nodes * 8, "d2h_bytes_per_step": 4 * 8},
        "gpu_launches": args.steps * (step_launches(args, k) + 1 + 2),
        "clocks": clk.summary(),
        "nusselt_sherwood": [float(x) for x in nush],
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(n, n, spec, budget_s=args.cpu_budget)
    if rank == 0:
        print(json.dumps(line), flush=True)
    cav.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_batch(args):
    """Many uneven cavities (grids drawn from 32^2..256^2, parameters drawn from the
    mixed ranges) advanced together: one fused launch per L2-sized group per step,
    autotuned tiles, CUDA graphs; aggregate GLUPS against one launch per cavity."""
    import numpy as np
    import torch
    from paper_1708_07525_gb300 import lbm
    from paper_1708_07525_gb300.workloads import draw_batch
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    specs = draw_batch(args.count, seed=4)
    insts = [lbm.make_instance(s) for s in specs]
    nodes = sum(s.nx * s.ny for s in specs)
    b = lbm.Batch(insts, precision=args.precision, layout=args.layout, stream=stream.cuda_stream)
    t0 = time.perf_counter()
    report = b.autotune(trial_steps=16)
    tune_s = time.perf_counter() - t0
    b.step(64)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        e0.record(stream)
        b.step(args.batch_steps)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    glups = nodes * args.batch_steps / (ms / 1e3) / 1e9
    nush = b.nusselt_sherwood()
    b.close()
    # one launch per cavity per step, on one stream
    cavs = [lbm.Cavity(*s.args(), varpi=s.varpi, precision=args.precision, layout=args.layout,
                       seed=s.seed, noise=s.noise, stream=stream.cuda_stream, graph_chunk=-1)
            for s in specs]
    k = max(2, args.batch_steps // 50)
    for c in cavs:
        c.step(2)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(k):
        for c in cavs:
            c.step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    per_ms = e0.elapsed_time(e1)
    per_glups = nodes * k / (per_ms / 1e3) / 1e9
    del cavs
    line = {
        "metric": METRIC, "mode": "batch", "value": glups, "unit": "GLUPS", "n_gpus": 1,
        "steps": args.batch_steps, "higher_is_better": True, "dtype": args.precision,
        "data": "synthetic",
        "config": {"workload": f"{args.count} cavities, grids 32^2-256^2 drawn by seed 4, "
                               f"log-uniform Ra in [1e3,1e5], Da in [1e-4,1e-1], uniform eps, Le, N, "
                               f"sigma; {args.precision} {args.layout}",
                   "nodes": nodes, "time_steps": args.batch_steps},
        "one_launch_per_cavity_glups": per_glups,
        "speedup_vs_one_launch_per_cavity": glups / per_glups,
        "autotune_s": tune_s, "autotune": report.strip().splitlines(),
        "clocks": clk.summary(),
        "finite_nush": int(np.isfinite(nush).all(axis=1).sum()),
    }
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    """Continuous-batching solver service against plain one-at-a-time FP64 solves.
    Requests: grids from `--serve-sizes`, parameters from the mixed ranges, Poisson
    arrivals at 0.8 x the service capacity measured on a burst of the same requests."""
    import numpy as np
    import torch
    from paper_1708_07525_gb300 import lbm
    from paper_1708_07525_gb300.workloads import draw_batch, arrivals
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    sizes = tuple(int(x) for x in args.serve_sizes.split(","))
    specs = draw_batch(args.requests, seed=5, sizes=sizes)
    insts = [lbm.make_instance(s) for s in specs]
    cap_steps = args.max_steps
    check = args.check_every

    def serve(arrive):
        srv = lbm.Server(args.budget_gb * (1 << 30), max_slots=len(specs), check_every=check,
                         precision=args.precision, layout=args.layout, stream=stream.cuda_stream)
        t_start = time.perf_counter()
        pending = list(range(len(specs)))
        submitted_at = {}
        done = {}
        while len(done) < len(specs):
            now = time.perf_counter() - t_start
            while pending and arrive[pending[0]] <= now:
                k = pending.pop(0)
                srv.submit(insts[k], tol=args.serve_tol, nush_tol=args.nush_tol,
                           max_steps=cap_steps, rid=k)
                submitted_at[k] = now
            active = srv.tick()
            t_now = time.perf_counter() - t_start
            for r in srv.poll():
                done[r["id"]] = dict(r, arrival=arrive[r["id"]], finished=t_now)
            if active == 0 and pending and srv.info()["queued"] == 0:
                time.sleep(max(0.0, arrive[pending[0]] - (time.perf_counter() - t_start)))
        makespan = time.perf_counter() - t_start
        srv.close()
        return done, makespan

    burst, burst_s = serve(np.zeros(len(specs)))
    capacity = len(specs) / burst_s
    arr = arrivals(len(specs), 0.8 * capacity, seed=5)
    arr = arr - arr[0]
    served, served_s = serve(arr)
    lat = np.array([served[k]["finished"] - served[k]["arrival"] for k in served])

    # plain path: one FP64 cavity at a time, same check interval, residual < fp64_tol
    plain = {}
    plain_s = None
    if args.plain_cache and os.path.exists(args.plain_cache):
        with open(args.plain_cache) as f:
            cached = json.load(f)
        plain = {int(k): v for k, v in cached["plain"].items()}
        plain_s = cached["seconds"]
    t0 = time.perf_counter()
    for k, s in enumerate(specs if plain_s is None else []):
        if time.perf_counter() - t0 > args.plain_budget_s:
            break
        c = lbm.Cavity(*s.args(), varpi=s.varpi, precision="f64", seed=s.seed, noise=s.noise,
                       stream=stream.cuda_stream)
        status, steps = "unconverged", 0
        c.residual()
        while steps < cap_steps:
            c.step(check)
            steps += check
            if c.residual() < args.fp64_tol:
                status = "ok"
                break
        plain[k] = {"nush": c.nusselt_sherwood().tolist(), "steps": steps, "status": status}
        c.close()
    if plain_s is None:
        plain_s = time.perf_counter() - t0
        if args.plain_cache:
            with open(args.plain_cache, "w") as f:
                json.dump({"plain": plain, "seconds": plain_s}, f)
    errs = []
    for k, p in plain.items():
        if p["status"] == "ok" and served[k]["status"] == 0:
            a, b = np.array(served[k]["nush"]), np.array(p["nush"])
            errs.append(float(np.max(np.abs(a - b) / np.abs(b))))
    errs = np.array(errs) if errs else np.array([np.nan])
    statuses = [served[k]["status"] for k in served]
    line = {
        "metric": METRIC, "mode": "serve", "value": len(specs) / served_s, "unit": "solves/s",
        "higher_is_better": True, "dtype": args.precision, "data": "synthetic",
        "config": {"workload": f"{len(specs)} cavity solve requests, grids {sizes}, parameters "
                               f"from the mixed ranges (seed 5), Poisson arrivals at 0.8 x burst "
                               f"capacity; steady when residual < {args.serve_tol} or Nu/Sh change "
                               f"< {args.nush_tol} per {check} steps; cap {cap_steps} steps",
                   "precision": args.precision, "budget_gb": args.budget_gb},
        "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                      "max": float(lat.max())},
        "burst_capacity_solves_per_s": capacity,
        "served_status": {"ok": statuses.count(0), "unconverged": statuses.count(6),
                          "diverged": statuses.count(4)},
        "plain_fp64": {"solves": len(plain), "solves_per_s": len(plain) / plain_s,
                       "converged": sum(p["status"] == "ok" for p in plain.values()),
                       "tol": args.fp64_tol},
        "speedup_vs_plain_fp64": (len(specs) / served_s) / (len(plain) / plain_s),
        "nush_rel_err_vs_fp64": {"n": int(np.isfinite(errs).sum()),
                                 "max": float(np.nanmax(errs)), "median": float(np.nanmedian(errs)),
                                 "frac_le_1e-3": float(np.mean(errs <= 1e-3))},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_precision(args):
    """Storage-precision study on the 1024^2 cavity (Ra 1e5, Da 1e-2, eps 0.6, Le 10,
    N 2): FP64 (reference), FP32, and shifted FP16 / BF16 with stochastic rounding,
    all FP32 arithmetic but FP64; the same number of steps; errors of u, T, C
    (relative L2) and of Nu/Sh against FP64; FP64 reductions throughout."""
    import numpy as np
    import torch
    from paper_1708_07525_gb300 import lbm
    from paper_1708_07525_gb300.workloads import PRECISION_STUDY as spec
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    steps, check = args.prec_steps, args.prec_check
    out = {}
    ref = None
    for prec in args.prec_list.split(","):
        c = lbm.Cavity(*spec.args(), precision=prec, seed=spec.seed, noise=spec.noise,
                       stream=stream.cuda_stream)
        c.residual()
        hist = []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = 0.0
        while c.t < steps:
            e0.record(stream)
            c.step(min(check, steps - c.t))
            e1.record(stream)
            r = c.residual()
            ms += e0.elapsed_time(e1)
            hist.append([c.t, r] + c.nusselt_sherwood().tolist())
        fl = c.fields(("ux", "uy", "T", "C"))
        rec = {"glups": spec.nx * spec.ny * steps / (ms / 1e3) / 1e9, "final_residual": hist[-1][1],
               "nush": hist[-1][2:], "history": hist}
        if ref is None:
            ref = (fl, np.array(hist[-1][2:]))
        else:
            rec["rel_l2_err"] = {k: float(np.linalg.norm(fl[k] - ref[0][k]) / np.linalg.norm(ref[0][k]))
                                 for k in fl}
            rec["nush_rel_err"] = float(np.max(np.abs(np.array(hist[-1][2:]) - ref[1]) / np.abs(ref[1])))
        out[prec] = rec
        c.close()
        if args.partial_out:   # results so far, in case a long study is cut short
            with open(args.partial_out, "w") as f:
                json.dump(out, f)
    line = {"metric": METRIC, "mode": "precision", "unit": "relative error", "data": "synthetic",
            "config": {"workload": f"{spec.nx}x{spec.ny} cavity Ra={spec.Ra} Da={spec.Da} eps={spec.eps} "
                                   f"Le={spec.Le} N={spec.N}", "steps": steps, "check_every": check},
            "results": {k: {kk: vv for kk, vv in v.items() if kk != "history"} for k, v in out.items()}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=4096)
    ap.add_argument("--precision", default="f32", choices=["f64", "f32", "bf16", "f16"])
    ap.add_argument("--layout", default="ab", choices=["ab", "aa"])
    ap.add_argument("--walls", default="halfway", choices=["halfway", "nee"],
                    help="step mode: halfway walls (the workload's) or wall nodes (Sec. 3.3)")
    ap.add_argument("--bx", type=int, default=0)
    ap.add_argument("--by", type=int, default=0)
    ap.add_argument("--ref-steps", type=int, default=1)
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", default="step", choices=["step", "batch", "serve", "precision"])
    ap.add_argument("--prec-steps", type=int, default=2500000)
    ap.add_argument("--prec-check", type=int, default=100000)
    ap.add_argument("--prec-list", default="f64,f32,f16,bf16")
    ap.add_argument("--count", type=int, default=512)
    ap.add_argument("--batch-steps", type=int, default=5000)
    ap.add_argument("--requests", type=int, default=32)
    ap.add_argument("--serve-sizes", default="64,128")
    ap.add_argument("--serve-tol", type=float, default=1e-6)
    ap.add_argument("--nush-tol", type=float, default=0.0)
    ap.add_argument("--fp64-tol", type=float, default=1e-7)
    ap.add_argument("--check-every", type=int, default=500)
    ap.add_argument("--max-steps", type=int, default=300000)
    ap.add_argument("--budget-gb", type=float, default=8.0)
    ap.add_argument("--plain-budget-s", type=float, default=120.0)
    ap.add_argument("--plain-cache", default="")
    ap.add_argument("--partial-out", default="")
    args = ap.parse_args()
    if args.mode == "batch":
        return run_batch(args)
    if args.mode == "serve":
        return run_serve(args)
    if args.mode == "precision":
        return run_precision(args)
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
