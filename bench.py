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
        "config": {"workload": f"porous cavity {n}x{n}, Ra=1e5 Da=1e-3 eps=0.4 Pr=1 Le=5 N=-1, "
                               f"halfway walls",
                   "storage": "f64 (the oracle: FP64 throughout, push streaming)",
                   "nx": n, "ny": n, "bench_step": f"{per_step} time step(s) of the CPU oracle"},
        "cpu_baseline": {"value": value, "unit": "GLUPS", "cores": O.get_threads(), "kind": "oracle",
                         "sample": f"{n}x{n} cavity, {per_step} time step(s) per bench step"},
        "e2e": {"value": value, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def step_launches(args, k):
    """Kernels launched by k time steps of the benchmark cavity.  With FP32 arithmetic
    (FP32 and 16-bit storage) every step is one launch: the FP32 steps, the in-place odd
    step with its ring in the same launch, the step with wall nodes with its wall ring in
    the same launch, the 16-bit pair steps with their edge set.  FP64 splits the two-buffer
    step (also with wall nodes) and the in-place odd step into an inner-node launch and a
    ring launch on a second stream."""
    if args.precision != "f64":
        return k
    if args.layout == "aa":
        return k + k // 2
    return 2 * k


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
            "workload": f"porous cavity {n}x{n}, Ra=1e5 Da=1e-3 eps=0.4 Pr=1 Le=5 N=-1"
                        + (", wall nodes (Sec. 3.3)" if args.walls == "nee" else ", halfway walls"),
            "storage": f"{args.precision} "
                       f"{'two-buffer pull' if args.layout == 'ab' else 'in-place AA'}",
            "nx": n, "ny": n, "time_steps_per_bench_step": k,
            "bench_step": f"{k} fused time steps + FP64 Nu/Sh reduction + residual",
            "l2": "state larger than L2 (no flush needed)" if nodes * bpn / 2 > 129e6
                  else "state fits in L2 (cache-resident figure)",
            "parallelism": f"replicas x{world}",
        },
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_source": f"{peak_kind} hbm_gbs",
                     "kernel": ((f"step_ab_kernel<{args.precision}> (inner nodes) + nee_ring_kernel"
                                 if args.precision == "f64" else
                                 f"step_ab_nee_fused_kernel<{args.precision}> (wall ring and inner "
                                 f"nodes in one launch)")
                                if args.walls == "nee"
                                else (f"step_{args.layout}_pair kernels<{args.precision}> (two "
                                      f"nodes per thread; edge nodes one per thread in the "
                                      f"same launch)"
                                      if args.precision in ("bf16", "f16")
                                      else f"step_{args.layout}_kernel<{args.precision}>")),
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


def run_slab(args):
    """One cavity of n x (n * N) nodes cut into N slabs of n rows, one per rank (weak
    scaling: every rank advances n^2 nodes).  After every time step the ranks swap the
    five populations per column that cross each cut (lbm_halo_export / _import) with
    NCCL send / receive (--comm nccl, one GPU per rank) or through the host over gloo
    (--comm gloo).  One bench step = 100 time steps with their exchanges, then the FP64
    Nu / Sh (row means combined over ranks) and the residual (maxima combined)."""
    import numpy as np
    import torch
    import torch.distributed as dist
    rank, world, local = dist_setup(args.gpus)
    dev_index = local if args.comm == "nccl" else args.device
    torch.cuda.set_device(dev_index)
    if world > 1:
        if args.comm == "nccl":
            dist.init_process_group("nccl", device_id=torch.device("cuda", dev_index))
        else:
            dist.init_process_group("gloo")
    from paper_1708_07525_gb300 import lbm
    from paper_1708_07525_gb300.workloads import throughput_cavity
    n = args.size
    spec = throughput_cavity(n)
    p = lbm.lbm_derive_params(n, n * world, spec.Ra, spec.Da, spec.eps, spec.Pr, spec.Le, spec.N,
                              spec.J, spec.sigma, 0.0, spec.varpi)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    slab = lbm.Cavity(params=p, slab=(rank * n, n), precision=args.precision, seed=spec.seed,
                      noise=spec.noise, stream=stream.cuda_stream, block=(args.bx, args.by))
    nb = slab.halo_bytes()
    dev_faces = {k: torch.empty(nb, dtype=torch.uint8, device="cuda")
                 for k in ("down_out", "up_out", "below_in", "above_in")}
    host = args.comm != "nccl"
    host_faces = {k: torch.empty(nb, dtype=torch.uint8).pin_memory() for k in dev_faces} if host else {}
    lo, hi = rank > 0, rank < world - 1

    def exchange():
        if world == 1:
            return
        if lo:
            slab.halo_export(0, dev_faces["down_out"].data_ptr())
        if hi:
            slab.halo_export(1, dev_faces["up_out"].data_ptr())
        bufs = dev_faces
        if host:
            stream.synchronize()
            for k in ("down_out", "up_out"):
                host_faces[k].copy_(dev_faces[k])
            bufs = host_faces
        ops = []
        if lo:
            ops += [dist.P2POp(dist.isend, bufs["down_out"], rank - 1),
                    dist.P2POp(dist.irecv, bufs["below_in"], rank - 1)]
        if hi:
            ops += [dist.P2POp(dist.isend, bufs["up_out"], rank + 1),
                    dist.P2POp(dist.irecv, bufs["above_in"], rank + 1)]
        for r in dist.batch_isend_irecv(ops):
            r.wait()
        if host:
            for k in ("below_in", "above_in"):
                dev_faces[k].copy_(host_faces[k], non_blocking=True)
        if lo:
            slab.halo_import(0, dev_faces["below_in"].data_ptr())
        if hi:
            slab.halo_import(1, dev_faces["above_in"].data_ptr())

    k = STEPS_PER_BENCH_STEP

    def bench_step():
        for _ in range(k):
            slab.step(1)
            exchange()
        nush = torch.tensor(slab.nusselt_sherwood() * n, dtype=torch.float64)
        parts = torch.tensor(slab.residual_parts(), dtype=torch.float64)
        if world > 1:
            if not host:
                nush, parts = nush.cuda(), parts.cuda()
            dist.all_reduce(nush)
            dist.all_reduce(parts, op=dist.ReduceOp.MAX)
        nush = (nush / (n * world)).cpu().numpy()
        parts = parts.cpu().numpy()
        return nush, max(d / a if a > 0 else float("inf") for d, a in zip(parts[:4], parts[4:]))

    for _ in range(args.warmup):
        bench_step()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    barrier()
    with ClockSampler(dev_index) as clk:
        t0 = time.perf_counter()
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for _ in range(args.steps):
            nush, r = bench_step()
        stop.record(stream)
        torch.cuda.synchronize()
        wall_s = time.perf_counter() - t0
    barrier()
    total_ms = max_over_ranks(start.elapsed_time(stop), device="cuda" if not host else None)
    value = aggregate_value(n * n * k * args.steps, total_ms / 1e3, world) / 1e9
    line = {
        "metric": METRIC, "mode": "slab", "value": value, "unit": "GLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": args.precision, "data": "synthetic",
        "config": {"workload": f"porous cavity {n}x{n * world} (Ra=1e5 Da=1e-3 eps=0.4 Pr=1 Le=5 "
                               f"N=-1, L = nx = {n}) cut into {world} slabs of {n} rows, "
                               f"{args.precision} two-buffer pull, halo exchange every step "
                               f"over {args.comm}",
                   "parallelism": f"y-slabs x{world}", "wall_s": wall_s},
        "halo_bytes_per_step_per_cut": 2 * nb,
        "clocks": clk.summary(),
        "nusselt_sherwood": [float(x) for x in nush], "residual": r,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    slab.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def l2_copy_gbs(stream, mb):
    """Best-of-10 copy bandwidth (read + write bytes) of `mb` MB each way, copied back and
    forth `passes` times inside one launch (paper_1708_07525_gb300/csrc/probe/l2_copy.cu),
    so that launch gaps do not count."""
    import ctypes
    import torch
    from paper_1708_07525_gb300 import build as B
    probe = ctypes.CDLL(B.build_probe())
    probe.probe_l2_copy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    nbytes = mb * (1 << 20)
    a = torch.rand(nbytes // 4, device="cuda")
    b = torch.empty_like(a)
    blocks = torch.cuda.get_device_properties(0).multi_processor_count * 8
    passes = max(20, int(8e9 / (2 * nbytes)))
    args = (a.data_ptr(), b.data_ptr(), nbytes, passes, blocks, stream.cuda_stream)
    assert probe.probe_l2_copy(*args) == 0
    best = 0.0
    for _ in range(10):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        assert probe.probe_l2_copy(*args) == 0
        e1.record(stream)
        torch.cuda.synchronize()
        best = max(best, 2 * nbytes * passes / (e0.elapsed_time(e1) / 1e3) / 1e9)
    return best


def run_l2peak(args):
    """Copy bandwidth of a working set that stays in L2 (the bound of the batched step,
    whose L2 blocking keeps a group's state in L2 for most of its steps): torch copies
    b <- a of `--l2-mb` MB each way, repeated back to back, timed with CUDA events;
    read + write bytes over time, best of 10 rounds, for several sizes."""
    import torch
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    out = {str(mb): l2_copy_gbs(stream, mb) for mb in [int(x) for x in args.l2_mb.split(",")]}
    line = {"metric": "L2-resident copy bandwidth", "mode": "l2peak", "unit": "GB/s",
            "value": max(out.values()), "by_mb_each_way": out,
            "how": "copies back and forth between two buffers inside one launch (16-byte "
                   "loads and stores, 8 blocks of 256 threads per SM), read + write bytes, CUDA "
                   "events, best of 10 rounds",
            "l2_bytes": torch.cuda.get_device_properties(0).L2_cache_size}
    print(json.dumps(line), flush=True)
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
    # the roofline: L2 blocking keeps a group's state in L2 for all but the first of its
    # steps, so the bound is the L2-resident copy bandwidth (measured here, 16 MB each way)
    l2_peak = l2_copy_gbs(stream, 16)
    hbm_peak, peak_kind = measured_peaks()
    bpn = BYTES_PER_NODE[args.precision]
    achieved = glups * bpn
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
                               f"sigma, varpi = min(0.4, 0.8 min(eps, sigma)); "
                               f"{args.precision} {args.layout}",
                   "nodes": nodes, "time_steps": args.batch_steps},
        "roofline": {"bound": "l2", "achieved": achieved, "peak": l2_peak, "unit": "GB/s",
                     "frac": achieved / l2_peak, "traffic": None,
                     "peak_source": "L2-resident copy, 16 MB each way, measured in this run",
                     "kernel": f"batch_step_kernel<{args.precision}>",
                     "algorithmic_bytes_per_node": bpn,
                     "frac_of_hbm": achieved / hbm_peak, "hbm_peak": hbm_peak},
        "one_launch_per_cavity_glups": per_glups,
        "speedup_vs_one_launch_per_cavity": glups / per_glups,
        "autotune_s": tune_s, "autotune": report.strip().splitlines(),
        "clocks": clk.summary(),
        "finite_nush": int(np.isfinite(nush).all(axis=1).sum()),
    }
    print(json.dumps(line), flush=True)
    return 0


def solve_alone(lbm, spec, precision, layout, stream, tol, nush_tol, check, cap, round_nearest=False):
    """One cavity solve on its own (the single-cavity step kernels, CUDA graphs), stopped
    by the server's rule: at a check every `check` steps it is steady if the residual
    over those steps is below tol, or (from the second check on) if every Nu_L, Sh_L,
    Nu_R, Sh_R moved by less than nush_tol relative since the previous check; past `cap`
    steps it is unconverged; a non-finite value makes it diverged."""
    import numpy as np
    c = lbm.Cavity(*spec.args(), varpi=spec.varpi, precision=precision, layout=layout,
                   seed=spec.seed, noise=spec.noise, stream=stream, round_nearest=round_nearest)
    prev = np.zeros(4)
    steps, checks, status, r, ns = 0, 0, 6, float("inf"), prev
    while True:
        c.step(check)
        steps += check
        checks += 1
        try:
            r = c.residual()
            ns = c.nusselt_sherwood()
        except lbm.LbmError:
            status = 4
            break
        dn = float(np.max(np.abs(ns - prev) / np.maximum(np.abs(ns), 1e-300)))
        prev = ns
        if (tol > 0 and r < tol) or (nush_tol > 0 and checks > 1 and dn < nush_tol):
            status = 0
            break
        if steps >= cap:
            break
    c.close()
    return {"status": status, "steps": steps, "residual": r, "nush": list(map(float, ns))}


def fifo_latency(arrive, service):
    """Latencies of a one-at-a-time server (FIFO, one request on the device at a time)
    for the given arrival times and measured service times."""
    t, lat = 0.0, []
    for a, s in zip(arrive, service):
        t = max(t, a) + s
        lat.append(t - a)
    return lat


def run_serve(args):
    """Continuous-batching solver service against one-at-a-time solves of the same
    requests in the same storage precision and in plain FP64, all stopped by the same
    rule.  Requests: grids from `--serve-sizes`, parameters from the mixed ranges (seed 5),
    Poisson arrivals at 0.8 x the service capacity measured on a burst of the same
    requests (or `--arrival-rate`)."""
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
    check, tol, ntol = args.check_every, args.serve_tol, args.nush_tol
    # every time scale in steps grows like the grid width (the mapping of Sec. 4.1 fixes U):
    # the step cap is --max-steps at 64^2, scaled by L / 64
    caps = [max(check, int(args.max_steps * s.nx / 64)) for s in specs]

    def serve(arrive):
        srv = lbm.Server(args.budget_gb * (1 << 30), max_slots=len(specs), check_every=check,
                         precision=args.precision, layout=args.layout, stream=stream.cuda_stream,
                         round_nearest=args.round_nearest)
        t_start = time.perf_counter()
        pending = list(range(len(specs)))
        done = {}
        while len(done) < len(specs):
            now = time.perf_counter() - t_start
            while pending and arrive[pending[0]] <= now:
                k = pending.pop(0)
                srv.submit(insts[k], tol=tol, nush_tol=ntol, max_steps=caps[k], rid=k)
            active = srv.tick()
            t_now = time.perf_counter() - t_start
            for r in srv.poll():
                done[r["id"]] = dict(r, arrival=arrive[r["id"]], finished=t_now)
            if active == 0 and pending and srv.info()["queued"] == 0:
                time.sleep(max(0.0, arrive[pending[0]] - (time.perf_counter() - t_start)))
        makespan = time.perf_counter() - t_start
        srv.close()
        return done, makespan

    if args.arrival_rate > 0:
        capacity = None
        rate = args.arrival_rate
    else:
        _, burst_s = serve(np.zeros(len(specs)))
        capacity = len(specs) / burst_s
        rate = 0.8 * capacity
    arr = arrivals(len(specs), rate, seed=5)
    arr = arr - arr[0]
    served, served_s = serve(arr)
    lat = np.array([served[k]["finished"] - served[k]["arrival"] for k in served])

    fp64_service = [None]

    def alone(precision, budget_s, order):
        """One request at a time in `order`, until the time budget is spent."""
        res, service = {}, []
        if precision == "f64":
            fp64_service[0] = service
        t0 = time.perf_counter()
        for k in order:
            if time.perf_counter() - t0 > budget_s:
                break
            t1 = time.perf_counter()
            res[k] = solve_alone(lbm, specs[k], precision, "ab", stream.cuda_stream, tol, ntol,
                                 check, caps[k], args.round_nearest and precision != "f64")
            torch.cuda.synchronize()
            service.append(time.perf_counter() - t1)
            res[k]["seconds"] = service[-1]
        secs = time.perf_counter() - t0
        done = [k for k in order if k in res]
        l = (np.array(fifo_latency(arr[done], service)) if done == list(range(len(done)))
             else np.array([np.nan]))
        return res, secs, l

    same, same_s, same_lat = alone(args.precision, args.alone_budget_s, range(len(specs)))
    if args.fp64_cache and os.path.exists(args.fp64_cache):   # the FP64 arm of an earlier run
        with open(args.fp64_cache) as f:
            cached = json.load(f)
        fp64 = {int(k): v for k, v in cached["results"].items()}
        fp64_s = cached["seconds"]
        fp64_lat = np.array([np.nan])
    else:
        # smallest grids first, so that the budget covers as many requests as it can
        order = sorted(range(len(specs)), key=lambda k: (specs[k].nx, k))
        fp64, fp64_s, fp64_lat = alone("f64", args.plain_budget_s, order)
        if args.fp64_cache:
            with open(args.fp64_cache, "w") as f:
                json.dump({"results": fp64, "seconds": fp64_s, "service": fp64_service[0]}, f)

    def errs_vs(ref, other):
        e = []
        for k, p in ref.items():
            if k in other and p["status"] == 0 and other[k]["status"] == 0:
                a, b = np.array(other[k]["nush"]), np.array(p["nush"])
                e.append(float(np.max(np.abs(a - b) / np.abs(b))))
        return np.array(e) if e else np.array([np.nan])

    def status_counts(res):
        st = [r["status"] for r in res.values()]
        return {"ok": st.count(0), "unconverged": st.count(6), "diverged": st.count(4)}

    def pct(a, q):
        return float(np.nanpercentile(a, q)) if np.isfinite(a).any() else None

    e_served = errs_vs(fp64, served)
    e_same = errs_vs(fp64, same)
    nodes = {k: s.nx * s.ny for k, s in enumerate(specs)}
    # FP64 one at a time over the whole prefix, estimated from its measured rate per grid
    # size (lattice updates per second of the requests it finished; a size it did not reach
    # takes the rate of the largest size it did)
    rate64 = {}
    for k, r in fp64.items():
        n = specs[k].nx
        u, t = rate64.get(n, (0.0, 0.0))
        rate64[n] = (u + nodes[k] * r["steps"], t + r["seconds"])
    est64 = None
    if rate64:
        largest = max(rate64)
        est64 = 0.0
        for k in served:
            n = specs[k].nx if specs[k].nx in rate64 else largest
            u, t = rate64[n]
            est64 += nodes[k] * served[k]["steps"] / (u / t)
    line = {
        "metric": METRIC, "mode": "serve", "value": len(specs) / served_s, "unit": "solves/s",
        "higher_is_better": True, "dtype": args.precision, "data": "synthetic",
        "config": {"workload": f"first {len(specs)} of the seeded cavity solve requests (seed 5), "
                               f"grids {sizes}, parameters from the mixed ranges with varpi = "
                               f"min(0.4, 0.8 min(eps, sigma)), Poisson arrivals at "
                               f"{rate:.3g}/s; every arm stops a request at the first check "
                               f"(every {check} steps) where the residual < {tol} or every "
                               f"Nu/Sh moved < {ntol} relative, else at {args.max_steps} x L / 64 "
                               f"steps",
                   "precision": args.precision, "layout": args.layout,
                   "rounding": ("to nearest" if args.round_nearest else "stochastic")
                               if args.precision in ("bf16", "f16") else "n/a",
                   "budget_gb": args.budget_gb,
                   "grids": {str(n): sum(1 for s in specs if s.nx == n) for n in sizes},
                   "lattice_updates": int(sum(nodes[k] * served[k]["steps"] for k in served))},
        "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                      "max": float(lat.max())},
        "burst_capacity_solves_per_s": capacity,
        "served_status": status_counts(served),
        "one_at_a_time": {
            "precision": args.precision, "solves": len(same), "seconds": same_s,
            "solves_per_s": len(same) / same_s, "status": status_counts(same),
            "latency_s": {"p50": pct(same_lat, 50), "p99": pct(same_lat, 99)},
            "nush_rel_err_vs_fp64": {"n": int(np.isfinite(e_same).sum()),
                                     "max": float(np.nanmax(e_same)) if np.isfinite(e_same).any() else None}},
        "plain_fp64": {
            "solves": len(fp64), "seconds": fp64_s, "status": status_counts(fp64),
            "order": "smallest grids first, within --plain-budget-s",
            "grids": {str(n): sum(1 for k in fp64 if specs[k].nx == n) for n in sizes},
            "glups_by_grid": {str(n): u / t / 1e9 for n, (u, t) in sorted(rate64.items())},
            "estimated_seconds_for_all_requests": est64,
            "estimated_solves_per_s": len(specs) / est64 if est64 else None},
        "speedup_vs_one_at_a_time": (len(specs) / served_s) / (len(same) / same_s)
                                    if len(same) == len(specs) else None,
        "speedup_vs_plain_fp64_estimated": est64 / served_s if est64 else None,
        "nush_rel_err_vs_fp64": {"n": int(np.isfinite(e_served).sum()),
                                 "max": float(np.nanmax(e_served)) if np.isfinite(e_served).any() else None,
                                 "median": float(np.nanmedian(e_served)) if np.isfinite(e_served).any() else None,
                                 "frac_le_1e-3": float(np.mean(e_served <= 1e-3))},
        "steps": {str(k): served[k]["steps"] for k in sorted(served)},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_serve_cost(args):
    """Total lattice updates of the seeded request stream (`--requests-total` requests,
    seed 5, grids from `--serve-sizes`) under the serving stop rule.  Every request's
    parameters are solved at 64^2 in the server (storage `--precision`); the steps to
    the stop rule scale with the grid width (the mapping of Sec. 4.1 fixes U and makes
    nu, alpha_e, D_e grow with L, so every time scale in steps grows like L), so a
    request on an L^2 grid is estimated at steps_64 * L / 64 steps of L^2 nodes."""
    import numpy as np
    import torch
    from dataclasses import replace
    from paper_1708_07525_gb300 import lbm
    from paper_1708_07525_gb300.workloads import draw_batch
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    sizes = tuple(int(x) for x in args.serve_sizes.split(","))
    specs = draw_batch(args.requests_total, seed=5, sizes=sizes)
    small = [lbm.make_instance(replace(s, nx=64, ny=64)) for s in specs]
    cap64 = args.max_steps
    srv = lbm.Server(args.budget_gb * (1 << 30), max_slots=len(specs),
                     check_every=args.check_every, precision=args.precision,
                     stream=stream.cuda_stream)
    t0 = time.perf_counter()
    for k, inst in enumerate(small):
        srv.submit(inst, tol=args.serve_tol, nush_tol=args.nush_tol, max_steps=cap64, rid=k)
    res = {r["id"]: r for r in srv.drain()}
    secs = time.perf_counter() - t0
    srv.close()
    steps64 = np.array([res[k]["steps"] for k in range(len(specs))], dtype=float)
    status = np.array([res[k]["status"] for k in range(len(specs))])
    L = np.array([s.nx for s in specs], dtype=float)
    steps = steps64 * L / 64.0
    updates = steps * L * L
    cum = np.cumsum(updates)
    prefixes = {str(n): float(cum[n - 1]) for n in (8, 16, 24, 32, 64, 128, 256, 512, 1000,
                                                    2000) if n <= len(specs)}
    line = {
        "metric": METRIC, "mode": "serve_cost", "value": float(updates.sum()), "unit": "lattice updates",
        "data": "synthetic", "dtype": args.precision,
        "config": {"workload": f"{len(specs)} seeded cavity solve requests (seed 5), grids {sizes}; "
                               f"stop rule: residual < {args.serve_tol} or Nu/Sh change < "
                               f"{args.nush_tol} per {args.check_every} steps; each request "
                               f"solved at 64^2 (cap {cap64} steps), steps scaled by L / 64"},
        "calibration_seconds": secs,
        "calibration_status_64": {"ok": int((status == 0).sum()), "unconverged": int((status == 6).sum()),
                                  "diverged": int((status == 4).sum())},
        "steps_64": {"p50": float(np.median(steps64)), "p90": float(np.percentile(steps64, 90)),
                     "max": float(steps64.max())},
        "updates_by_grid": {str(int(n)): float(updates[L == n].sum()) for n in sizes},
        "count_by_grid": {str(int(n)): int((L == n).sum()) for n in sizes},
        "cumulative_updates_of_prefix": prefixes,
        "hours_at_40_glups": float(updates.sum() / 40e9 / 3600),
    }
    print(json.dumps(line), flush=True)
    return 0


def run_precision(args):
    """Storage-precision study on the 1024^2 cavity (Ra 1e5, Da 1e-2, eps 0.6, Le 10, N 2)
    against a steady FP64 state.  FP32 storage runs `--prec-steps` steps to its rounding
    floor; its state is loaded into an FP64 context (exact widening of every stored
    deviation) and run on in FP64 until the relative change of u, T, C over
    `--prec-check` steps is below `--steady-tol` (the reference, steady in FP64).  FP16 and
    BF16 storage (FP32 arithmetic, stochastic rounding) run `--prec-steps` steps from t = 0.
    Every result is compared with the reference: relative L2 error of u, T, C and the
    largest relative error of Nu_L, Sh_L, Nu_R, Sh_R (Eq. 38); reductions in FP64."""
    import numpy as np
    import torch
    from paper_1708_07525_gb300 import lbm
    from paper_1708_07525_gb300.workloads import PRECISION_STUDY as spec
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    steps, check = args.prec_steps, args.prec_check

    def r100(c):
        """The steady-state test of the paper's steady runs as read here: the relative
        change of u, T, C over the next 100 steps."""
        c.residual()
        c.step(100)
        return c.residual()

    def run(c, until, stop_tol=0.0):
        """Steps to `until` in chunks of `check` (the residual over each chunk recorded);
        with stop_tol, stops at the first chunk end where the change over 100 steps is
        below it.  Each history row: t, r over the chunk, r over 100 steps, Nu/Sh."""
        c.residual()
        hist, ms = [], 0.0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t_begin = c.t
        while c.t < until:
            e0.record(stream)
            c.step(min(check, until - c.t))
            e1.record(stream)
            r = c.residual()
            ms += e0.elapsed_time(e1)
            rk = r100(c) if (stop_tol > 0 or c.t >= until) else float("nan")
            hist.append([c.t, r, rk] + c.nusselt_sherwood().tolist())
            c.residual()
            if stop_tol > 0 and rk < stop_tol:
                break
        glups = spec.nx * spec.ny * (c.t - t_begin) / (ms / 1e3) / 1e9
        return hist, glups

    def make(prec):
        return lbm.Cavity(*spec.args(), precision=prec, seed=spec.seed, noise=spec.noise,
                          stream=stream.cuda_stream)

    out = {}
    c32 = make("f32")
    hist32, g32 = run(c32, steps)
    f32 = c32.fields(("ux", "uy", "T", "C"))
    blob = c32.save()
    c32.close()
    c64 = make("f64")
    c64.load(blob)
    hist64, g64 = run(c64, steps + args.polish_cap, stop_tol=args.steady_tol)
    ref = (c64.fields(("ux", "uy", "T", "C")), np.array(hist64[-1][3:]))
    c64.close()
    out["f64"] = {"glups": g64, "start": f"the FP32 state at {steps} steps", "steps": hist64[-1][0],
                  "residual_per_check": hist64[-1][1], "residual_100": hist64[-1][2],
                  "steady": hist64[-1][2] < args.steady_tol, "nush": hist64[-1][3:]}

    def compare(fl, nush):
        return ({k: float(np.linalg.norm(fl[k] - ref[0][k]) / np.linalg.norm(ref[0][k])) for k in fl},
                float(np.max(np.abs(np.array(nush) - ref[1]) / np.abs(ref[1]))))

    e, en = compare(f32, hist32[-1][3:])
    out["f32"] = {"glups": g32, "steps": steps, "residual_per_check": hist32[-1][1],
                  "residual_100": hist32[-1][2], "nush": hist32[-1][3:], "rel_l2_err": e,
                  "nush_rel_err": en}
    for prec in [p for p in args.prec_list.split(",") if p in ("bf16", "f16")]:
        c = make(prec)
        hist, g = run(c, steps)
        fl = c.fields(("ux", "uy", "T", "C"))
        c.close()
        e, en = compare(fl, hist[-1][3:])
        out[prec] = {"glups": g, "steps": steps, "residual_per_check": hist[-1][1],
                     "residual_100": hist[-1][2], "nush": hist[-1][3:], "rel_l2_err": e,
                     "nush_rel_err": en}
        if args.partial_out:   # results so far, in case a long study is cut short
            with open(args.partial_out, "w") as f:
                json.dump(out, f)
    line = {"metric": METRIC, "mode": "precision", "unit": "relative error", "data": "synthetic",
            "config": {"workload": f"{spec.nx}x{spec.ny} cavity Ra={spec.Ra} Da={spec.Da} eps={spec.eps} "
                                   f"Le={spec.Le} N={spec.N}", "steps": steps, "check_every": check,
                       "reference": f"FP64 from the FP32 state at {steps} steps until the relative "
                                    f"change over 100 steps < {args.steady_tol} (checked every "
                                    f"{check} steps)"},
            "results": out}
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
    ap.add_argument("--split", default="replicas", choices=["replicas", "slab"],
                    help="N > 1: independent cavities per rank, or one cavity cut into y-slabs")
    ap.add_argument("--comm", default="nccl", choices=["nccl", "gloo"],
                    help="slab exchange: NCCL send/recv, or host-staged over gloo")
    ap.add_argument("--device", type=int, default=0, help="--comm gloo: the GPU every rank uses")
    ap.add_argument("--mode", default="step",
                    choices=["step", "batch", "serve", "serve_cost", "precision", "l2peak"])
    ap.add_argument("--l2-mb", default="4,8,16,24,32,48")
    ap.add_argument("--prec-steps", type=int, default=4000000)
    ap.add_argument("--prec-check", type=int, default=100000)
    ap.add_argument("--prec-list", default="f32,f16,bf16")
    ap.add_argument("--steady-tol", type=float, default=1e-8)
    ap.add_argument("--polish-cap", type=int, default=3000000)
    ap.add_argument("--count", type=int, default=512)
    ap.add_argument("--batch-steps", type=int, default=5000)
    ap.add_argument("--requests", type=int, default=32)
    ap.add_argument("--requests-total", type=int, default=2000)
    ap.add_argument("--arrival-rate", type=float, default=0.0)
    ap.add_argument("--serve-sizes", default="64,128,256,512,1024")
    ap.add_argument("--serve-tol", type=float, default=1e-7)
    ap.add_argument("--nush-tol", type=float, default=1e-7)
    ap.add_argument("--check-every", type=int, default=500)
    ap.add_argument("--max-steps", type=int, default=300000)
    ap.add_argument("--budget-gb", type=float, default=8.0)
    ap.add_argument("--round-nearest", action="store_true",
                    help="serve: 16-bit storage rounded to nearest instead of stochastically")
    ap.add_argument("--plain-budget-s", type=float, default=300.0)
    ap.add_argument("--alone-budget-s", type=float, default=3600.0)
    ap.add_argument("--partial-out", default="")
    ap.add_argument("--fp64-cache", default="",
                    help="serve: file holding the FP64 one-at-a-time arm (written if absent)")
    args = ap.parse_args()
    if args.mode == "batch":
        return run_batch(args)
    if args.mode == "serve":
        return run_serve(args)
    if args.mode == "serve_cost":
        return run_serve_cost(args)
    if args.mode == "l2peak":
        return run_l2peak(args)
    if args.mode == "precision":
        return run_precision(args)
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.split == "slab":
        return run_slab(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
