"""Multi-rank paths on CPU ranks (gloo, world size 2).

* bench.py's N-GPU timing rule: every rank runs its own cavity (replicas, no
  data-path collective); the job time is the slowest rank's and the value is
  the units of all ranks over that time.
* The y-slab split of one cavity with a one-row halo exchange per step: two
  ranks each advance half of the rows with the oracle (their slab plus one
  ghost row received from the neighbour every step) and must reproduce the
  single-rank oracle bit for bit.  This is the exchange a multi-GPU version of
  the fused step would need (boundary rows of pre-collision state).
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _init(rank, world, port):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    return dist


def _timing_worker(rank, world, port, q):
    dist = _init(rank, world, port)
    import bench
    t = [0.75, 1.25][rank]
    worst = bench.max_over_ranks(t)
    q.put((rank, worst, bench.aggregate_value(1000.0, worst, world)))
    dist.destroy_process_group()


def test_bench_timing_takes_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_timing_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for rank, worst, value in out:
        assert worst == 1.25
        assert value == pytest.approx(2 * 1000.0 / 1.25)


NX, NY, STEPS = 12, 10, 60
ARGS = (NX, NY, 1e5, 1e-2, 0.6, 1.0, 2.0, -1.0)


def _slab_worker(rank, world, port, q):
    """Rank 0 owns rows [0, NY/2), rank 1 rows [NY/2, NY); each keeps one ghost row."""
    dist = _init(rank, world, port)
    import torch
    from oracle import oracle as O
    O.set_threads(1)
    half = NY // 2
    full = O.Oracle(O.derive(*ARGS), seed=5, noise=0.05)      # initial state source only
    f, g, h, hist = full.get()
    # extended slab: rank 0 rows [0, half], rank 1 rows [half-1, NY)
    lo, hi = (0, half + 1) if rank == 0 else (half - 1, NY)
    p = O.derive(*ARGS)
    p.ny = hi - lo
    slab = O.Oracle(p, seed=5, noise=0.05)
    slab.set(f[:, lo:hi], g[:, lo:hi], h[:, lo:hi], hist[:, lo:hi])
    own = slice(0, half) if rank == 0 else slice(1, hi - lo)     # owned rows in the slab
    send_row = half - 1 - lo if rank == 0 else 1                  # my boundary row
    ghost_row = half - lo if rank == 0 else 0                     # neighbour's boundary row
    peer = 1 - rank
    for _ in range(STEPS):
        slab.step(1)
        fs, gs, hs, hs4 = slab.get()
        state = np.concatenate([fs[:, send_row], gs[:, send_row], hs[:, send_row], hs4[:, send_row]])
        out = torch.from_numpy(np.ascontiguousarray(state))
        inc = torch.empty_like(out)
        if rank == 0:
            dist.send(out, peer)
            dist.recv(inc, peer)
        else:
            dist.recv(inc, peer)
            dist.send(out, peer)
        inc = inc.numpy()
        fs[:, ghost_row], gs[:, ghost_row] = inc[:9], inc[9:14]
        hs[:, ghost_row], hs4[:, ghost_row] = inc[14:19], inc[19:23]
        slab.set(fs, gs, hs, hs4)
    fl = slab.fields()
    q.put((rank, {k: v[own].copy() for k, v in fl.items()}))
    dist.destroy_process_group()


def test_two_rank_slab_split_equals_single_rank_oracle():
    from oracle import oracle as O
    O.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_slab_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    parts = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    ref = O.Oracle(O.derive(*ARGS), seed=5, noise=0.05)
    ref.step(STEPS)
    fr = ref.fields()
    assert np.abs(fr["ux"]).max() > 1e-6
    for k in ("ux", "uy", "T", "C", "rho"):
        got = np.concatenate([parts[0][k], parts[1][k]], axis=0)
        assert np.array_equal(got, fr[k]), k


def test_fifo_latency_of_one_at_a_time_service():
    """The one-at-a-time arm's latencies: FIFO service of one request at a time, each
    starting when it has arrived and the previous one is done."""
    import bench
    arrive = [0.0, 1.0, 1.5, 10.0]
    service = [2.0, 1.0, 3.0, 0.5]
    # finishes: 2.0, 3.0, 6.0, 10.5
    assert bench.fifo_latency(arrive, service) == [2.0, 2.0, 4.5, 0.5]
