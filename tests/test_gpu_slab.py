"""A cavity split along y into slabs (lbm_create_slab) reproduces the undivided cavity.

Streaming (Eq. 11) is the only step that couples nodes: after every time step each slab
hands the five populations per column that cross each of its cuts (f2, f5, f6, g2, h2
upward, f4, f7, f8, g4, h4 downward) to its neighbour's ghost row.  With that exchange the
per-node arithmetic of every slab row is the undivided cavity's, so the fields agree bit
for bit; Nu / Sh (Eq. 38) are row means, combined as the h-weighted mean over slabs; the
steady-state residual combines the slabs' maxima (lbm_residual_parts).

The exchange goes through device buffers with cudaMemcpy-ordered launches on one GPU, and,
in the two-process test, through the host over gloo between two processes that each own
one slab (their kernels never wait on one another: every exchange happens on the host
between steps)."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1708_07525_gb300 import lbm
from paper_1708_07525_gb300.workloads import CavitySpec

pytestmark = pytest.mark.gpu
KEYS = ("ux", "uy", "T", "C")
SPEC = CavitySpec(40, 37, Ra=1e5, Da=1e-2, eps=0.6, Le=2.0, N=-1.5, sigma=1.3, seed=8, noise=0.02)


def exchange(slabs, faces):
    """Export every cut face of every slab, then import each into its neighbour."""
    import torch
    for k, s in enumerate(slabs):
        if k > 0:
            s.halo_export(0, faces[k][0].data_ptr())
        if k + 1 < len(slabs):
            s.halo_export(1, faces[k][1].data_ptr())
    torch.cuda.synchronize()        # every slab runs on a stream of its own
    for k, s in enumerate(slabs):
        if k > 0:
            s.halo_import(0, faces[k - 1][1].data_ptr())     # what the slab below sent up
        if k + 1 < len(slabs):
            s.halo_import(1, faces[k + 1][0].data_ptr())     # what the slab above sent down
    torch.cuda.synchronize()


def make_split(precision, cuts):
    import torch
    p = lbm.lbm_derive_params(*SPEC.args())
    bounds = [0] + list(cuts) + [p.ny]
    slabs = [lbm.Cavity(params=p, slab=(a, b - a), precision=precision, seed=SPEC.seed,
                        noise=SPEC.noise) for a, b in zip(bounds[:-1], bounds[1:])]
    nb = slabs[0].halo_bytes()
    faces = [[torch.empty(nb, dtype=torch.uint8, device="cuda") for _ in range(2)] for _ in slabs]
    return slabs, faces, bounds


def advance(slabs, faces, steps):
    for _ in range(steps):
        for s in slabs:
            s.step(1)
        exchange(slabs, faces)


def whole_cavity(precision):
    """The undivided cavity.  16-bit storage runs two nodes per thread on a whole cavity but
    one node per thread on slabs; a single slab of all rows runs the one-node kernels."""
    if precision in ("bf16", "f16"):
        return lbm.Cavity(params=lbm.lbm_derive_params(*SPEC.args()), slab=(0, SPEC.ny),
                          precision=precision, seed=SPEC.seed, noise=SPEC.noise)
    return lbm.Cavity(*SPEC.args(), precision=precision, seed=SPEC.seed, noise=SPEC.noise)


@pytest.mark.parametrize("precision", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("cuts", [(18,), (1, 20, 36)], ids=["two", "four-with-1-row-slabs"])
def test_slabs_reproduce_the_whole_cavity(precision, cuts):
    steps = 300
    whole = whole_cavity(precision)
    whole.step(steps)
    fw = whole.fields()
    slabs, faces, bounds = make_split(precision, cuts)
    advance(slabs, faces, steps)
    for s, a, b in zip(slabs, bounds[:-1], bounds[1:]):
        assert s.t == steps
        fs = s.fields()
        for k in KEYS:
            assert np.array_equal(fs[k], fw[k][a:b]), (precision, a, b, k)
    # Nu / Sh: the row means combine as an h-weighted mean
    nush = sum((b - a) * s.nusselt_sherwood() for s, a, b in zip(slabs, bounds[:-1], bounds[1:]))
    np.testing.assert_allclose(nush / SPEC.ny, whole.nusselt_sherwood(), rtol=1e-12, atol=0)
    # the residual of the whole cavity from the slabs' maxima, over the next 50 steps
    whole.residual()
    parts = [s.residual_parts() for s in slabs]
    assert all(np.all(np.isinf(q[:4])) for q in parts)
    whole.step(50)
    r_whole = whole.residual()
    advance(slabs, faces, 50)
    parts = np.array([s.residual_parts() for s in slabs])
    dmax, amax = parts[:, :4].max(axis=0), parts[:, 4:].max(axis=0)
    r_split = max(d / a if a > 0 else (np.inf if d > 0 else 0.0) for d, a in zip(dmax, amax))
    assert r_split == r_whole, (r_split, r_whole)


def test_slab_walls_and_misuse():
    p = lbm.lbm_derive_params(*SPEC.args())
    import torch
    top = lbm.Cavity(params=p, slab=(20, 17), precision="f32")
    face = torch.empty(top.halo_bytes(), dtype=torch.uint8, device="cuda")
    with pytest.raises(lbm.LbmError) as ei:          # the top of this slab is the lid wall
        top.halo_export(1, face.data_ptr())
    assert ei.value.status == lbm.ERR_INVALID
    with pytest.raises(lbm.LbmError) as ei:
        top.nusselt_sherwood_tb()
    assert ei.value.status == lbm.ERR_INVALID
    top.halo_export(0, face.data_ptr())
    assert top.fields()["T"].shape == (17, SPEC.nx)


WORKER = r"""
import os, sys, numpy as np, torch, torch.distributed as dist
sys.path.insert(0, sys.argv[1])
from paper_1708_07525_gb300 import lbm
from paper_1708_07525_gb300.workloads import CavitySpec
spec = CavitySpec(40, 37, Ra=1e5, Da=1e-2, eps=0.6, Le=2.0, N=-1.5, sigma=1.3, seed=8, noise=0.02)
dist.init_process_group("gloo")
rank = dist.get_rank()
p = lbm.lbm_derive_params(*spec.args())
cut = 18
y0, h = (0, cut) if rank == 0 else (cut, spec.ny - cut)
s = lbm.Cavity(params=p, slab=(y0, h), precision="f64", seed=spec.seed, noise=spec.noise)
nb = s.halo_bytes()
face = torch.empty(nb, dtype=torch.uint8, device="cuda")
host_out = torch.empty(nb, dtype=torch.uint8)
host_in = torch.empty(nb, dtype=torch.uint8)
side = 1 if rank == 0 else 0
for _ in range(200):
    s.step(1)
    s.halo_export(side, face.data_ptr())
    torch.cuda.synchronize()
    host_out.copy_(face)
    # the two ranks swap faces over gloo (send / recv ordered by rank)
    if rank == 0:
        dist.send(host_out, 1); dist.recv(host_in, 1)
    else:
        dist.recv(host_in, 0); dist.send(host_out, 0)
    face.copy_(host_in)
    torch.cuda.synchronize()
    s.halo_import(side, face.data_ptr())
f = s.fields()
np.save(sys.argv[2] + f"_{rank}.npy", np.stack([f[k] for k in ("ux", "uy", "T", "C")]))
dist.barrier()
dist.destroy_process_group()
"""


def test_two_processes_exchange_over_gloo(tmp_path):
    """Two processes, one slab each (on the same GPU), swap their faces through the host
    with torch.distributed (gloo) after every step; together they give the undivided
    cavity's fields bit for bit."""
    script = tmp_path / "worker.py"
    script.write_text(WORKER)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = str(tmp_path / "slab")
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT="29631", WORLD_SIZE="2")
    procs = [subprocess.Popen([sys.executable, str(script), root, out],
                              env=dict(env, RANK=str(r), LOCAL_RANK=str(r)))
             for r in range(2)]
    rcs = [p.wait(timeout=600) for p in procs]
    assert rcs == [0, 0]
    whole = lbm.Cavity(*SPEC.args(), precision="f64", seed=SPEC.seed, noise=SPEC.noise)
    whole.step(200)
    fw = whole.fields()
    ref = np.stack([fw[k] for k in KEYS])
    a, b = np.load(out + "_0.npy"), np.load(out + "_1.npy")
    assert np.array_equal(np.concatenate([a, b], axis=1), ref)
