"""Programmatic dependent launches keep plain stream order.

The steps that are one kernel (the FP32 two-buffer step, the in-place even step, the FP32
in-place odd step with or without its ring of outermost nodes split into block rows of
their own, the 16-bit steps with two nodes per thread and their edge nodes in the same
launch, the batch's one-node tile step) go out as
programmatic dependent launches on the context's own stream: the next step's CTAs may be
placed while the step before still runs, and each waits (griddepcontrol.wait) for that
step to complete before it touches the state.  On the legacy default stream the library
makes ordinary launches and steps without graphs.  A step that read its neighbours before
the step before had written them, or wrote before a reader had finished, would change the
trajectory; every pair of runs below must agree bit for bit, with residual and Nu / Sh
read-outs (ordinary launches) between the chunks of steps."""
import numpy as np
import pytest

from paper_1708_07525_gb300 import lbm
from paper_1708_07525_gb300.workloads import CavitySpec, draw_batch

pytestmark = pytest.mark.gpu
KEYS = ("ux", "uy", "T", "C")
LEGACY = 1          # cudaStreamLegacy: ordinary launches, no graphs


def run(spec, layout, chunks, precision="f32", **kw):
    c = lbm.Cavity(*spec.args(), precision=precision, layout=layout, seed=spec.seed, noise=spec.noise,
                   **kw)
    reads = []
    c.residual()
    for n in chunks:
        c.step(n)
        reads.append((c.residual(), tuple(c.nusselt_sherwood())))
    return c.fields(), reads


@pytest.mark.parametrize("layout", ["ab", "aa"])
@pytest.mark.parametrize("n", [96, 768], ids=["one-kernel-steps", "split-odd-step"])
def test_cavity_programmatic_launches_equal_ordinary(layout, n):
    # 96 x 51: every step one kernel with the wall logic for every node; 768^2 (above 2^17
    # nodes): the in-place odd step runs the ring's block rows and the inner nodes in one
    # launch
    spec = CavitySpec(n, n // 2 + 3 if n < 500 else n, Ra=1e5, Da=1e-2, eps=0.6, Le=2.0, N=-1.5,
                      sigma=1.3, seed=8, noise=0.02)
    chunks = [37, 128, 64, 71] if n < 500 else [37, 66]
    ref, ref_reads = run(spec, layout, chunks, stream=LEGACY)
    for kw in ({}, {"graph_chunk": -1}):       # own stream with and without graph replay
        got, reads = run(spec, layout, chunks, **kw)
        for k in KEYS:
            assert np.array_equal(got[k], ref[k]), (kw, k)
        assert reads == ref_reads, kw


@pytest.mark.parametrize("precision", ["bf16", "f16"])
@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_16bit_pair_steps_equal_ordinary(layout, precision):
    """Two nodes per thread with the edge set in the first block rows of the same launch
    (ragged: odd nx, and an even nx whose last pair column is an edge column)."""
    for nx, ny in ((97, 41), (130, 67)):
        spec = CavitySpec(nx, ny, Ra=1e5, Da=1e-2, eps=0.6, Le=2.0, N=-1.5, sigma=1.3, seed=8,
                          noise=0.02)
        chunks = [37, 128, 71]
        ref, ref_reads = run(spec, layout, chunks, precision, stream=LEGACY)
        for kw in ({}, {"graph_chunk": -1}):
            got, reads = run(spec, layout, chunks, precision, **kw)
            for k in KEYS:
                assert np.array_equal(got[k], ref[k]), (nx, kw, k)
            assert reads == ref_reads, (nx, kw)


@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_batch_programmatic_launches_equal_ordinary(layout):
    specs = draw_batch(24, seed=4, sizes=(32, 64, 128))
    runs = []
    for kw in ({"stream": LEGACY}, {}, {"graph_chunk": -1}):
        b = lbm.Batch([lbm.make_instance(s) for s in specs], precision="f32", layout=layout, **kw)
        b.step(75)
        r1 = b.nusselt_sherwood().copy()
        b.step(131)
        runs.append(([b.fields(k) for k in range(len(specs))], r1, b.nusselt_sherwood().copy()))
        b.close()
    ref = runs[0]
    for got in runs[1:]:
        assert np.array_equal(got[1], ref[1]) and np.array_equal(got[2], ref[2])
        for fg, fr in zip(got[0], ref[0]):
            for k in KEYS:
                assert np.array_equal(fg[k], fr[k]), k
