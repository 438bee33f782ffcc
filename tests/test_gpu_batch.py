"""The batched path (many cavities, one fused launch per step): parity with the
oracle, bitwise independence of a cavity from the rest of the batch, dynamic
membership at odd times, tile-shape invariance, arena admission."""
import os

import numpy as np
import pytest

from paper_1708_07525_gb300 import lbm
from paper_1708_07525_gb300.workloads import CavitySpec, draw_batch

pytestmark = pytest.mark.gpu
KEYS = ("ux", "uy", "T", "C")


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


MIX = [
    CavitySpec(33, 17, Ra=1e5, Da=1e-1, eps=0.8, Le=3.0, N=2.0, sigma=1.7, seed=13, noise=0.02),
    CavitySpec(64, 64, Ra=1e4, Da=1e-2, eps=0.6, Le=2.0, N=1.0, seed=1),
    CavitySpec(130, 67, Ra=3e4, Da=1e-2, eps=0.5, Le=0.7, N=-2.0, sigma=0.6, seed=14, noise=0.01),
    CavitySpec(5, 7, Ra=1e5, Da=1e-3, eps=0.4, Le=5.0, N=-1.0, seed=12, noise=0.05),
]


@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_batch_matches_oracle_f32(oracle_mod, layout):
    oracle_mod.set_threads(os.cpu_count() or 1)
    b = lbm.Batch([lbm.make_instance(s) for s in MIX], precision="f32", layout=layout)
    b.step(1000)
    nush = b.nusselt_sherwood()
    for k, s in enumerate(MIX):
        o = oracle_mod.Oracle(oracle_mod.derive(*s.args()), seed=s.seed, noise=s.noise)
        o.step(1000)
        fo, fg = o.fields(), b.fields(k)
        for key in KEYS:
            assert rel_l2(fg[key], fo[key]) <= 1e-5, (s, key)
        np.testing.assert_allclose(nush[k], o.nusselt_sherwood(), rtol=1e-4)


@pytest.mark.parametrize("precision,layout", [("f32", "ab"), ("f32", "aa"), ("bf16", "ab"),
                                              ("f16", "aa")])
def test_alone_equals_in_mix_bitwise(precision, layout):
    target = MIX[2]
    others = draw_batch(20, seed=4, sizes=(32, 64, 128))
    alone = lbm.Batch([lbm.make_instance(target)], precision=precision, layout=layout)
    mix = lbm.Batch([lbm.make_instance(s) for s in others[:7]] + [lbm.make_instance(target)]
                    + [lbm.make_instance(s) for s in others[7:]], precision=precision, layout=layout)
    alone.step(357)
    mix.step(357)
    fa, fm = alone.fields(0), mix.fields(7)
    for key in KEYS:
        assert np.array_equal(fa[key], fm[key]), key
    assert np.array_equal(alone.nusselt_sherwood()[0], mix.nusselt_sherwood()[7])


def test_batch_equals_single_cavity_path():
    s = MIX[1]
    single = lbm.Cavity(*s.args(), precision="f32", seed=s.seed, noise=s.noise)
    b = lbm.Batch([lbm.make_instance(x) for x in MIX], precision="f32")
    single.step(500)
    b.step(500)
    fs, fb = single.fields(), b.fields(1)
    for key in KEYS:
        assert rel_l2(fb[key], fs[key]) <= 1e-6, key


@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_add_at_odd_time_and_remove(layout):
    """A cavity added at an odd batch time evolves exactly as one added at t = 0."""
    target = MIX[0]
    ref = lbm.Batch([lbm.make_instance(target)], precision="f32", layout=layout)
    ref.step(200)
    need = lbm.batch_instance_bytes(64, 64, "f32", layout) * 6
    b = lbm.Batch([lbm.make_instance(MIX[1])], capacity=4, arena_bytes=need, precision="f32",
                  layout=layout)
    b.step(77)
    slot = b.add(lbm.make_instance(target))
    assert b.time(slot) == 0
    b.step(200)
    assert b.time(slot) == 200
    fr, fb = ref.fields(0), b.fields(slot)
    for key in KEYS:
        assert np.array_equal(fr[key], fb[key]), key
    b.remove(0)
    b.step(3)
    assert b.time(0) == -1 and b.time(slot) == 203
    assert b.info()["used"] == 1


def test_arena_admission_budget():
    need = lbm.batch_instance_bytes(64, 64, "bf16", "ab")
    b = lbm.Batch([], capacity=8, arena_bytes=2 * need + 1024, precision="bf16")
    s0 = b.add(lbm.make_instance(MIX[1]))
    s1 = b.add(lbm.make_instance(MIX[1]))
    with pytest.raises(lbm.LbmError) as ei:
        b.add(lbm.make_instance(MIX[1]))
    assert ei.value.status == lbm.ERR_NOMEM
    b.remove(s0)
    s2 = b.add(lbm.make_instance(MIX[1]))
    assert s2 == s0 and b.info()["used"] == 2
    b.step(10)


def test_autotune_keeps_results_and_residual_per_slot():
    insts = [lbm.make_instance(s) for s in draw_batch(12, seed=9, sizes=(32, 64, 128))]
    a = lbm.Batch(insts, precision="f32")
    c = lbm.Batch(insts, precision="f32")
    rep = a.autotune(trial_steps=6)
    lines = [ln.split() for ln in rep.strip().splitlines() if not ln.startswith("#")]
    assert {(int(x[0]), int(x[1])) for x in lines} == {(i.params.nx, i.params.ny) for i in insts}
    for x in lines:
        assert int(x[2]) in (32, 64, 128, 256) and float(x[4]) > 0
    a.step(150)
    c.step(150)
    for k in range(len(insts)):
        fa, fc = a.fields(k), c.fields(k)
        for key in KEYS:
            assert np.array_equal(fa[key], fc[key]), (k, key)
    r0, d0 = a.residual()
    assert np.all(np.isinf(r0)) and not d0.any()
    a.step(100)
    r1, d1 = a.residual()
    assert np.all(np.isfinite(r1)) and np.all(r1 > 0) and not d1.any()
    single = lbm.Cavity(params=insts[3].params, precision="f32", seed=insts[3].seed,
                        noise=insts[3].noise)
    single.step(150)
    single.residual()
    single.step(100)
    assert abs(single.residual() - r1[3]) <= 1e-5 * r1[3]


@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_l2_blocking_keeps_results_bitwise(layout):
    insts = [lbm.make_instance(s) for s in draw_batch(16, seed=11, sizes=(32, 64, 128))]
    a = lbm.Batch(insts, precision="f32", layout=layout)
    b = lbm.Batch(insts, precision="f32", layout=layout)
    a.set_blocking(1)
    b.set_blocking(6, l2_bytes=1 << 20)      # many small groups, 6 steps each
    a.step(137)
    b.step(137)
    for k in range(len(insts)):
        fa, fb = a.fields(k), b.fields(k)
        for key in KEYS:
            assert np.array_equal(fa[key], fb[key]), (k, key)


def test_wall_node_cavities_in_a_batch_equal_the_single_cavity_bitwise():
    """Cavities with the paper's own walls (Sec. 3.3, a convective wall) share a batch with
    halfway-wall cavities: each gives bit for bit the fields of the single-cavity path
    (the same per-node arithmetic), and Nu / Sh with the node stencil."""
    pc = lbm.lbm_derive_params_convective(40, 1e4, 1e-2, 0.6, 1.0, 1.0, 1.0, 1.0, 200.0)
    pn = lbm.lbm_derive_params_nee(37, 29, 5e4, 1e-2, 0.6, 1.0, 3.0, -1.5)
    insts = [lbm.make_instance(MIX[0]), lbm.make_instance(params=pc, seed=3, noise=0.02),
             lbm.make_instance(MIX[1]), lbm.make_instance(params=pn, seed=5, noise=0.02)]
    b = lbm.Batch(insts, precision="f32")
    b.step(357)
    nush = b.nusselt_sherwood()
    for k, (p, seed) in ((1, (pc, 3)), (3, (pn, 5))):
        single = lbm.Cavity(params=p, precision="f32", seed=seed, noise=0.02)
        single.step(357)
        fs, fb = single.fields(), b.fields(k)
        for key in KEYS:
            assert np.array_equal(fs[key], fb[key]), (k, key)
        np.testing.assert_allclose(nush[k], single.nusselt_sherwood(), rtol=1e-12)
        single.close()
    # the halfway cavities of the same batch are untouched by the wall-node kernel
    alone = lbm.Batch([lbm.make_instance(MIX[1])], precision="f32")
    alone.step(357)
    for key in KEYS:
        assert np.array_equal(alone.fields(0)[key], b.fields(2)[key]), key


def test_wall_node_cavity_rejected_by_in_place_batches():
    pc = lbm.lbm_derive_params_convective(40, 1e4, 1e-2, 0.6, 1.0, 1.0, 1.0, 1.0, 1.0)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.Batch([lbm.make_instance(params=pc)], precision="f32", layout="aa")
    assert ei.value.status == lbm.ERR_INVALID


@pytest.mark.parametrize("precision,layout", [("f32", "ab"), ("f32", "aa"), ("bf16", "ab")])
def test_cavity_beyond_its_l2_share_runs_the_single_cavity_kernels(precision, layout):
    """A 512^2 cavity (44 MB of FP32 state, more than a lane's quarter of L2) is stepped by
    the single-cavity kernels inside the batch: bit for bit the single-cavity run (one node
    per thread), while the small cavities beside it keep their tile kernel."""
    big = CavitySpec(512, 512, Ra=1e5, Da=1e-2, eps=0.6, Le=2.0, N=-1.0, seed=21, noise=0.02)
    b = lbm.Batch([lbm.make_instance(MIX[0]), lbm.make_instance(big), lbm.make_instance(MIX[2])],
                  precision=precision, layout=layout)
    b.step(101)
    if precision == "f32":
        single = lbm.Cavity(*big.args(), precision=precision, layout=layout, seed=big.seed,
                            noise=big.noise)
    else:   # the one-node 16-bit kernels (a one-slab cavity runs them, see lbm_create_slab)
        single = lbm.Cavity(params=lbm.lbm_derive_params(*big.args()), slab=(0, big.ny),
                            precision=precision, layout=layout, seed=big.seed, noise=big.noise)
    single.step(101)
    fb, fs = b.fields(1), single.fields()
    for key in KEYS:
        assert np.array_equal(fb[key], fs[key]), key
    alone = lbm.Batch([lbm.make_instance(MIX[2])], precision=precision, layout=layout)
    alone.step(101)
    for key in KEYS:
        assert np.array_equal(alone.fields(0)[key], b.fields(2)[key]), key
