"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: FP64 storage and arithmetic 1e-12 relative L2 on u, T, C; FP32
1e-5 relative L2 after 1000 steps.  Both sides draw the initial noise from
their own SplitMix64 implementation with the same seed and key.
"""
import os

import numpy as np
import pytest

from paper_1708_07525_gb300 import lbm
from paper_1708_07525_gb300.workloads import SMALL_AIDING, CavitySpec, throughput_cavity

pytestmark = pytest.mark.gpu

KEYS = ("ux", "uy", "T", "C")


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module", autouse=True)
def _threads(oracle_mod):
    oracle_mod.set_threads(os.cpu_count() or 1)


def make_pair(O, spec: CavitySpec, precision="f64", layout="ab", **kw):
    gpu = lbm.Cavity(*spec.args(), precision=precision, layout=layout, seed=spec.seed,
                     noise=spec.noise, **kw)
    p = O.derive(*spec.args())
    ora = O.Oracle(p, seed=spec.seed, noise=spec.noise)
    return gpu, ora


def compare(gpu, ora, tol, nush_tol=None, u_atol=0.0):
    """Relative L2 error of u, T, C within tol.  u_atol admits an absolute error
    on u for states where u is so small that the unshifted FP64 oracle's own
    rounding (about 1e-17 absolute on sums of O(0.1) populations) dominates."""
    fg = gpu.fields()
    fo = ora.fields()
    errs = {k: rel_l2(fg[k], fo[k]) for k in KEYS}
    for k in KEYS:
        if k in ("ux", "uy") and np.abs(fg[k] - fo[k]).max() <= u_atol:
            continue
        assert errs[k] <= tol, (k, errs)
    assert np.abs(fg["rho"] - fo["rho"]).max() <= 1e3 * tol
    if nush_tol is not None:
        ng, no = gpu.nusselt_sherwood(), ora.nusselt_sherwood()
        np.testing.assert_allclose(ng, no, rtol=nush_tol, atol=0)
    return errs


SMALL = [
    CavitySpec(3, 3, Ra=1e4, Da=1e-2, eps=0.6, Le=2.0, N=1.0, seed=11, noise=0.05),
    CavitySpec(5, 7, Ra=1e5, Da=1e-3, eps=0.4, Le=5.0, N=-1.0, seed=12, noise=0.05),
    CavitySpec(33, 17, Ra=1e5, Da=1e-1, eps=0.8, Le=3.0, N=2.0, sigma=1.7, seed=13, noise=0.02),
    CavitySpec(130, 67, Ra=3e4, Da=1e-2, eps=0.5, Le=0.7, N=-2.0, sigma=0.6, seed=14, noise=0.01),
]


@pytest.mark.parametrize("layout", ["ab", "aa"])
@pytest.mark.parametrize("nsteps", [0, 1, 2, 3])
def test_first_steps_f64(oracle_mod, layout, nsteps):
    """Initial state and the first steps (pull initialisation, AA parity)."""
    spec = SMALL[2]
    gpu, ora = make_pair(oracle_mod, spec, "f64", layout)
    gpu.step(nsteps)
    ora.step(nsteps)
    assert gpu.t == nsteps
    compare(gpu, ora, 1e-13, nush_tol=1e-13, u_atol=1e-15)


@pytest.mark.parametrize("layout", ["ab", "aa"])
@pytest.mark.parametrize("spec", SMALL, ids=lambda s: f"{s.nx}x{s.ny}")
def test_f64_1000_steps(oracle_mod, spec, layout):
    gpu, ora = make_pair(oracle_mod, spec, "f64", layout)
    gpu.step(1000)
    ora.step(1000)
    compare(gpu, ora, 1e-12, nush_tol=1e-11)


@pytest.mark.parametrize("layout", ["ab", "aa"])
@pytest.mark.parametrize("spec", SMALL[1:], ids=lambda s: f"{s.nx}x{s.ny}")
def test_f32_1000_steps(oracle_mod, spec, layout):
    gpu, ora = make_pair(oracle_mod, spec, "f32", layout)
    gpu.step(1000)
    ora.step(1000)
    compare(gpu, ora, 1e-5)


@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_small_aiding_cavity_10000_steps_f64(oracle_mod, layout):
    """64 x 64 porous cavity, Ra = 1e4, Da = 1e-2, eps = 0.6, Le = 2, N = 1, FP64."""
    gpu, ora = make_pair(oracle_mod, SMALL_AIDING, "f64", layout)
    gpu.step(10000)
    ora.step(10000)
    compare(gpu, ora, 1e-12, nush_tol=1e-12)


@pytest.mark.parametrize("precision", ["f32"])
def test_small_aiding_cavity_1000_steps_f32(oracle_mod, precision):
    gpu, ora = make_pair(oracle_mod, SMALL_AIDING, precision, "ab")
    gpu.step(1000)
    ora.step(1000)
    compare(gpu, ora, 1e-5)


def test_throughput_cavity_full_size_f32(oracle_mod):
    """4096^2 opposing-buoyancy cavity in FP32, the benchmark's launch
    configuration (two-buffer pull, default tile, graph replay), against the
    oracle over a short run on the whole grid."""
    spec = throughput_cavity(4096)
    gpu, ora = make_pair(oracle_mod, spec, "f32", "ab")
    n = 4
    gpu.step(n)
    ora.step(n)
    compare(gpu, ora, 1e-5)


def test_graph_and_tile_invariance_bitwise(oracle_mod):
    spec = SMALL[3]
    a = lbm.Cavity(*spec.args(), precision="f32", seed=spec.seed, noise=spec.noise, graph_chunk=-1)
    b = lbm.Cavity(*spec.args(), precision="f32", seed=spec.seed, noise=spec.noise, graph_chunk=16,
                   block=(32, 4))
    a.step(101)
    b.step(101)
    fa, fb = a.fields(), b.fields()
    for k in KEYS:
        assert np.array_equal(fa[k], fb[k]), k


@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_checkpoint_resume_bitwise(layout):
    spec = SMALL[2]
    a = lbm.Cavity(*spec.args(), precision="f32", layout=layout, seed=spec.seed, noise=spec.noise)
    a.step(333)
    blob = a.save()
    a.step(400)
    b = lbm.Cavity(*spec.args(), precision="f32", layout=layout, seed=99, noise=spec.noise)
    b.load(blob)
    assert b.t == 333
    b.step(400)
    fa, fb = a.fields(), b.fields()
    for k in KEYS:
        assert np.array_equal(fa[k], fb[k]), k


@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_checkpoint_across_precisions(layout):
    """A checkpoint loads into a context of another storage precision: widening is exact
    (FP32 -> FP64 -> FP32 gives back the FP32 state bit for bit; a 16-bit state read in FP32
    gives the same fields), and the widened state steps on in the new precision."""
    spec = SMALL[2]
    args = dict(layout=layout, seed=spec.seed, noise=spec.noise)
    a = lbm.Cavity(*spec.args(), precision="f32", **args)
    a.step(333)
    blob = a.save()
    b = lbm.Cavity(*spec.args(), precision="f64", **args)
    b.load(blob)
    assert b.t == 333
    c = lbm.Cavity(*spec.args(), precision="f32", **args)
    c.load(b.save())
    fa, fb, fc = a.fields(), b.fields(), c.fields()
    for k in KEYS:
        assert np.array_equal(fa[k], fc[k]), k
        assert rel_l2(fb[k], fa[k]) <= 1e-6, k
    a.step(500)
    b.step(500)
    fa, fb = a.fields(), b.fields()
    for k in KEYS:
        assert rel_l2(fa[k], fb[k]) <= 1e-5, k
    for prec in ("bf16", "f16"):
        h = lbm.Cavity(*spec.args(), precision=prec, **args)
        h.step(101)
        w = lbm.Cavity(*spec.args(), precision="f32", **args)
        w.load(h.save())
        fh, fw = h.fields(), w.fields()
        for k in KEYS:
            assert np.array_equal(fh[k], fw[k]), (prec, k)


def test_user_initial_fields_match_oracle(oracle_mod):
    from paper_1708_07525_gb300.workloads import random_fields
    spec = SMALL[2]
    T, Cc = random_fields(spec.nx, spec.ny, seed=5, amp=0.05)
    gpu = lbm.Cavity(*spec.args(), precision="f64", T_init=T, C_init=Cc)
    ora = oracle_mod.Oracle(oracle_mod.derive(*spec.args()), T_init=T, C_init=Cc)
    fg = gpu.fields()
    assert np.abs(fg["T"] - T).max() < 1e-15 and np.abs(fg["C"] - Cc).max() < 1e-15
    gpu.step(200)
    ora.step(200)
    compare(gpu, ora, 1e-12)


def test_residual_and_divergence_flag():
    spec = SMALL_AIDING
    g = lbm.Cavity(*spec.args(), precision="f32", seed=1)
    assert g.residual() == float("inf")     # no snapshot yet
    g.step(5000)
    r1 = g.residual()
    g.step(100)
    r2 = g.residual()
    assert 0 < r2 < 0.1 and r2 < r1
    # a non-finite initial value (made on the host) must be reported, not propagated silently
    T = np.full((16, 16), 0.5)
    T[8, 8] = np.nan
    bad = lbm.Cavity(16, 16, 1e4, 1e-2, 0.6, 1.0, 2.0, 1.0, precision="f32", T_init=T,
                     C_init=np.full((16, 16), 0.5))
    bad.step(50)
    with pytest.raises(lbm.LbmError) as ei:
        bad.residual()
    assert ei.value.status == lbm.ERR_DIVERGED
    bad.step(200)
    with pytest.raises(lbm.LbmError) as ei:
        bad.nusselt_sherwood()
    assert ei.value.status == lbm.ERR_DIVERGED


def test_precision_study_cavity_fp64_against_oracle(oracle_mod):
    """The 1024^2 precision-study cavity (Ra 1e5, Da 1e-2, eps 0.6, Le 10, N 2) in FP64
    against the oracle over a fixed 200 steps: the FP64 GPU path serves as the
    steady-state reference for the storage-precision study."""
    from paper_1708_07525_gb300.workloads import PRECISION_STUDY
    gpu, ora = make_pair(oracle_mod, PRECISION_STUDY, "f64", "ab")
    gpu.step(200)
    ora.step(200)
    # after 200 steps most of this large cavity is still at rest: u ~ 1e-6 there, below the
    # unshifted oracle's own rounding on sums of O(0.1) populations
    compare(gpu, ora, 1e-12, nush_tol=1e-12, u_atol=1e-15)


@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_model_a_f64_against_oracle(oracle_mod, layout):
    """The model-A equilibria (Eqs. 30-32) on the GPU against the oracle's."""
    spec = SMALL[3]
    p = lbm.lbm_params_model_a(lbm.lbm_derive_params(*spec.args()))
    po = oracle_mod.to_model_a(oracle_mod.derive(*spec.args()))
    assert abs(p.zeta[1] - po.zeta[1]) < 1e-14 and abs(p.eta[1] - po.eta[1]) < 1e-14
    gpu = lbm.Cavity(params=p, precision="f64", layout=layout, seed=spec.seed, noise=spec.noise)
    ora = oracle_mod.Oracle(po, seed=spec.seed, noise=spec.noise)
    gpu.step(1000)
    ora.step(1000)
    compare(gpu, ora, 1e-12, nush_tol=1e-11)


def smooth_fields(nx, ny, seed):
    """A porosity field in [0.45, 0.95] and a permeability field within a factor 3 of
    each other, smooth in space (sum of a few seeded Fourier modes)."""
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:ny, 0:nx] + 0.5
    e = np.zeros((ny, nx))
    k = np.zeros((ny, nx))
    for _ in range(3):
        a, b, ph = rng.uniform(0.5, 2.5, 3)
        e += np.sin(2 * np.pi * (a * x / nx + b * y / ny) + ph)
        k += np.cos(2 * np.pi * (b * x / nx - a * y / ny) + ph)
    eps = 0.7 + 0.25 * e / np.abs(e).max()
    K = 0.01 * nx * nx * np.exp(0.55 * k / np.abs(k).max())
    return eps, K


@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f32", 1e-5)])
@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_porous_fields_against_oracle(oracle_mod, precision, tol, layout):
    spec = CavitySpec(48, 37, Ra=5e4, Da=1e-2, eps=0.6, Le=3.0, N=-1.5, sigma=1.3, seed=21,
                      noise=0.02)
    eps, K = smooth_fields(spec.nx, spec.ny, seed=3)
    gpu = lbm.Cavity(*spec.args(), precision=precision, layout=layout, seed=spec.seed,
                     noise=spec.noise, eps_field=eps, K_field=K)
    ora = oracle_mod.Oracle(oracle_mod.derive(*spec.args()), seed=spec.seed, noise=spec.noise,
                            eps_field=eps, K_field=K)
    gpu.step(1000)
    ora.step(1000)
    compare(gpu, ora, tol, nush_tol=(1e-11 if precision == "f64" else None))


def test_porous_field_rejects_bad_values():
    eps = np.full((16, 16), 0.5)
    eps[3, 4] = 1.5
    with pytest.raises(lbm.LbmError) as ei:
        lbm.Cavity(16, 16, 1e4, 1e-2, 0.6, 1.0, 2.0, 1.0, eps_field=eps)
    assert ei.value.status == lbm.ERR_INVALID and "(4, 3)" in str(ei.value)
