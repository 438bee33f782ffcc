"""The steady-state residual of every GPU path against the oracle's (or_residual).

The residual decides when a steady run stops (the steady states of Sec. 4) and when the
server retires a request.  Each GPU path (lbm_residual, lbm_residual_noalloc, the batch
residual) is called on the same trajectory as the oracle, with the same number of steps
between calls, and its r must equal the oracle's within a bound derived from the field
errors measured at the two calls:

For one field let a, b be the GPU's values now and at the previous call, a', b' the
oracle's, e_a = max|a - a'|, e_b = max|b - b'|, D = max|a - b|, A = max|a| (D', A' the
oracle's, r' = D'/A').  Then |D - D'| <= e_a + e_b and |A - A'| <= e_a, so

    |D/A - D'/A'| <= (e_a + e_b + r' e_a) / (A' - e_a),

and the maximum over the four fields moves by no more than the largest of the four
bounds.  The GPU takes the differences in its compute precision on u, T - T0, C - C0 and
the maxima of |u|, |T|, |C| in that precision: another 4 units of its rounding times
(1 + r') each.  The bound is asserted to be small against r (so a wrong time level, a
wrong denominator or a missing field cannot hide in it), then r is held to it.
"""
import os

import numpy as np
import pytest

from paper_1708_07525_gb300 import lbm
from paper_1708_07525_gb300.workloads import CavitySpec

pytestmark = pytest.mark.gpu

KEYS = ("ux", "uy", "T", "C")
UNIT = {"f64": 2.0 ** -53, "f32": 2.0 ** -24, "bf16": 2.0 ** -24, "f16": 2.0 ** -24}

SPECS = [
    CavitySpec(33, 17, Ra=1e5, Da=1e-1, eps=0.8, Le=3.0, N=2.0, sigma=1.7, seed=13, noise=0.02),
    CavitySpec(130, 67, Ra=3e4, Da=1e-2, eps=0.5, Le=0.7, N=-2.0, sigma=0.6, seed=14, noise=0.01),
]


@pytest.fixture(scope="module", autouse=True)
def _threads(oracle_mod):
    oracle_mod.set_threads(os.cpu_count() or 1)


def stack(f):
    return np.stack([f[k] for k in KEYS])


def bound(g_now, o_now, g_prev, o_prev, r_or, precision):
    """Largest |r_gpu - r_oracle| the measured field errors allow (see the module text)."""
    worst = 0.0
    for q in range(4):
        A = np.abs(o_now[q]).max()
        ea = np.abs(g_now[q] - o_now[q]).max()
        eb = np.abs(g_prev[q] - o_prev[q]).max()
        if A == 0.0:
            continue
        b = (ea + eb + r_or * ea) / max(A - ea, 1e-300) + 4 * UNIT[precision] * (1 + r_or)
        worst = max(worst, b)
    return worst


def check_sequence(gpu_residual, gpu_step, gpu_fields, ora, plan, precision, rel_floor):
    """Step both sides by the counts in plan, calling the residuals after each; the first
    call must give +inf on both.  rel_floor: the bound must stay below rel_floor * r."""
    r_g = gpu_residual()
    r_o, bad = ora.residual()
    assert r_g == np.inf and r_o == np.inf and not bad
    g_prev, o_prev = stack(gpu_fields()), stack(ora.fields())
    checked = 0
    for n in plan:
        gpu_step(n)
        ora.step(n)
        r_g = gpu_residual()
        r_o, bad = ora.residual()
        assert not bad
        g_now, o_now = stack(gpu_fields()), stack(ora.fields())
        b = bound(g_now, o_now, g_prev, o_prev, r_o, precision)
        assert b <= rel_floor * r_o, (n, b, r_o)
        assert abs(r_g - r_o) <= b, (n, r_g, r_o, b)
        g_prev, o_prev = g_now, o_now
        checked += 1
    return checked


def cavity_pair(O, spec, precision, layout, params=None, oparams=None):
    if params is None:
        gpu = lbm.Cavity(*spec.args(), precision=precision, layout=layout, seed=spec.seed,
                         noise=spec.noise)
        ora = O.Oracle(O.derive(*spec.args()), seed=spec.seed, noise=spec.noise)
    else:
        gpu = lbm.Cavity(params=params, precision=precision, layout=layout, seed=spec.seed,
                         noise=spec.noise)
        ora = O.Oracle(oparams, seed=spec.seed, noise=spec.noise)
    return gpu, ora


# odd counts put the in-place layout's reads at both parities (local and pulled slots)
PLAN = (200, 101, 100, 37, 300)


@pytest.mark.parametrize("precision,floor", [("f64", 1e-9), ("f32", 2e-3)])
@pytest.mark.parametrize("layout", ["ab", "aa"])
@pytest.mark.parametrize("spec", SPECS, ids=lambda s: f"{s.nx}x{s.ny}")
def test_lbm_residual_against_oracle(oracle_mod, spec, layout, precision, floor):
    gpu, ora = cavity_pair(oracle_mod, spec, precision, layout)
    n = check_sequence(gpu.residual, gpu.step, gpu.fields, ora, PLAN, precision, floor)
    assert n == len(PLAN)
    gpu.close()


@pytest.mark.parametrize("precision,floor", [("f64", 1e-9), ("f32", 2e-3)])
def test_lbm_residual_with_wall_nodes_against_oracle(oracle_mod, precision, floor):
    """The paper's own walls (Sec. 3.3) with a convective right wall (Eq. 39): the residual
    reads the wall nodes through their rebuild."""
    args = (24, 1e4, 1e-2, 0.6, 1.0, 1.0, 1.0, 1.0, 200.0)
    spec = CavitySpec(25, 25, Ra=1e4, Da=1e-2, eps=0.6, seed=5, noise=0.02)
    gpu, ora = cavity_pair(oracle_mod, spec, precision, "ab",
                           params=lbm.lbm_derive_params_convective(*args),
                           oparams=oracle_mod.derive_convective(*args))
    check_sequence(gpu.residual, gpu.step, gpu.fields, ora, PLAN, precision, floor)
    gpu.close()


@pytest.mark.parametrize("which", ["T", "C"])
@pytest.mark.parametrize("precision,floor", [("f64", 1e-9), ("f32", 2e-3)])
@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_lbm_residual_of_each_scalar_alone(oracle_mod, which, precision, floor, layout):
    """No buoyancy (u = 0 throughout) and only one scalar driven by its walls (1 / 0) while
    the other's walls sit at its mean (its noise just decays): r is that scalar's change
    alone, so a slip in the T or in the C part of a GPU residual cannot hide behind the
    larger change of u or of the other scalar."""
    spec = SPECS[0]
    p = lbm.lbm_derive_params(*spec.args())
    po = oracle_mod.derive(*spec.args())
    for q in (p, po):
        q.gbT = q.gbC = 0.0
        hot, flat = (q.Tw, q.Cw) if which == "T" else (q.Cw, q.Tw)
        hot[0], hot[1] = 1.0, 0.0
        flat[0], flat[1] = 0.5, 0.5
    gpu, ora = cavity_pair(oracle_mod, spec, precision, layout, params=p, oparams=po)
    check_sequence(gpu.residual, gpu.step, gpu.fields, ora, PLAN, precision, floor)
    fl = ora.fields()
    assert np.abs(fl["ux"]).max() == 0.0 and np.abs(fl["uy"]).max() == 0.0
    gpu.close()


@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_lbm_residual_with_porous_field_against_oracle(oracle_mod, layout):
    """A porosity / permeability field (each node its own eps, K): T from Eq. 26 with the
    node's eps in C."""
    spec = CavitySpec(40, 29, Ra=5e4, Da=1e-2, eps=0.6, Le=3.0, N=-1.5, sigma=1.3, seed=21,
                      noise=0.02)
    y, x = np.mgrid[0:spec.ny, 0:spec.nx] + 0.5
    eps = 0.65 + 0.25 * np.sin(2 * np.pi * x / spec.nx) * np.cos(np.pi * y / spec.ny)
    K = 0.01 * spec.nx ** 2 * np.exp(0.4 * np.cos(2 * np.pi * (x + y) / spec.nx))
    gpu = lbm.Cavity(*spec.args(), precision="f64", layout=layout, seed=spec.seed,
                     noise=spec.noise, eps_field=eps, K_field=K)
    ora = oracle_mod.Oracle(oracle_mod.derive(*spec.args()), seed=spec.seed, noise=spec.noise,
                            eps_field=eps, K_field=K)
    check_sequence(gpu.residual, gpu.step, gpu.fields, ora, PLAN, "f64", 1e-9)
    gpu.close()


@pytest.mark.parametrize("precision,layout,floor", [("f64", "ab", 1e-9), ("f64", "aa", 1e-9),
                                                    ("f32", "aa", 2e-3)])
def test_lbm_residual_noalloc_against_oracle(oracle_mod, precision, layout, floor):
    """The entry point that allocates nothing, with the caller's snapshot buffer."""
    import torch
    spec = SPECS[1]
    gpu, ora = cavity_pair(oracle_mod, spec, precision, layout)
    snap = torch.zeros(4 * spec.nx * spec.ny, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    state = {"have": False}

    def res():
        r = gpu.residual_noalloc(snap.data_ptr(), state["have"])
        state["have"] = True
        return r

    check_sequence(res, gpu.step, gpu.fields, ora, PLAN, precision, floor)
    gpu.close()


@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_batch_residual_against_oracle(oracle_mod, layout):
    """Every slot of a batch (FP32) against its own oracle; the batch steps all slots
    together, so one plan serves them all."""
    specs = SPECS + [CavitySpec(64, 64, Ra=1e4, Da=1e-2, eps=0.6, Le=2.0, N=1.0, seed=1,
                                noise=0.01)]
    b = lbm.Batch([lbm.make_instance(s) for s in specs], precision="f32", layout=layout)
    oras = [oracle_mod.Oracle(oracle_mod.derive(*s.args()), seed=s.seed, noise=s.noise)
            for s in specs]
    r_g, d = b.residual()
    assert np.all(r_g[:len(specs)] == np.inf) and not d.any()
    prev_g = [stack(b.fields(k)) for k in range(len(specs))]
    prev_o = []
    for o in oras:
        assert o.residual()[0] == np.inf
        prev_o.append(stack(o.fields()))
    for n in PLAN:
        b.step(n)
        r_g, d = b.residual()
        assert not d.any()
        for k, o in enumerate(oras):
            o.step(n)
            r_o, _ = o.residual()
            g_now, o_now = stack(b.fields(k)), stack(o.fields())
            bd = bound(g_now, o_now, prev_g[k], prev_o[k], r_o, "f32")
            assert bd <= 2e-3 * r_o, (k, n, bd, r_o)
            assert abs(r_g[k] - r_o) <= bd, (k, n, r_g[k], r_o, bd)
            prev_g[k], prev_o[k] = g_now, o_now
    b.close()


@pytest.mark.parametrize("precision", ["bf16", "f16"])
def test_lbm_residual_16bit_storage_transient(oracle_mod, precision):
    """16-bit storage early in the transient, where r is large: the same bound, with the
    field errors of 16-bit storage, still fixes r to a few per cent."""
    spec = CavitySpec(64, 64, Ra=1e5, Da=1e-2, eps=0.6, Le=2.0, N=1.0, seed=7, noise=0.05)
    gpu, ora = cavity_pair(oracle_mod, spec, precision, "ab")
    check_sequence(gpu.residual, gpu.step, gpu.fields, ora, (100, 100, 100), precision, 0.1)
    gpu.close()
