"""Walls with nodes on them (Sec. 3.3, Eqs. 33-37) and convective walls (Eq. 39) on
the GPU, through the C ABI, against the FP64 oracle: FP64 1e-12 relative L2 on
u, T, C (and Nu / Sh to 1e-11), FP32 1e-5 after 1000 steps.  Cases: the
convective cavity of Sec. 4.2 (both Biot numbers, model A), Dirichlet walls
with porosity / permeability fields, a moving lid, a ragged grid; and the
paper's Tables 2-3 through the stored oracle values."""
import json
import os

import numpy as np
import pytest

from paper_1708_07525_gb300 import lbm

pytestmark = pytest.mark.gpu
KEYS = ("ux", "uy", "T", "C")
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module", autouse=True)
def _threads(oracle_mod):
    oracle_mod.set_threads(os.cpu_count() or 1)


def edit(p, **kw):
    """Apply the same wall edits to a GPU or an oracle parameter struct."""
    for k, v in kw.items():
        if k in ("Tw", "Cw", "BiT", "BiC"):
            for s, x in enumerate(v):
                getattr(p, k)[s] = x
        elif k == "uw":
            for s, (a, b) in enumerate(v):
                p.uw[s][0], p.uw[s][1] = a, b
        elif k == "tb_dirichlet":
            if hasattr(p, "wall_tb"):
                p.wall_lr, p.wall_tb = (lbm.WALL_ADIABATIC, lbm.WALL_DIRICHLET) if v else \
                    (lbm.WALL_DIRICHLET, lbm.WALL_ADIABATIC)
            else:
                p.scalar_lr, p.scalar_tb = (1, 0) if v else (0, 1)
        else:
            setattr(p, k, v)
    return p


def convective_pair(O, Nx, BiC, precision="f64", model_a=False, seed=3, noise=0.02, **kw):
    args = (Nx, 1e4, 1e-2, 0.6, 1.0, 1.0, 1.0, 1.0, BiC)
    pg = lbm.lbm_derive_params_convective(*args)
    po = O.derive_convective(*args)
    if model_a:
        lbm.lbm_params_model_a(pg)
        O.to_model_a(po)
    gpu = lbm.Cavity(params=pg, precision=precision, seed=seed, noise=noise, **kw)
    ora = O.Oracle(po, seed=seed, noise=noise, eps_field=kw.get("eps_field"),
                   K_field=kw.get("K_field"))
    return gpu, ora


def nee_pair(O, nx, ny, args, edits, precision="f64", seed=5, noise=0.02, **kw):
    pg = edit(lbm.lbm_derive_params_nee(nx, ny, *args), **edits)
    po = edit(O.derive(nx, ny, *args, nee=True), **edits)
    gpu = lbm.Cavity(params=pg, precision=precision, seed=seed, noise=noise, **kw)
    ora = O.Oracle(po, seed=seed, noise=noise, eps_field=kw.get("eps_field"),
                   K_field=kw.get("K_field"))
    return gpu, ora


def check(gpu, ora, tol, nush_tol=None, lr=True, tb=False, u_atol=1e-15):
    fg, fo = gpu.fields(), ora.fields()
    errs = {k: rel_l2(fg[k], fo[k]) for k in KEYS}
    for k in KEYS:
        # velocities of O(1e-7) in the first steps: the unshifted oracle's own rounding
        if k in ("ux", "uy") and np.abs(fg[k] - fo[k]).max() <= u_atol:
            continue
        assert errs[k] <= tol, (k, errs)
    if nush_tol is not None:
        if lr:     # the wall pair with the temperature difference
            np.testing.assert_allclose(gpu.nusselt_sherwood(), ora.nusselt_sherwood(),
                                       rtol=nush_tol)
        if tb:
            np.testing.assert_allclose(gpu.nusselt_sherwood_tb(), ora.nusselt_sherwood_tb(),
                                       rtol=nush_tol)
    return errs


@pytest.mark.parametrize("nsteps", [0, 1, 7, 1000])
@pytest.mark.parametrize("BiC", [1.0, 200.0])
def test_convective_cavity_f64(oracle_mod, BiC, nsteps):
    gpu, ora = convective_pair(oracle_mod, 40, BiC)
    gpu.step(nsteps)
    ora.step(nsteps)
    check(gpu, ora, 1e-12, nush_tol=1e-11)
    gpu.close()


def test_convective_cavity_model_a_f64(oracle_mod):
    gpu, ora = convective_pair(oracle_mod, 32, 1.0, model_a=True)
    gpu.step(1000)
    ora.step(1000)
    check(gpu, ora, 1e-12, nush_tol=1e-11)
    gpu.close()


@pytest.mark.parametrize("precision", ["f32"])
def test_convective_cavity_f32_1000_steps(oracle_mod, precision):
    gpu, ora = convective_pair(oracle_mod, 64, 200.0, precision=precision)
    gpu.step(1000)
    ora.step(1000)
    check(gpu, ora, 1e-5)
    gpu.close()


def smooth_fields(nx, ny, seed):
    """Porosity in about [0.45, 0.95] and a permeability within a factor 3 of
    Da L^2, smooth in space (a few seeded Fourier modes)."""
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    e = np.zeros((ny, nx))
    k = np.zeros((ny, nx))
    for _ in range(3):
        a, b, ph = rng.uniform(0.5, 2.5, 3)
        e += np.sin(2 * np.pi * (a * x / nx + b * y / ny) + ph)
        k += np.cos(2 * np.pi * (b * x / nx - a * y / ny) + ph)
    eps = 0.7 + 0.25 * e / np.abs(e).max()
    K = 0.01 * (nx - 1) ** 2 * np.exp(0.55 * k / np.abs(k).max())
    return eps, K


@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_dirichlet_walls_with_porous_fields(oracle_mod, precision, tol):
    """Ragged grid (the rebuild reads each node's own porosity: eps_b in f^eq of the
    wall node, eps_f at x_f, eps at x_ff for C_ff), opposing buoyancy."""
    nx, ny = 45, 29
    eps, K = smooth_fields(nx, ny, seed=8)
    gpu, ora = nee_pair(oracle_mod, nx, ny, (5e4, 1e-2, 0.6, 1.0, 3.0, -1.5),
                        dict(sigma=1.3), precision=precision, eps_field=eps, K_field=K)
    gpu.step(1000)
    ora.step(1000)
    check(gpu, ora, tol, nush_tol=(1e-11 if precision == "f64" else None))
    gpu.close()


@pytest.mark.parametrize("nsteps", [1, 1000])
def test_moving_lid_with_wall_nodes_f64(oracle_mod, nsteps):
    """Eq. 33 with u_w = (U0, 0) on the top wall (corner nodes take the top wall's
    velocity), Dirichlet top / bottom, adiabatic sides, a convective bottom-left mix:
    BiT on the left side exercises Eq. 36 with a gradient condition on a vertical wall."""
    edits = dict(tb_dirichlet=True, Tw=(0.5, 0.5, 0.0, 1.0), Cw=(0.5, 0.5, 0.0, 1.0),
                 uw=((0, 0), (0, 0), (0, 0), (0.08, 0)), BiT=(0.7, 0, 0, 0), BiC=(0, 2.5, 0, 0))
    gpu, ora = nee_pair(oracle_mod, 37, 31, (2e4, 1e-1, 0.8, 1.0, 1.5, 0.5), edits)
    gpu.step(nsteps)
    ora.step(nsteps)
    check(gpu, ora, 1e-12, nush_tol=1e-11, lr=False, tb=True)
    gpu.close()


def test_residual_and_window_on_wall_nodes(oracle_mod):
    """Read-outs go through the same rebuild: a window on the right (convective) wall
    equals the full fields there, and the residual is finite and falls."""
    gpu, ora = convective_pair(oracle_mod, 30, 200.0)
    gpu.step(300)
    full = gpu.fields()
    win = gpu.fields_window(27, 0, 4, 31)
    for k in KEYS:
        np.testing.assert_array_equal(win[k], full[k][:, 27:31])
    assert gpu.residual() == float("inf")
    gpu.step(100)
    r1 = gpu.residual()
    gpu.step(3000)
    gpu.residual()
    gpu.step(100)
    r2 = gpu.residual()
    assert np.isfinite(r1) and 0 < r2 < r1
    gpu.close()


def stream_max(ux):
    """max |psi| with u_x = d psi / dy, psi = 0 on the bottom wall node (trapezoids
    up each column)."""
    psi = np.concatenate([np.zeros((1, ux.shape[1])),
                          np.cumsum(0.5 * (ux[1:] + ux[:-1]), axis=0)])
    return np.abs(psi).max()


@pytest.mark.parametrize("case", ["bic1", "bic200", "bic1_model_a"])
def test_tables_2_3_gpu_against_stored_oracle(case):
    """The GPU FP64 run to the oracle's step count reproduces the stored oracle
    values of Tables 2-3's quantities (written by tests/golden/make_table2.py)."""
    with open(os.path.join(GOLD, "table2_oracle.json")) as f:
        ora = json.load(f)
    rec = ora[case]
    pg = lbm.lbm_derive_params_convective(100, 1e4, 1e-2, 0.6, 1.0, 1.0, 1.0, 1.0, rec["bi_c"])
    if rec["model_a"]:
        lbm.lbm_params_model_a(pg)
    gpu = lbm.Cavity(params=pg, precision="f64", seed=ora["seed"], noise=ora["noise"])
    gpu.step(rec["steps"])
    ns = gpu.nusselt_sherwood()
    fl = gpu.fields(("ux", "T", "C"))
    np.testing.assert_allclose(ns, [rec["nu_left"], rec["sh_left"], rec["nu_right"],
                                    rec["sh_right"]], rtol=1e-9)
    assert abs(fl["T"].min() - rec["theta_min"]) < 1e-9
    assert abs(fl["C"].min() - rec["phi_min"]) < 1e-9
    alpha = pg.nu / 1.0
    assert abs(stream_max(fl["ux"]) / alpha - rec["psi_max_over_alpha"]) < 1e-7
    gpu.close()


@pytest.mark.parametrize("precision", ["bf16", "f16"])
def test_convective_cavity_16bit_storage(oracle_mod, precision):
    """16-bit storage with the rebuild: the wall values are imposed in the FP32 arithmetic
    of the read-out (the rebuilt g sums to sigma T_w whatever x_f stored), and the fields
    follow the FP64 oracle within the rounding noise of 8-11 significant bits."""
    gpu, ora = convective_pair(oracle_mod, 40, 200.0, precision=precision)
    gpu.step(1000)
    ora.step(1000)
    fg, fo = gpu.fields(), ora.fields()
    np.testing.assert_allclose(fg["T"][:, 0], 1.0, rtol=0, atol=1e-6)
    np.testing.assert_allclose(fg["C"][:, 0], 1.0, rtol=0, atol=1e-6)
    for k in ("T", "C"):
        assert rel_l2(fg[k], fo[k]) <= 2e-2, (k, rel_l2(fg[k], fo[k]))
    assert np.isfinite(gpu.nusselt_sherwood()).all()
    gpu.close()


def test_checkpoint_resume_with_wall_nodes_bitwise():
    """A checkpoint carries the wall-node parameters (nee, Biot numbers): a plain cavity
    of the same grid that loads it resumes bit for bit; an in-place context refuses it."""
    p = lbm.lbm_derive_params_convective(36, 1e4, 1e-2, 0.6, 1.0, 1.0, 1.0, 1.0, 200.0)
    a = lbm.Cavity(params=p, precision="f32", seed=3, noise=0.02)
    a.step(333)
    blob = a.save()
    a.step(400)
    b = lbm.Cavity(37, 37, 1e4, 1e-2, 0.6, 1.0, 1.0, 1.0, precision="f32", seed=99)
    b.load(blob)
    assert b.t == 333 and b.params.nee == 1 and b.params.BiC[1] == 200.0
    b.step(400)
    fa, fb = a.fields(), b.fields()
    for k in KEYS:
        assert np.array_equal(fa[k], fb[k]), k
    np.testing.assert_array_equal(a.nusselt_sherwood(), b.nusselt_sherwood())
    c = lbm.Cavity(37, 37, 1e4, 1e-2, 0.6, 1.0, 1.0, 1.0, precision="f32", layout="aa")
    with pytest.raises(lbm.LbmError) as ei:
        c.load(blob)
    assert ei.value.status == lbm.ERR_INVALID
    for x in (a, b, c):
        x.close()


@pytest.mark.parametrize("nx,ny", [(5, 5), (5, 9), (11, 5)])
def test_smallest_wall_node_grids_f64(oracle_mod, nx, ny):
    """The smallest grids the rebuild allows (x_ff two nodes in from each wall): every
    node is within two of a wall, corners meet, and a convective wall is on."""
    edits = dict(BiT=(0, 1.5, 0, 0), BiC=(0, 0.5, 0, 0))
    gpu, ora = nee_pair(oracle_mod, nx, ny, (1e4, 1e-2, 0.6, 1.0, 2.0, 1.0), edits, noise=0.05)
    gpu.step(300)
    ora.step(300)
    check(gpu, ora, 1e-12, nush_tol=1e-11, tb=False)
    gpu.close()
