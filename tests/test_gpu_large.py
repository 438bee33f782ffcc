"""Full-size and maximum-size grids, checked on sampled windows.

After n steps the state of a node depends only on the initial state within n
nodes of it, so the oracle run on a small window (with the full grid's lattice
constants and the full grid's noise keys) reproduces the big grid exactly at
every node farther than n + 1 nodes from the window's artificial edges (edges
that coincide with the cavity's walls are the real walls).  The big grid is
read back window by window (lbm_fields_window)."""
import os

import numpy as np
import pytest

from paper_1708_07525_gb300 import lbm
from paper_1708_07525_gb300.workloads import CavitySpec, throughput_cavity

pytestmark = pytest.mark.gpu


def oracle_window(O, spec, x0, y0, w, h, steps):
    p = O.derive(*spec.args(), varpi=spec.varpi)
    p.nx, p.ny = w, h                      # constants of the full grid, window extent
    nfull = spec.nx * spec.ny
    T = np.empty((h, w))
    C = np.empty((h, w))
    for jj in range(h):
        for ii in range(w):
            k = (y0 + jj) * spec.nx + (x0 + ii)
            T[jj, ii] = 0.5 + spec.noise * (2.0 * O.uniform(spec.seed, k) - 1.0)
            C[jj, ii] = 0.5 + spec.noise * (2.0 * O.uniform(spec.seed, nfull + k) - 1.0)
    o = O.Oracle(p, seed=spec.seed, noise=spec.noise, T_init=T, C_init=C)
    o.step(steps)
    return o.fields()


def trusted_mask(spec, x0, y0, w, h, steps):
    m = np.ones((h, w), bool)
    d = steps + 1
    if x0 > 0:
        m[:, :d] = False
    if x0 + w < spec.nx:
        m[:, w - d:] = False
    if y0 > 0:
        m[:d, :] = False
    if y0 + h < spec.ny:
        m[h - d:, :] = False
    return m


def check_windows(O, cav, spec, windows, steps, tol_rel, keys=("ux", "uy", "T", "C")):
    for (x0, y0, w, h) in windows:
        fo = oracle_window(O, spec, x0, y0, w, h, steps)
        fg = cav.fields_window(x0, y0, w, h)
        m = trusted_mask(spec, x0, y0, w, h, steps)
        assert m.sum() > 100
        for k in keys:
            a, b = fg[k][m], fo[k][m]
            if k in ("T", "C"):                 # compare deviations from the reference value
                a, b = a - 0.5, b - 0.5
            err = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)
            assert err <= tol_rel, ((x0, y0), k, err)


@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_benchmark_cavity_4096_f32_sampled(oracle_mod, layout):
    """In place, the odd steps at this size run the ring of outermost nodes and the inner
    nodes in one launch (the ring's block rows first)."""
    spec = throughput_cavity(4096)
    steps = 40
    cav = lbm.Cavity(*spec.args(), precision="f32", layout=layout, seed=spec.seed, noise=spec.noise)
    cav.step(steps)
    wins = [(0, 0, 96, 96), (0, 2000, 96, 96), (4000, 4000, 96, 96), (2000, 2000, 96, 96),
            (4000, 17, 96, 96)]
    check_windows(oracle_mod, cav, spec, wins, steps, 1e-5, keys=("T", "C"))
    # at step 40 the velocity is ~1e-4 of its final size; FP32 rounding of the O(1e-3)
    # populations it is formed from gives a few 1e-5 relative
    check_windows(oracle_mod, cav, spec, wins, steps, 1e-4, keys=("ux", "uy"))


def test_benchmark_cavity_4096_f32_1000_steps_windows(oracle_mod):
    """The 4096^2 benchmark cavity in FP32 in the benchmark's launch configuration over
    1000 steps, against oracle windows of 1100 x 1100 nodes at the four corners and of
    1100 x 2100 nodes on the left wall: each trusts the nodes more than 1001 nodes from
    its artificial edges (99 x 99 at a corner).  The bar is FP32's 1e-5 relative L2 on
    u, T - T0, C - C0.  After 1000 steps the flow near the walls is still ~1e-5 in size
    and, half way up the left wall, u_x is ~1e-9: below the resolution of the O(1e-4)
    populations it is summed from (FP32 ulp ~1e-11), so u also passes where its absolute
    error stays below 1e-10."""
    O = oracle_mod
    O.set_threads(os.cpu_count() or 1)
    spec = throughput_cavity(4096)
    n, steps, W = spec.nx, 1000, 1100
    cav = lbm.Cavity(*spec.args(), precision="f32", seed=spec.seed, noise=spec.noise)
    cav.step(steps)
    wins = [(0, 0, W, W), (n - W, 0, W, W), (0, n - W, W, W), (n - W, n - W, W, W),
            (0, 1500, W, 2100)]
    for (x0, y0, w, h) in wins:
        p = O.derive(*spec.args(), varpi=spec.varpi)
        p.nx, p.ny = w, h                  # constants of the full grid, window extent
        T, C = O.noise_window(spec.seed, spec.noise, n, n, x0, y0, w, h)
        o = O.Oracle(p, seed=spec.seed, noise=spec.noise, T_init=T, C_init=C)
        o.step(steps)
        fo = o.fields()
        fg = cav.fields_window(x0, y0, w, h)
        m = trusted_mask(spec, x0, y0, w, h, steps)
        assert m.sum() >= 99 * 98
        for k in ("ux", "uy", "T", "C"):
            a, b = fg[k][m], fo[k][m]
            if k in ("T", "C"):
                a, b = a - 0.5, b - 0.5
            err = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)
            if k in ("ux", "uy") and np.abs(a - b).max() <= 1e-10:
                continue
            assert err <= 1e-5, ((x0, y0), k, err)
    cav.close()


def test_beyond_2_31_nodes_f16_aa_sampled(oracle_mod):
    """46400^2 = 2.15e9 nodes (> 2^31) in FP16 in-place storage (about 116 GB)."""
    n = 46400
    spec = CavitySpec(n, n, Ra=1e5, Da=1e-3, eps=0.4, Le=5.0, N=-1.0, seed=9, noise=0.05)
    steps = 6
    cav = lbm.Cavity(*spec.args(), precision="f16", layout="aa", seed=spec.seed, noise=spec.noise)
    assert cav.device_bytes() > 100e9
    cav.step(steps)
    wins = [(0, 0, 48, 48), (n - 48, n - 48, 48, 48), (n // 2, n - 48, 48, 48),
            (n - 48, 12345, 48, 48), (31000, 40000, 48, 48)]
    # FP16 storage (11 significant bits, stochastic rounding) against FP64.  A wrong
    # index would give O(1) errors; the velocity after 6 steps is far below the rounding
    # noise of the pressure-dominated populations and is not compared.
    check_windows(oracle_mod, cav, spec, wins, steps, 2e-2, keys=("T", "C"))
    cav.close()


def test_window_and_empty_step_edges():
    spec = CavitySpec(37, 29, Ra=1e4, Da=1e-2, eps=0.6, Le=2.0, N=1.0, seed=3)
    cav = lbm.Cavity(*spec.args(), precision="f32", seed=spec.seed)
    before = cav.fields()
    cav.step(0)                                    # an empty step is a no-op
    assert cav.t == 0
    after = cav.fields()
    for k in before:
        assert np.array_equal(before[k], after[k])
    cav.step(17)
    full = cav.fields()
    win = cav.fields_window(5, 3, 20, 11)
    for k in full:
        assert np.array_equal(win[k], full[k][3:14, 5:25])
    for bad in ((-1, 0, 5, 5), (30, 0, 10, 5), (0, 0, 0, 5), (0, 25, 5, 5)):
        with pytest.raises(lbm.LbmError) as ei:
            cav.fields_window(*bad)
        assert ei.value.status == lbm.ERR_INVALID


def test_wall_nodes_4096_f32_sampled(oracle_mod):
    """The paper's own walls (Sec. 3.3) on the 4096^2 benchmark cavity in the benchmark's
    launch configuration (inner kernel + wall-ring kernel), checked on windows at the
    four corners and two walls.  The rebuild reads two nodes in from the wall, so the
    trusted region keeps steps + 2 nodes away from a window's artificial edges."""
    O = oracle_mod
    spec = throughput_cavity(4096)
    n, steps = spec.nx, 30
    p = lbm.lbm_derive_params_nee(n, n, spec.Ra, spec.Da, spec.eps, spec.Pr, spec.Le, spec.N)
    cav = lbm.Cavity(params=p, precision="f32", seed=spec.seed, noise=spec.noise)
    cav.step(steps)
    wins = [(0, 0, 80, 80), (n - 80, 0, 80, 80), (0, n - 80, 80, 80), (n - 80, n - 80, 80, 80),
            (0, 2000, 80, 80), (2000, n - 80, 80, 80)]
    nfull = n * n
    for (x0, y0, w, h) in wins:
        po = O.derive(n, n, spec.Ra, spec.Da, spec.eps, spec.Pr, spec.Le, spec.N, nee=True)
        po.nx, po.ny = w, h                 # constants of the full grid, window extent
        jj, ii = np.mgrid[0:h, 0:w]
        k = (y0 + jj) * n + (x0 + ii)
        T = 0.5 + spec.noise * (2.0 * np.vectorize(lambda q: O.uniform(spec.seed, int(q)))(k) - 1.0)
        C = 0.5 + spec.noise * (2.0 * np.vectorize(lambda q: O.uniform(spec.seed, int(nfull + q)))(k) - 1.0)
        o = O.Oracle(po, seed=spec.seed, noise=spec.noise, T_init=T, C_init=C)
        o.step(steps)
        fo = o.fields()
        fg = cav.fields_window(x0, y0, w, h)
        m = np.ones((h, w), bool)
        d = steps + 2
        if x0 > 0:
            m[:, :d] = False
        if x0 + w < n:
            m[:, w - d:] = False
        if y0 > 0:
            m[:d, :] = False
        if y0 + h < n:
            m[h - d:, :] = False
        assert m.sum() > 100
        for key, tol in (("T", 1e-5), ("C", 1e-5), ("ux", 1e-4), ("uy", 1e-4)):
            a, b = fg[key][m], fo[key][m]
            if key in ("T", "C"):
                a, b = a - 0.5, b - 0.5
            err = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)
            assert err <= tol, ((x0, y0), key, err)
        # the Dirichlet walls carry their values on the wall nodes
        if x0 == 0:
            np.testing.assert_allclose(fg["T"][:, 0], 1.0, rtol=0, atol=1e-6)
        if x0 + w == n:
            np.testing.assert_allclose(fg["T"][:, -1], 0.0, rtol=0, atol=1e-6)
    cav.close()
