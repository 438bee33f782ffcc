"""Pins of the oracle's single-node collision against independent forms.

The oracle collides in moment space (Eq. 10 with Eqs. 12-15; Eqs. 21-25 and
27) and gets the velocity from the closed form (Eqs. 18-19).  These tests
recompute the same post-collision state another way:

* velocity space, Eq. 9, with the collision matrix M^-1 Lambda M built here by
  numpy, the velocity-space equilibrium of Eq. 20, and the velocity-space
  forcing term of the Guo-type scheme the paper cites for Eq. 15
  (S~_i = w_i rho0 [e.F/cs^2 + (e.u)(e.F)/(eps cs^4) - u.F/(eps cs^2)]);
* the velocity from the implicit definition Eq. 17, solved by Newton's
  method instead of the closed form;
* for D2Q5, Eq. 21 in velocity space with the velocity-space equilibria of
  Eq. 28 instead of the modified moments of Eqs. 24-25.

A dropped term, a wrong sign, a wrong relaxation index or a transposed
matrix in the oracle shows up as a mismatch here.
"""
import numpy as np
import pytest

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], float)
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], float)
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
CS2 = 1.0 / 3.0

# Eq. 13 (Lallemand-Luo ordering), Eq. 23
M = np.array([
    [1, 1, 1, 1, 1, 1, 1, 1, 1],
    [-4, -1, -1, -1, -1, 2, 2, 2, 2],
    [4, -2, -2, -2, -2, 1, 1, 1, 1],
    [0, 1, 0, -1, 0, 1, -1, -1, 1],
    [0, -2, 0, 2, 0, 1, -1, -1, 1],
    [0, 0, 1, 0, -1, 1, 1, -1, -1],
    [0, 0, -2, 0, 2, 1, 1, -1, -1],
    [0, 1, -1, 1, -1, 0, 0, 0, 0],
    [0, 0, 0, 0, 0, 1, -1, 1, -1]], float)
NM = np.array([
    [1, 1, 1, 1, 1],
    [0, 1, 0, -1, 0],
    [0, 0, 1, 0, -1],
    [-4, 1, 1, 1, 1],
    [0, 1, -1, 1, -1]], float)


def force(p, ux, uy, T, C):
    """Eq. 5 with Eq. 6 (G along y plus the test-only constant Gx)."""
    Gy = p.gbT * (T - p.T0) + p.gbC * (C - p.C0)
    Gx = p.Gx
    um = np.hypot(ux, uy)
    Fx = -p.eps * p.nu / p.K * ux - p.eps * p.Feps / np.sqrt(p.K) * um * ux + p.eps * Gx
    Fy = -p.eps * p.nu / p.K * uy - p.eps * p.Feps / np.sqrt(p.K) * um * uy + p.eps * Gy
    return Fx, Fy


def velocity_newton(p, f, T, C):
    """Solve Eq. 17, rho0 u = sum e f + (1/2) rho0 F(u), by Newton iteration."""
    jx, jy = EX @ f, EY @ f
    u = np.array([jx, jy]) / p.rho0

    def res(u):
        Fx, Fy = force(p, u[0], u[1], T, C)
        return p.rho0 * u - np.array([jx, jy]) - 0.5 * p.rho0 * np.array([Fx, Fy])

    for _ in range(60):
        r = res(u)
        Jm = np.zeros((2, 2))
        hstep = 1e-7
        for k in range(2):
            du = np.zeros(2)
            du[k] = hstep
            Jm[:, k] = (res(u + du) - res(u - du)) / (2 * hstep)
        u = u - np.linalg.solve(Jm, r)
        if np.max(np.abs(res(u))) < 1e-17:
            break
    return u


def feq9(p, rho, ux, uy):
    """Eq. 20."""
    eu = EX * ux + EY * uy
    u2 = ux * ux + uy * uy
    return W9 * (rho + p.rho0 * (eu / CS2 + eu ** 2 / (2 * p.eps * CS2 ** 2) - u2 / (2 * p.eps * CS2)))


def guo_force(p, ux, uy, Fx, Fy):
    eu = EX * ux + EY * uy
    eF = EX * Fx + EY * Fy
    uF = ux * Fx + uy * Fy
    return W9 * p.rho0 * (eF / CS2 + eu * eF / (p.eps * CS2 ** 2) - uF / (p.eps * CS2))


def geq5(p, cap, Phi, ux, uy):
    """Eq. 28 (cap = sigma for T, eps for C)."""
    wt = np.array([1 - p.varpi] + [p.varpi / 4] * 4)
    out = wt * Phi * (1 + (EX[:5] * ux + EY[:5] * uy) / p.csT2)
    out[0] = cap * Phi - (1 - wt[0]) * Phi
    return out


def velocity_space_collision(p, f, g, h, hist):
    rho = f.sum()
    T = g.sum() / p.sigma
    C = h.sum() / p.eps
    ux, uy = velocity_newton(p, f, T, C)
    Fx, Fy = force(p, ux, uy, T, C)
    Lam = np.diag(np.array(p.s[:]))
    Lt = np.linalg.inv(M) @ Lam @ M               # collision matrix of Eq. 9
    St = guo_force(p, ux, uy, Fx, Fy)
    fs = f - Lt @ (f - feq9(p, rho, ux, uy)) + St - 0.5 * Lt @ St   # Eq. 9
    wt = np.array([1 - p.varpi] + [p.varpi / 4] * 4)
    Ni = np.linalg.inv(NM)
    out = []
    for d, cap, Phi, rates, hx, hy in ((g, p.sigma, T, p.zeta, hist[0], hist[1]),
                                        (h, p.eps, C, p.eta, hist[2], hist[3])):
        Th = np.diag(np.array(rates[:]))
        X = (Phi * ux - hx, Phi * uy - hy)
        Sv = wt * (EX[:5] * X[0] + EY[:5] * X[1]) / p.csT2        # Eq. 27
        ds = d - Ni @ Th @ NM @ (d - geq5(p, cap, Phi, ux, uy)) \
            + Ni @ (np.eye(5) - Th / 2) @ NM @ Sv
        out.append(ds)
    return fs, out[0], out[1], (ux, uy, T, C, Fx, Fy)


def random_params(O, rng, Feps=True):
    p = O.derive(64, 64, Ra=10 ** rng.uniform(3, 5), Da=10 ** rng.uniform(-4, -1),
                 eps=rng.uniform(0.3, 1.0), Pr=rng.uniform(0.5, 2), Le=rng.uniform(0.5, 10),
                 N=rng.uniform(-5, 5), sigma=rng.uniform(0.5, 2))
    # strengthen the nonlinear force terms so that they matter at this tolerance
    p.gbT *= 50
    p.gbC *= 50
    p.K = rng.uniform(2, 20)
    if not Feps:
        p.Feps = 0.0
    p.Gx = rng.uniform(-1e-3, 1e-3)
    return p


def random_node(p, rng):
    ux, uy = rng.uniform(-0.08, 0.08, 2)
    f = feq9(p, 1 + rng.uniform(-0.01, 0.01), ux, uy) * (1 + rng.uniform(-0.05, 0.05, 9))
    T = rng.uniform(0, 1)
    C = rng.uniform(0, 1)
    g = geq5(p, p.sigma, T, ux, uy) + rng.uniform(-0.01, 0.01, 5)
    h = geq5(p, p.eps, C, ux, uy) + rng.uniform(-0.01, 0.01, 5)
    hist = rng.uniform(-0.05, 0.05, 4)
    return f, g, h, hist


@pytest.mark.parametrize("seed", range(12))
def test_moment_space_equals_velocity_space(oracle_mod, seed):
    O = oracle_mod
    rng = np.random.default_rng(seed)
    p = random_params(O, rng, Feps=(seed % 3 != 0))
    f, g, h, hist = random_node(p, rng)
    fs, gs, hs, hist_new, mac = O.collide_node(p, f, g, h, hist)
    fs_v, gs_v, hs_v, (ux, uy, T, C, Fx, Fy) = velocity_space_collision(p, f, g, h, hist)
    assert abs(mac["ux"] - ux) < 1e-15 and abs(mac["uy"] - uy) < 1e-15
    assert abs(mac["Fx"] - Fx) < 1e-15 and abs(mac["Fy"] - Fy) < 1e-15
    np.testing.assert_allclose(fs, fs_v, rtol=0, atol=2e-15)
    np.testing.assert_allclose(gs, gs_v, rtol=0, atol=2e-15)
    np.testing.assert_allclose(hs, hs_v, rtol=0, atol=2e-15)
    # history becomes (T u, C u) of this collision (explicit d(Tu)/dt, Sec. 3.2)
    np.testing.assert_allclose(hist_new, [T * ux, T * uy, C * ux, C * uy], rtol=0, atol=1e-16)


def test_collision_conserves_mass_and_scalars(oracle_mod):
    """Eq. 10 leaves rho unchanged (S_0 = 0, m_eq,0 = rho); Eqs. 21-22 leave
    sum g = sigma T and sum h = eps C unchanged (zeroth source moment is 0)."""
    O = oracle_mod
    rng = np.random.default_rng(99)
    for _ in range(20):
        p = random_params(O, rng)
        f, g, h, hist = random_node(p, rng)
        fs, gs, hs, _, _ = O.collide_node(p, f, g, h, hist)
        assert abs(fs.sum() - f.sum()) < 1e-15
        assert abs(gs.sum() - g.sum()) < 1e-15
        assert abs(hs.sum() - h.sum()) < 1e-15


def test_equilibrium_is_fixed_point(oracle_mod):
    """At F = 0 and d(Tu)/dt = 0 the equilibria of Eqs. 20 and 28 do not change
    under collision (m = m_eq, n = n_eq)."""
    O = oracle_mod
    rng = np.random.default_rng(5)
    p = O.derive(32, 32, 1e4, 1e-2, 0.6, 1, 2, 1)
    p.gbT = p.gbC = 0.0
    p.K = 1e300
    for _ in range(10):
        ux, uy = rng.uniform(-0.1, 0.1, 2)
        T, C = rng.uniform(0, 1, 2)
        f = feq9(p, 1.003, ux, uy)
        g = geq5(p, p.sigma, T, ux, uy)
        h = geq5(p, p.eps, C, ux, uy)
        hist = np.array([T * ux, T * uy, C * ux, C * uy])
        fs, gs, hs, _, mac = O.collide_node(p, f, g, h, hist)
        np.testing.assert_allclose(fs, f, atol=1e-16)
        np.testing.assert_allclose(gs, g, atol=1e-16)
        np.testing.assert_allclose(hs, h, atol=1e-16)


def test_splitmix64_definition(oracle_mod):
    """SplitMix64 (Steele, Lea & Flood 2014): the k-th output is the mix of
    seed + (k+1) * 0x9E3779B97F4A7C15; checked here by an independent Python
    implementation of the published stepping form (state advanced in a loop)."""
    O = oracle_mod
    mask = (1 << 64) - 1

    def seq(seed, n):
        x = seed
        out = []
        for _ in range(n):
            x = (x + 0x9E3779B97F4A7C15) & mask
            z = x
            z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
            z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
            out.append(z ^ (z >> 31))
        return out

    for seed in (0, 1, 12345, 2 ** 63 + 7):
        vals = seq(seed, 40)
        for k in (0, 1, 17, 39):
            assert O.uniform(seed, k) == (vals[k] >> 11) * 2.0 ** -53

    # the initial state (reading r8): T = T0 + a (2 u - 1), C = C0 + a (2 u' - 1) with u
    # the output at key j nx + i and u' at key (ny + j) nx + i
    nx, ny, a, seed = 5, 4, 0.03, 77
    p = O.derive(nx, ny, 1e4, 1e-2, 0.7, 1.0, 2.0, 1.0, sigma=1.3)
    fl = O.Oracle(p, seed=seed, noise=a).fields()
    u = np.array([(v >> 11) * 2.0 ** -53 for v in seq(seed, 2 * nx * ny)]).reshape(2, ny, nx)
    np.testing.assert_allclose(fl["T"], p.T0 + a * (2 * u[0] - 1), rtol=0, atol=1e-15)
    np.testing.assert_allclose(fl["C"], p.C0 + a * (2 * u[1] - 1), rtol=0, atol=1e-15)
    # a window of a larger cavity takes the whole cavity's keys
    T, Cw = O.noise_window(seed, a, nx, ny, 1, 2, 3, 2)
    np.testing.assert_array_equal(T, p.T0 + a * (2 * u[0][2:4, 1:4] - 1))
    np.testing.assert_array_equal(Cw, p.C0 + a * (2 * u[1][2:4, 1:4] - 1))
