"""Pins of the oracle's full time step (collision + streaming + walls) against
closed forms and invariants of the continuum model (Sec. 2, Eqs. 1-4) and of
the lattice scheme.

* conservation of mass and of sigma*T, eps*C on periodic and closed grids;
* steady linear conduction between Dirichlet walls, exact on the lattice, and
  Nu = Sh = 1 (Eq. 38);
* the Brinkman-Darcy channel (Eqs. 2 and 5, fully developed flow) in closed
  form, with second-order convergence; with the Forchheimer term, a fine-grid
  1-D boundary-value solve;
* a decaying advected sine wave of Eq. 3 / Eq. 4: decay rate alpha_e k^2 / sigma
  and phase speed u / sigma, which holds only if the source term of Eq. 27 is
  present and alpha_e does not depend on sigma (Eq. 29);
* the implicit velocity definition Eq. 17 at every node of a running cavity;
* the decoupling claim of Sec. 3.2: at Le = 1 the steady T and C coincide and
  neither depends on sigma;
* the state at t = 0 (the equilibria of Eqs. 20 and 28, or of model A's
  Eqs. 30-31, at rest) gives back the T and C it was made from through Eq. 26,
  also with a porosity that varies from node to node.
"""
import numpy as np
import pytest
from scipy.linalg import solve_banded

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], float)
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], float)
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def feq9(p, rho, ux, uy):
    eu = EX[:, None, None] * ux + EY[:, None, None] * uy
    u2 = ux * ux + uy * uy
    cs2 = 1 / 3
    return W9[:, None, None] * (rho + p.rho0 * (eu / cs2 + eu ** 2 / (2 * p.eps * cs2 ** 2)
                                                - u2 / (2 * p.eps * cs2)))


def geq5(p, cap, Phi, ux, uy):
    wt = np.array([1 - p.varpi] + [p.varpi / 4] * 4)
    eu = EX[:5, None, None] * ux + EY[:5, None, None] * uy
    out = wt[:, None, None] * Phi * (1 + eu / p.csT2)
    out[0] = cap * Phi - (1 - wt[0]) * Phi
    return out


def test_conservation_periodic(oracle_mod):
    O = oracle_mod
    p = O.derive(12, 10, 1e5, 1e-2, 0.5, 1, 3, 2, sigma=1.5)
    p.periodic_x = p.periodic_y = 1
    p.gbT *= 100  # vigorous flow from the large initial noise
    o = O.Oracle(p, seed=3, noise=0.2)
    f0, g0, h0, _ = o.get()
    o.step(1000)
    f1, g1, h1, _ = o.get()
    fl = o.fields()
    assert np.abs(fl["ux"]).max() > 1e-4, "flow should develop"
    for a, b in ((f0, f1), (g0, g1), (h0, h1)):
        assert abs(a.sum() - b.sum()) <= 1e-13 * abs(a.sum())


def test_conservation_closed_adiabatic_cavity(oracle_mod):
    O = oracle_mod
    p = O.derive(9, 7, 1e5, 1e-1, 0.7, 1, 2, -1.5, sigma=0.8)
    p.scalar_lr = O.ADIABATIC
    p.gbT *= 100
    o = O.Oracle(p, seed=4, noise=0.2)
    f0, g0, h0, _ = o.get()
    o.step(1000)
    f1, g1, h1, _ = o.get()
    assert np.abs(o.fields()["uy"]).max() > 1e-4
    for a, b in ((f0, f1), (g0, g1), (h0, h1)):
        assert abs(a.sum() - b.sum()) <= 1e-13 * abs(a.sum())


@pytest.mark.parametrize("zeta_a", [0.3, 1.0, 1.7])
@pytest.mark.parametrize("cap", [0.5, 1.0, 2.0])
def test_linear_conduction_exact(oracle_mod, zeta_a, cap):
    """No buoyancy, Dirichlet left/right, adiabatic top/bottom: the steady
    profile of Eq. 3 is T = 1 - x/L, sampled at x = i + 1/2, and the halfway
    anti-bounce-back reproduces it exactly; so Nu = 1 on both walls."""
    O = oracle_mod
    nx, ny = 8, 3
    p = O.derive(nx, ny, 1e4, 1e-2, min(cap, 1.0), 1, 1, 1, sigma=cap)
    p.gbT = p.gbC = 0.0
    for k in (1, 2):
        p.zeta[k] = zeta_a
        p.eta[k] = 2.0 - zeta_a
    o = O.Oracle(p, seed=9, noise=0.3)
    for _ in range(40):
        o.step(2000)
        fl = o.fields()
        exact = 1.0 - (np.arange(nx) + 0.5) / nx
        if (np.abs(fl["T"] - exact).max() < 1e-14 and np.abs(fl["C"] - exact).max() < 1e-14):
            break
    np.testing.assert_allclose(fl["T"], np.broadcast_to(exact, (ny, nx)), rtol=0, atol=1e-13)
    np.testing.assert_allclose(fl["C"], np.broadcast_to(exact, (ny, nx)), rtol=0, atol=1e-13)
    np.testing.assert_allclose(o.nusselt_sherwood(), [1, 1, 1, 1], rtol=0, atol=1e-12)
    assert np.abs(fl["ux"]).max() < 1e-15


def test_linear_conduction_with_distinct_wall_values(oracle_mod):
    """T and C with different Dirichlet values (T: 1 | 0, C: 0.2 | 0.9): each is linear
    between its own wall values, exactly."""
    O = oracle_mod
    nx, ny = 8, 3
    p = O.derive(nx, ny, 1e4, 1e-2, 0.6, 1, 1.5, 1, sigma=1.4)
    p.gbT = p.gbC = 0.0
    for k in (1, 2):
        p.zeta[k], p.eta[k] = 1.0, 0.8
    p.Cw[0], p.Cw[1] = 0.2, 0.9
    o = O.Oracle(p, seed=9, noise=0.3)
    x = (np.arange(nx) + 0.5) / nx
    eT, eC = 1.0 - x, 0.2 + 0.7 * x
    for _ in range(40):
        o.step(2000)
        fl = o.fields()
        if np.abs(fl["T"] - eT).max() < 1e-14 and np.abs(fl["C"] - eC).max() < 1e-14:
            break
    np.testing.assert_allclose(fl["T"], np.broadcast_to(eT, (ny, nx)), rtol=0, atol=1e-13)
    np.testing.assert_allclose(fl["C"], np.broadcast_to(eC, (ny, nx)), rtol=0, atol=1e-13)


def _channel(O, ny, Feps, G=1e-5, eps=0.6, s_nu=1.0, Da=0.02, steps=None):
    """Fully developed flow along periodic x between no-slip walls at y = 0, H."""
    p = O.derive(4, ny, 1e4, 1e-2, eps, 1, 1, 0)
    p.periodic_x = 1
    p.gbT = p.gbC = 0.0
    p.Gx = G
    p.s[7] = p.s[8] = s_nu
    p.nu_e = (1 / s_nu - 0.5) / 3.0
    p.nu = p.nu_e
    p.K = Da * ny * ny
    p.Feps = Feps
    o = O.Oracle(p, seed=1, noise=0.0)
    prev = None
    for _ in range(200):
        o.step(500)
        u = o.fields()["ux"][:, 0].copy()
        if prev is not None and np.abs(u - prev).max() < 1e-15 * max(np.abs(u).max(), 1e-30):
            break
        prev = u
    return p, o.fields()


def test_brinkman_darcy_channel_closed_form(oracle_mod):
    """Eq. 2 with Eq. 5 (F_eps = 0): nu_e u'' - eps nu/K u + eps G = 0, u(0)=u(H)=0
    => u = (G K / nu) [1 - cosh(r (y - H/2)) / cosh(r H / 2)], r^2 = eps nu / (K nu_e)."""
    O = oracle_mod
    errs = []
    for ny in (16, 32, 64):
        p, fl = _channel(O, ny, 0.0)
        y = np.arange(ny) + 0.5
        H = ny
        r = np.sqrt(p.eps * p.nu / (p.K * p.nu_e))
        exact = p.Gx * p.K / p.nu * (1 - np.cosh(r * (y - H / 2)) / np.cosh(r * H / 2))
        u = fl["ux"][:, 0]
        assert np.abs(fl["ux"] - u[:, None]).max() < 1e-14
        assert np.abs(fl["uy"]).max() < 1e-14
        errs.append(np.linalg.norm(u - exact) / np.linalg.norm(exact))
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 1e-3, errs
    assert order.min() > 1.8, (errs, order)


def test_forchheimer_channel_against_bvp(oracle_mod):
    """With the Forchheimer term: nu_e u'' - eps nu/K u - eps F/sqrt(K) u^2 + eps G = 0,
    solved on a fine grid by Newton's method (second-order FD, 4001 points)."""
    O = oracle_mod
    ny = 64
    Feps = 1.75 / np.sqrt(150 * 0.6 ** 3)
    p, fl = _channel(O, ny, Feps, G=4e-4)
    H = ny
    n = 4001
    yy = np.linspace(0, H, n)
    dy = yy[1] - yy[0]
    a = p.eps * p.nu / p.K
    b = p.eps * p.Feps / np.sqrt(p.K)
    c = p.eps * p.Gx
    u = np.zeros(n)
    for _ in range(50):
        ui = u[1:-1]
        lap = (u[2:] - 2 * ui + u[:-2]) / dy ** 2
        R = p.nu_e * lap - a * ui - b * np.abs(ui) * ui + c
        main = -2 * p.nu_e / dy ** 2 - a - 2 * b * np.abs(ui)
        off = np.full(n - 2, p.nu_e / dy ** 2)
        off[0] = off[-1] = 0.0
        du = solve_banded((1, 1), np.vstack([off, main, off]), -R)
        u[1:-1] += du
        if np.abs(du).max() < 1e-18:
            break
    uref = np.interp(np.arange(ny) + 0.5, yy, u)
    ulb = fl["ux"][:, 0]
    rel = np.linalg.norm(ulb - uref) / np.linalg.norm(uref)
    assert b * uref.max() > 0.2 * a, "Forchheimer term should matter in this case"
    assert rel < 2e-3, rel


@pytest.mark.parametrize("cap", [0.5, 1.0, 2.0])
def test_advected_wave_decay_and_speed(oracle_mod, cap):
    """Eq. 3 with uniform u: T = T0 + A exp(-alpha_e k^2 t / sigma) sin(k (x - u t / sigma)).
    alpha_e = c_sT^2 (1/zeta_a - 1/2) (Eq. 29) independently of sigma; without the source
    term of Eq. 27 the decay would be off by (1/zeta_a - 1/2) u^2 / sigma (~10-20 %)."""
    O = oracle_mod
    nx, ny = 128, 3
    p = O.derive(nx, ny, 1e4, 1e-2, 0.6, 1, 1, 0, sigma=cap)
    p.periodic_x = p.periodic_y = 1
    p.gbT = p.gbC = 0.0
    p.K = 1e300
    ux0 = 0.1
    za = 1.0
    for k in (1, 2):
        p.zeta[k] = za
        p.eta[k] = za
    alpha = p.csT2 * (1 / za - 0.5)
    x = np.arange(nx) + 0.5
    kw = 2 * np.pi / nx
    A = 0.1
    T0f = np.broadcast_to(0.5 + A * np.sin(kw * x), (ny, nx)).copy()
    o = O.Oracle(p, seed=1, noise=0.0, T_init=T0f, C_init=T0f)
    ux = np.full((ny, nx), ux0)
    uy = np.zeros((ny, nx))
    f = feq9(p, np.ones((ny, nx)), ux, uy)
    g = geq5(p, p.sigma, T0f, ux, uy)
    h = geq5(p, p.eps, T0f, ux, uy)
    hist = np.stack([T0f * ux, T0f * uy, T0f * ux, T0f * uy])
    o.set(f, g, h, hist)
    nsteps = 600
    o.step(nsteps)
    fl = o.fields()
    for key, capk in (("T", cap), ("C", p.eps)):
        row = fl[key][0] - 0.5
        c = (row * np.exp(-1j * kw * x)).sum() * 2 / nx   # = A(t) (-i) exp(-i k shift)
        amp = np.abs(c)
        shift = -np.angle(c * 1j) / kw
        amp_exact = A * np.exp(-alpha * kw ** 2 * nsteps / capk)
        shift_exact = ux0 * nsteps / capk
        assert abs(amp / amp_exact - 1) < 2e-3, (key, amp, amp_exact)
        dshift = (shift - shift_exact + nx / 2) % nx - nx / 2   # phase is known modulo nx
        assert abs(dshift) < 1e-2 * shift_exact, (key, shift, shift_exact)


def test_velocity_closed_form_satisfies_eq17(oracle_mod):
    """At every node of a running porous cavity, u from Eq. 18 satisfies
    rho0 u = sum e f + (1/2) rho0 F(u) (Eq. 17) with F from Eq. 5."""
    O = oracle_mod
    p = O.derive(16, 12, 1e5, 1e-3, 0.4, 1, 5, -1)
    p.gbT *= 20
    o = O.Oracle(p, seed=2, noise=0.05)
    o.step(300)
    f, g, h, _ = o.get()
    fl = o.fields()
    ux, uy, T, C = fl["ux"], fl["uy"], fl["T"], fl["C"]
    assert np.abs(ux).max() > 1e-5
    jx = np.tensordot(EX, f, 1)
    jy = np.tensordot(EY, f, 1)
    Gy = p.gbT * (T - p.T0) + p.gbC * (C - p.C0)
    um = np.hypot(ux, uy)
    Fx = -p.eps * p.nu / p.K * ux - p.eps * p.Feps / np.sqrt(p.K) * um * ux
    Fy = -p.eps * p.nu / p.K * uy - p.eps * p.Feps / np.sqrt(p.K) * um * uy + p.eps * Gy
    assert np.abs(p.rho0 * ux - jx - 0.5 * p.rho0 * Fx).max() < 1e-15
    assert np.abs(p.rho0 * uy - jy - 0.5 * p.rho0 * Fy).max() < 1e-15


def _steady(O, p, tol=1e-11, chunk=2000, cap=200):
    o = O.Oracle(p, seed=1, noise=1e-3)
    prev = None
    for _ in range(cap):
        o.step(chunk)
        fl = o.fields()
        if prev is not None:
            r = max(np.abs(fl[k] - prev[k]).max() / np.abs(fl[k]).max() for k in ("ux", "uy", "T", "C"))
            if r < tol:
                break
        prev = fl
    return o, fl


def test_decoupling_steady_state_independent_of_sigma(oracle_mod):
    """Sec. 3.2: with the modified equilibria (Eqs. 24-25, 29) sigma and eps
    only affect the transient.  At Le = 1 with the same wall data the steady T
    and C coincide, Nu = Sh, and sigma = 0.5, 1, 2 give the same steady T."""
    O = oracle_mod
    res = {}
    for sigma in (0.5, 1.0, 2.0):
        p = O.derive(12, 12, 2e3, 1e-1, 0.6, 1, 1, 1, sigma=sigma)
        o, fl = _steady(O, p)
        nush = o.nusselt_sherwood()
        assert np.abs(fl["T"] - fl["C"]).max() < 1e-8
        assert abs(nush[0] - nush[1]) < 1e-8 and abs(nush[2] - nush[3]) < 1e-8
        res[sigma] = fl["T"]
        assert nush[0] > 1.05, "convection should raise Nu above conduction"
    assert np.abs(res[0.5] - res[1.0]).max() < 1e-8
    assert np.abs(res[2.0] - res[1.0]).max() < 1e-8


@pytest.mark.parametrize("model_a", [False, True])
@pytest.mark.parametrize("field", [False, True])
def test_initial_state_holds_the_given_fields(oracle_mod, model_a, field):
    O = oracle_mod
    nx, ny = 11, 8
    p = O.derive(nx, ny, 1e4, 1e-2, 0.55, 1.0, 2.0, 1.0, sigma=1.6)
    if model_a:
        O.to_model_a(p)
    rng = np.random.default_rng(3)
    T0, C0 = rng.uniform(0, 1, (ny, nx)), rng.uniform(0, 1, (ny, nx))
    eps = rng.uniform(0.4, 0.9, (ny, nx)) if field else None
    o = O.Oracle(p, seed=1, noise=0.0, T_init=T0, C_init=C0, eps_field=eps)
    fl = o.fields()
    np.testing.assert_allclose(fl["T"], T0, rtol=0, atol=1e-15)
    np.testing.assert_allclose(fl["C"], C0, rtol=0, atol=1e-15)


@pytest.mark.parametrize("model_a", [False, True])
def test_scalar_content_changes_by_the_wall_link_fluxes(oracle_mod, model_a):
    """Over one step the total sum g (= sum sigma T) changes only by what the D2Q5 links
    carry through the walls: the collision conserves it (the source term of Eq. 27 has
    no zeroth moment), streaming moves it, bounce-back on the adiabatic walls returns
    it.  Through a Dirichlet wall, anti-bounce-back gives the entering population
    g_in = -g*_out + 2 k w~ Phi_w (k = 1; model A: the capacity), so the net inflow of
    a link is 2 g_in - 2 k w~ Phi_w, read from the state after the step.  Same for h."""
    O = oracle_mod
    nx, ny = 12, 9
    p = O.derive(nx, ny, 5e4, 1e-2, 0.6, 1.0, 2.0, -0.5, sigma=1.3)
    p.Cw[0], p.Cw[1] = 0.9, 0.15
    if model_a:
        O.to_model_a(p)
    o = O.Oracle(p, seed=4, noise=0.05)
    o.step(60)
    _, g0, h0, _ = o.get()
    o.step(1)
    _, g1, h1, _ = o.get()
    wt = p.varpi / 4
    for a0, a1, W, cap in ((g0, g1, p.Tw, p.sigma), (h0, h1, p.Cw, p.eps)):
        k = cap if model_a else 1.0
        inflow = (2 * a1[1, :, 0] - 2 * k * wt * W[0]).sum() + (2 * a1[3, :, nx - 1] - 2 * k * wt * W[1]).sum()
        change = a1.sum() - a0.sum()
        assert abs(inflow) > 1e-6                       # the walls do carry something
        assert abs(change - inflow) <= 1e-13 * abs(a1.sum()), (change, inflow)
