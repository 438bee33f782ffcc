"""Pins of the oracle's walls with nodes on them (Sec. 3.3: the non-equilibrium
extrapolation of Eqs. 33-35, the gradient extrapolation of Eqs. 36-37) and of the
convective (Robin) wall of Eq. 39.

* Conduction (no buoyancy) between Dirichlet walls: T = 1 - x / L exactly at
  steady state, L = nx - 1, with adiabatic top and bottom walls (Eq. 36 with a
  zero gradient); Nu = Sh = 1 on both walls with the node-on-wall stencil.
* Conduction against a convective wall: dtheta/dX = -Bi theta on the right wall
  (outward normal +x) gives theta = 1 - Bi / (1 + Bi) X exactly; on the left
  wall the mirror image theta = (1 + Bi X) / (1 + Bi); on the top wall with
  H != L the Biot number keeps the width L as its length scale.
* The Brinkman-Darcy channel between no-slip walls at y = 0 and y = H = ny - 1:
  second-order convergence to the closed form of Eqs. 2 and 5.
* Couette flow between a resting wall node row and a moving one: the linear
  profile u = U y / H is reproduced exactly for any viscosity (the extrapolated
  non-equilibrium part of Eq. 33 carries the wall shear; the equilibrium alone
  misses it by ~1e-3).
* Conduction between Dirichlet top and bottom wall nodes: T = C = y / H exactly,
  Nu = Sh = 1 on both walls.
* At t = 0 (interior at rest) every wall node holds the equilibrium of Eq. 20 at
  the wall's velocity and its own porosity.
* Sec. 3.2's claim on a convective cavity: at Le = 1 and equal wall data, the
  steady T and C coincide and Nu = Sh; the coupled equilibria of "model A"
  (Eqs. 30-32) break the equality.
"""
import numpy as np
import pytest


def _conduction(O, nx, ny, sigma=1.0, eps=0.8):
    p = O.derive(nx, ny, 1e4, 1e-2, eps, 1, 1, 1, sigma=sigma, nee=True)
    p.gbT = p.gbC = 0.0
    return p


def _run_to(o, exact_T, exact_C=None, chunk=2000, cap=100, tol=1e-13):
    for _ in range(cap):
        o.step(chunk)
        fl = o.fields()
        err = np.abs(fl["T"] - exact_T).max()
        if exact_C is not None:
            err = max(err, np.abs(fl["C"] - exact_C).max())
        if err < tol:
            break
    return o.fields()


@pytest.mark.parametrize("sigma,eps", [(1.0, 0.8), (0.6, 0.45), (1.7, 1.0)])
def test_nee_dirichlet_conduction_exact(oracle_mod, sigma, eps):
    O = oracle_mod
    nx, ny = 12, 9
    p = _conduction(O, nx, ny, sigma, eps)
    o = O.Oracle(p, seed=5, noise=0.05)
    L = nx - 1
    exact = np.broadcast_to(1.0 - np.arange(nx) / L, (ny, nx))
    fl = _run_to(o, exact, exact)
    np.testing.assert_allclose(fl["T"], exact, rtol=0, atol=1e-12)
    np.testing.assert_allclose(fl["C"], exact, rtol=0, atol=1e-12)
    assert np.abs(fl["ux"]).max() < 1e-15 and np.abs(fl["uy"]).max() < 1e-15
    np.testing.assert_allclose(o.nusselt_sherwood(), [1, 1, 1, 1], rtol=0, atol=1e-12)


def test_nee_wall_values_imposed_exactly(oracle_mod):
    """After every step the wall nodes carry the Dirichlet value (Eqs. 34-35: the
    non-equilibrium part sums to zero), from the first step on."""
    O = oracle_mod
    p = O.derive(14, 10, 1e4, 1e-2, 0.6, 1, 2, 1, nee=True)
    o = O.Oracle(p, seed=2, noise=0.1)
    for _ in range(3):
        fl = o.fields()
        np.testing.assert_allclose(fl["T"][:, 0], 1.0, rtol=0, atol=1e-15)
        np.testing.assert_allclose(fl["T"][:, -1], 0.0, rtol=0, atol=1e-15)
        np.testing.assert_allclose(fl["C"][:, 0], 1.0, rtol=0, atol=1e-15)
        np.testing.assert_allclose(fl["C"][:, -1], 0.0, rtol=0, atol=1e-15)
        o.step(7)


@pytest.mark.parametrize("Bi", [0.4, 2.5])
def test_convective_right_wall_exact(oracle_mod, Bi):
    """Eq. 39 on the right wall, read as the convective condition
    dtheta/dX = -Bi theta (heat leaves through the wall to the ambient theta = 0):
    theta = 1 - Bi / (1 + Bi) X, X = x / L, exactly; corners included (Eq. 36
    along the diagonal link with both walls' conditions)."""
    O = oracle_mod
    nx, ny = 13, 8
    p = _conduction(O, nx, ny, sigma=0.9, eps=0.7)
    p.BiT[1], p.BiC[1] = Bi, 2 * Bi
    o = O.Oracle(p, seed=4, noise=0.05)
    X = np.arange(nx) / (nx - 1)
    eT = np.broadcast_to(1.0 - Bi / (1 + Bi) * X, (ny, nx))
    eC = np.broadcast_to(1.0 - 2 * Bi / (1 + 2 * Bi) * X, (ny, nx))
    fl = _run_to(o, eT, eC)
    np.testing.assert_allclose(fl["T"], eT, rtol=0, atol=1e-12)
    np.testing.assert_allclose(fl["C"], eC, rtol=0, atol=1e-12)
    # Nu on the hot wall = -dtheta/dX = Bi / (1 + Bi)
    nush = o.nusselt_sherwood()
    np.testing.assert_allclose(nush[:2], [Bi / (1 + Bi), 2 * Bi / (1 + 2 * Bi)], rtol=1e-11)


def test_convective_left_wall_mirror(oracle_mod):
    """The same condition on the left wall (outward normal -x), ambient 0, hot right
    wall theta = 1: theta = (1 + Bi X) / (1 + Bi)."""
    O = oracle_mod
    nx, ny, Bi = 11, 7, 1.3
    p = _conduction(O, nx, ny)
    p.Tw[0], p.Tw[1] = 0.0, 1.0
    p.Cw[0], p.Cw[1] = 0.0, 1.0
    p.BiT[0] = p.BiC[0] = Bi
    o = O.Oracle(p, seed=4, noise=0.05)
    X = np.arange(nx) / (nx - 1)
    e = np.broadcast_to((1 + Bi * X) / (1 + Bi), (ny, nx))
    fl = _run_to(o, e, e)
    np.testing.assert_allclose(fl["T"], e, rtol=0, atol=1e-12)
    np.testing.assert_allclose(fl["C"], e, rtol=0, atol=1e-12)


def test_convective_top_wall_uses_width_as_length(oracle_mod):
    """Hot bottom wall (theta = 1), convective top wall, adiabatic sides, H != L:
    dtheta/dy = -(Bi / L) theta at y = H gives theta = 1 - s y with
    s = (Bi / L) / (1 + Bi H / L)."""
    O = oracle_mod
    nx, ny, Bi = 9, 14, 0.8
    p = _conduction(O, nx, ny)
    p.scalar_lr, p.scalar_tb = O.ADIABATIC, O.DIRICHLET
    p.Tw[2] = p.Cw[2] = 1.0
    p.Tw[3] = p.Cw[3] = 0.0
    p.BiT[3] = p.BiC[3] = Bi
    o = O.Oracle(p, seed=6, noise=0.05)
    L, H = nx - 1, ny - 1
    s = (Bi / L) / (1 + Bi * H / L)
    e = np.broadcast_to((1 - s * np.arange(ny))[:, None], (ny, nx))
    fl = _run_to(o, e, e)
    np.testing.assert_allclose(fl["T"], e, rtol=0, atol=1e-12)


def _nee_channel(O, ny, G=1e-5, eps=0.6, s_nu=1.0, Da=0.02):
    """Fully developed flow along periodic x between no-slip wall nodes at j = 0 and
    j = ny - 1 (Eq. 33 with u_w = 0)."""
    p = O.derive(5, ny, 1e4, 1e-2, eps, 1, 1, 0, nee=True)
    p.periodic_x = 1
    p.gbT = p.gbC = 0.0
    p.Gx = G
    p.s[7] = p.s[8] = s_nu
    p.nu_e = (1 / s_nu - 0.5) / 3.0
    p.nu = p.nu_e
    H = ny - 1
    p.K = Da * H * H
    p.Feps = 0.0
    o = O.Oracle(p, seed=1, noise=0.0)
    prev = None
    for _ in range(200):
        o.step(500)
        u = o.fields()["ux"][:, 0].copy()
        if prev is not None and np.abs(u - prev).max() < 1e-15 * max(np.abs(u).max(), 1e-30):
            break
        prev = u
    return p, o.fields()


def test_nee_brinkman_channel_second_order(oracle_mod):
    """nu_e u'' - (eps nu / K) u + eps G = 0, u(0) = u(H) = 0 =>
    u = (G K / nu) [1 - cosh(r (y - H/2)) / cosh(r H / 2)], r^2 = eps nu / (K nu_e),
    with the wall nodes at y = 0 and y = H."""
    O = oracle_mod
    errs = []
    for ny in (17, 33, 65):
        p, fl = _nee_channel(O, ny)
        H = ny - 1
        y = np.arange(ny, dtype=float)
        r = np.sqrt(p.eps * p.nu / (p.K * p.nu_e))
        exact = p.Gx * p.K / p.nu * (1 - np.cosh(r * (y - H / 2)) / np.cosh(r * H / 2))
        u = fl["ux"][:, 0]
        assert np.abs(fl["ux"] - u[:, None]).max() < 1e-14
        # the extrapolated wall populations do not conserve mass exactly: a small
        # wall-normal velocity remains (NEE is not a bounce-back rule)
        assert np.abs(fl["uy"]).max() < 1e-6 * np.abs(u).max()
        errs.append(np.linalg.norm(u - exact) / np.linalg.norm(exact))
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 1e-3, errs
    assert order.min() > 1.8, (errs, order)


@pytest.mark.parametrize("s_nu", [0.7, 1.0, 1.6])
def test_nee_couette_exact(oracle_mod, s_nu):
    """Wall nodes at j = 0 (at rest) and j = H = ny - 1 (moving with U, Eq. 33 with
    u_w = (U, 0)), periodic x, no medium: u = U y / H at every node."""
    O = oracle_mod
    ny, U = 16, 0.05
    p = O.derive(5, ny, 1e4, 1e-2, 0.7, 1, 1, 0, nee=True)
    p.periodic_x = 1
    p.gbT = p.gbC = 0.0
    p.Feps = 0.0
    p.K = 1e300
    p.s[7] = p.s[8] = s_nu
    p.nu_e = p.nu = (1 / s_nu - 0.5) / 3.0
    p.uw[3][0] = U
    o = O.Oracle(p, seed=1, noise=0.0)
    prev = None
    for _ in range(400):
        o.step(500)
        u = o.fields()["ux"][:, 0].copy()
        if prev is not None and np.abs(u - prev).max() < 1e-16:
            break
        prev = u
    fl = o.fields()
    y, H = np.arange(ny), ny - 1
    exact = U * y / H
    np.testing.assert_allclose(fl["ux"], np.broadcast_to(exact[:, None], fl["ux"].shape), rtol=0, atol=1e-13)
    assert np.abs(fl["uy"]).max() < 1e-14
    # stream function from the wall node (psi = 0): U y^2 / (2 H)
    psi = o.stream_function()
    np.testing.assert_allclose(psi, np.broadcast_to((U * y ** 2 / (2 * H))[:, None], psi.shape),
                               rtol=0, atol=2e-12)   # ny velocity errors of <= 1e-13 summed


EX9 = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], float)
EY9 = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], float)
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def _feq9(rho, rho0, eps, ux, uy, cs2=1.0 / 3.0):
    """Eq. 20 in velocity space."""
    eu = EX9 * ux + EY9 * uy
    u2 = ux * ux + uy * uy
    return W9 * (rho + rho0 * (eu / cs2 + eu ** 2 / (2 * eps * cs2 ** 2) - u2 / (2 * eps * cs2)))


def test_nee_initial_wall_state_is_the_wall_equilibrium(oracle_mod):
    """At t = 0 the interior is at rest (f = w_i rho0), so Eq. 33 leaves every wall node
    with f^eq(rho0, u_w) at its own porosity: the lid velocity on the top row, corners
    included (the top wall's u_w at a corner), rest elsewhere; checked against Eq. 20 in
    velocity space with a porosity that varies from node to node."""
    O = oracle_mod
    nx, ny, U = 9, 7, 0.08
    p = O.derive_lid(nx, ny, 100.0, 1e3, 1e-2, 0.6, 1.0, 2.0, 1.0, U0=U, nee=True)
    yy, xx = np.mgrid[0:ny, 0:nx]
    eps = 0.45 + 0.4 * (xx + 2 * yy) / (nx + 2 * ny)
    o = O.Oracle(p, seed=3, noise=0.0, eps_field=eps)
    f = o.get()[0]
    for j in range(ny):
        for i in range(nx):
            if 0 < i < nx - 1 and 0 < j < ny - 1:
                continue
            u = U if j == ny - 1 else 0.0
            np.testing.assert_allclose(f[:, j, i], _feq9(p.rho0, p.rho0, eps[j, i], u, 0.0),
                                       rtol=0, atol=1e-15, err_msg=f"wall node ({i}, {j})")


def test_nee_top_bottom_conduction_exact(oracle_mod):
    """Dirichlet wall nodes at the bottom (T = C = 0) and top (T = C = 1), adiabatic
    sides, no flow: T = C = y / H with H = ny - 1, and Nu = Sh = 1 on both walls with
    the node stencil and L = ny - 1."""
    O = oracle_mod
    nx, ny = 6, 11
    p = O.derive_lid(nx, ny, 10.0, 1e3, 1e-2, 0.7, 1.0, 1.5, 1.0, sigma=1.4, nee=True)
    p.gbT = p.gbC = 0.0
    p.uw[3][0] = 0.0       # the lid at rest
    o = O.Oracle(p, seed=4, noise=0.1)
    exact = np.broadcast_to((np.arange(ny) / (ny - 1))[:, None], (ny, nx))
    fl = _run_to(o, exact, exact)
    np.testing.assert_allclose(fl["T"], exact, rtol=0, atol=1e-12)
    np.testing.assert_allclose(fl["C"], exact, rtol=0, atol=1e-12)
    np.testing.assert_allclose(o.nusselt_sherwood_tb(), [1, 1, 1, 1], rtol=0, atol=1e-11)


def _steady(O, p, tol=1e-11, chunk=2000, cap=150):
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


def test_convective_cavity_decoupling_and_model_a(oracle_mod):
    """Sec. 3.2 and Table 3 on a coarse convective cavity (20 spacings, Ra = 1e4,
    Da = 1e-2, eps = 0.6, Le = 1, N = 1, Bi_T = Bi_C = 1): the paper's equilibria
    give identical steady T and C (and Nu = Sh); the coupled equilibria of
    model A, with the same effective diffusivities (Eq. 32), do not, and give
    Nu > Sh as in Table 3."""
    O = oracle_mod
    p = O.derive_convective(20, 1e4, 1e-2, 0.6, 1.0, 1.0, 1.0, 1.0, 1.0)
    o, fl = _steady(O, p)
    nush = o.nusselt_sherwood()
    assert np.abs(fl["T"] - fl["C"]).max() < 1e-9
    assert abs(nush[0] - nush[1]) < 1e-9 and abs(nush[2] - nush[3]) < 1e-9
    assert 0.55 < nush[0] < 0.7, nush          # convection above the conduction value 0.5
    pa = O.to_model_a(O.derive_convective(20, 1e4, 1e-2, 0.6, 1.0, 1.0, 1.0, 1.0, 1.0))
    oa, fa = _steady(O, pa)
    na = oa.nusselt_sherwood()
    assert np.abs(fa["T"] - fa["C"]).max() > 1e-4
    assert na[0] - na[1] > 1e-4
