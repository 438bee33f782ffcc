"""Pins of the oracle's moving-wall bounce-back and top/bottom Dirichlet walls
(used by the lid-driven cavity of Sec. 4.3).

* Couette flow between a resting bottom wall and a top wall moving with U: the
  steady profile u = U y / H is reproduced exactly by halfway bounce-back, and the
  stream function (psi = 0 on the bottom wall) is its integral U y^2 / (2 H).
* Porous Couette flow (Eqs. 2, 5 with F_eps = 0): nu_e u'' - (eps nu / K) u = 0,
  u(0) = 0, u(H) = U => u = U sinh(r y) / sinh(r H), r^2 = eps nu / (K nu_e);
  second-order convergence.
* Conduction between a cold bottom and a hot top wall: T = y / H exactly and
  Nu = Sh = 1 on both walls.
"""
import numpy as np
import pytest


def couette(O, ny, U, K=1e300, eps=0.7, s_nu=1.0, steps_max=400):
    p = O.derive(4, ny, 1e4, 1e-2, eps, 1, 1, 0)
    p.periodic_x = 1
    p.gbT = p.gbC = 0.0
    p.Feps = 0.0
    p.K = K
    p.s[7] = p.s[8] = s_nu
    p.nu_e = p.nu = (1 / s_nu - 0.5) / 3.0
    p.uw[3][0] = U
    o = O.Oracle(p, seed=1, noise=0.0)
    prev = None
    for _ in range(steps_max):
        o.step(500)
        u = o.fields()["ux"][:, 0].copy()
        if prev is not None and np.abs(u - prev).max() < 1e-16:
            break
        prev = u
    fl = o.fields()
    fl["psi"] = o.stream_function()
    return p, fl


@pytest.mark.parametrize("s_nu", [0.7, 1.0, 1.6])
def test_couette_exact(oracle_mod, s_nu):
    ny, U = 16, 0.05
    p, fl = couette(oracle_mod, ny, U, s_nu=s_nu)
    y = np.arange(ny) + 0.5
    np.testing.assert_allclose(fl["ux"][:, 0], U * y / ny, rtol=0, atol=1e-13)
    assert np.abs(fl["uy"]).max() < 1e-14
    # stream function (u_x = d psi / dy, psi = 0 on the bottom wall at y = 0): the
    # integral of the linear profile, U y^2 / (2 H), exact for the trapezoid rule
    exact_psi = U * y ** 2 / (2 * ny)
    np.testing.assert_allclose(fl["psi"], np.broadcast_to(exact_psi[:, None], fl["psi"].shape),
                               rtol=0, atol=2e-12)   # ny velocity errors of <= 1e-13 summed


def test_porous_couette_closed_form(oracle_mod):
    U, errs = 0.05, []
    for ny in (16, 32, 64):
        K = 0.02 * ny * ny
        p, fl = couette(oracle_mod, ny, U, K=K, eps=0.6)
        r = np.sqrt(p.eps * p.nu / (p.K * p.nu_e))
        y = np.arange(ny) + 0.5
        exact = U * np.sinh(r * y) / np.sinh(r * ny)
        u = fl["ux"][:, 0]
        errs.append(np.linalg.norm(u - exact) / np.linalg.norm(exact))
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 1e-3 and order.min() > 1.8, (errs, order)


def test_top_bottom_conduction_exact(oracle_mod):
    O = oracle_mod
    nx, ny = 3, 8
    p = O.derive(nx, ny, 1e4, 1e-2, 0.8, 1, 1, 1, sigma=1.3)
    p.gbT = p.gbC = 0.0
    p.scalar_lr = O.ADIABATIC
    p.scalar_tb = O.DIRICHLET
    p.Tw[2], p.Tw[3] = 0.0, 1.0
    p.Cw[2], p.Cw[3] = 0.0, 1.0
    o = O.Oracle(p, seed=3, noise=0.2)
    exact = (np.arange(ny) + 0.5) / ny
    for _ in range(60):
        o.step(2000)
        fl = o.fields()
        if np.abs(fl["T"] - exact[:, None]).max() < 1e-14:
            break
    np.testing.assert_allclose(fl["T"], np.broadcast_to(exact[:, None], (ny, nx)), atol=1e-13)
    np.testing.assert_allclose(fl["C"], np.broadcast_to(exact[:, None], (ny, nx)), atol=1e-13)
    np.testing.assert_allclose(o.nusselt_sherwood_tb(), [1, 1, 1, 1], atol=1e-12)
