"""Spatially varying porosity and permeability (the REV model applied per node):
pins of the oracle.

* A uniform field reproduces the scalar-parameter run bit for bit.
* Fully developed channel flow through a medium whose eps(y) and K(y) vary
  smoothly across the channel: nu_e u'' - eps nu / K u - eps F_eps(eps) / sqrt(K) u^2
  + eps G = 0 (Eqs. 2, 5, 7 for u = u(y)), solved by Newton's method on a fine grid;
  the lattice solution converges to it at second order.
"""
import numpy as np
from scipy.linalg import solve_banded


def test_uniform_field_equals_scalar(oracle_mod):
    O = oracle_mod
    p = O.derive(17, 13, 3e4, 1e-2, 0.55, 1, 2, -1.5, sigma=1.2)
    a = O.Oracle(p, seed=8, noise=0.02)
    b = O.Oracle(p, seed=8, noise=0.02, eps_field=np.full((13, 17), 0.55),
                 K_field=np.full((13, 17), p.K))
    a.step(400)
    b.step(400)
    fa, fb = a.fields(), b.fields()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k


def eps_of(y, H):
    return 0.6 + 0.2 * np.cos(np.pi * y / H)


def K_of(y, H):
    return 0.02 * H * H * (1.0 + 0.5 * np.sin(2 * np.pi * y / H))


def lattice_channel(O, ny, G=2e-4):
    p = O.derive(4, ny, 1e4, 1e-2, 0.6, 1, 1, 0)
    p.periodic_x = 1
    p.gbT = p.gbC = 0.0
    p.Gx = G
    p.s[7] = p.s[8] = 1.0
    p.nu_e = p.nu = (1.0 - 0.5) / 3.0
    y = np.arange(ny) + 0.5
    eps = np.repeat(eps_of(y, ny)[:, None], 4, axis=1)
    K = np.repeat(K_of(y, ny)[:, None], 4, axis=1)
    o = O.Oracle(p, seed=1, noise=0.0, eps_field=eps, K_field=K)
    prev = None
    for _ in range(400):
        o.step(500)
        u = o.fields()["ux"][:, 0].copy()
        if prev is not None and np.abs(u - prev).max() < 1e-15 * np.abs(u).max():
            break
        prev = u
    return p, o.fields()


def bvp(p, H, G, n=8001):
    yy = np.linspace(0, H, n)
    dy = yy[1] - yy[0]
    e, K = eps_of(yy[1:-1], H), K_of(yy[1:-1], H)
    Fe = 1.75 / np.sqrt(150 * e ** 3)
    a = e * p.nu / K
    b = e * Fe / np.sqrt(K)
    c = e * G
    u = np.zeros(n)
    for _ in range(60):
        ui = u[1:-1]
        R = p.nu_e * (u[2:] - 2 * ui + u[:-2]) / dy ** 2 - a * ui - b * np.abs(ui) * ui + c
        main = -2 * p.nu_e / dy ** 2 - a - 2 * b * np.abs(ui)
        off = np.full(n - 2, p.nu_e / dy ** 2)
        off[0] = off[-1] = 0.0
        du = solve_banded((1, 1), np.vstack([off, main, off]), -R)
        u[1:-1] += du
        if np.abs(du).max() < 1e-18:
            break
    return yy, u


def test_varying_medium_channel_converges_to_bvp(oracle_mod):
    O = oracle_mod
    errs = []
    for ny in (16, 32, 64):
        p, fl = lattice_channel(O, ny)
        yy, u = bvp(p, ny, p.Gx)
        ref = np.interp(np.arange(ny) + 0.5, yy, u)
        errs.append(np.linalg.norm(fl["ux"][:, 0] - ref) / np.linalg.norm(ref))
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 2e-3 and order.min() > 1.7, (errs, order)
