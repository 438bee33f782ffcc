"""Pins of the oracle's parameter mapping (the dimensionless groups defined with the
governing equations, Sec. 2; the lattice choices of Sec. 4 / 4.1; Eq. 29).

The lattice quantities the mapping produces are put back into the definitions of the
groups, which must give back the inputs:
  Ra = g beta_T dT L^3 / (nu alpha_e), Pr = nu / alpha_e, Le = alpha_e / D_e,
  Da = K / L^2, J = nu_e / nu, N = beta_C dC / (beta_T dT), Ma = U / c_s with
  U = sqrt(g beta_T dT L); the lid-driven cavity's Re = L U0 / nu and
  Gr = g beta_T dT L^3 / nu^2 (Sec. 4.3).
The relaxation rates are checked through the transport coefficients they give:
nu_e = c_s^2 (1/s_nu - 1/2) and Eq. 29's alpha_e = c_sT^2 (1/zeta_a - 1/2),
D_e = c_sT^2 (1/eta_D - 1/2), with c_s^2 and c_sT^2 the second moments of the D2Q9
and D2Q5 weights, computed here from the weights.  This runs the mapping backwards,
so a slip in its forward algebra (a dropped J, Pr for sqrt(Pr), the wrong length
scale L) fails.
"""
import numpy as np
import pytest

D2Q9_W = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4
D2Q9_EX = [0, 1, 0, -1, 0, 1, -1, -1, 1]
D2Q5_EX = [0, 1, 0, -1, 0]


def _cs2():
    return sum(w * e * e for w, e in zip(D2Q9_W, D2Q9_EX))


def _csT2(varpi):
    w = [1 - varpi] + [varpi / 4] * 4
    return sum(wi * e * e for wi, e in zip(w, D2Q5_EX))


def _draws(seed, n):
    rng = np.random.default_rng(seed)
    for _ in range(n):
        yield dict(nx=int(rng.integers(8, 300)), ny=int(rng.integers(8, 300)),
                   Ra=10 ** rng.uniform(3, 7), Da=10 ** rng.uniform(-5, 2), eps=rng.uniform(0.2, 1.0),
                   Pr=rng.uniform(0.5, 10), Le=rng.uniform(0.5, 10), N=rng.uniform(-5, 5),
                   J=rng.uniform(0.5, 2), sigma=rng.uniform(0.5, 2), Ma=rng.uniform(0.05, 0.2),
                   varpi=rng.uniform(0.2, 0.6))


def _close(a, b, what):
    assert abs(a - b) <= 1e-12 * abs(b), (what, a, b)


def _check_common(p, d, L):
    cs2, csT2 = _cs2(), _csT2(d["varpi"])
    _close(p.cs2, cs2, "c_s^2")
    _close(p.csT2, csT2, "c_sT^2")
    _close(p.nu / p.alpha_e, d["Pr"], "Pr")
    _close(p.alpha_e / p.D_e, d["Le"], "Le")
    _close(p.K / L ** 2, d["Da"], "Da")
    _close(p.nu_e / p.nu, d["J"], "J")
    _close(p.gbC / p.gbT, d["N"], "N")
    for k in (7, 8):
        _close(cs2 * (1 / p.s[k] - 0.5), p.nu_e, "nu_e from s_nu")
    for k in (1, 2):
        _close(csT2 * (1 / p.zeta[k] - 0.5), p.alpha_e, "alpha_e from zeta_a (Eq. 29)")
        _close(csT2 * (1 / p.eta[k] - 0.5), p.D_e, "D_e from eta_D (Eq. 29)")


@pytest.mark.parametrize("nee", [False, True])
def test_mapping_returns_the_dimensionless_groups(oracle_mod, nee):
    O = oracle_mod
    checked = 0
    for d in _draws(7 + nee, 60):
        try:
            p = O.derive(d["nx"], d["ny"], d["Ra"], d["Da"], d["eps"], d["Pr"], d["Le"], d["N"],
                         d["J"], d["sigma"], d["Ma"], d["varpi"], nee=nee)
        except ValueError:      # a relaxation rate outside (0, 2): rejected, not mapped
            continue
        L = d["nx"] - 1 if nee else d["nx"]
        _check_common(p, d, L)
        _close(p.gbT * L ** 3 / (p.nu * p.alpha_e), d["Ra"], "Ra")
        _close(np.sqrt(p.gbT * L) / np.sqrt(p.cs2), d["Ma"], "Ma")
        checked += 1
    assert checked >= 20, checked


@pytest.mark.parametrize("nee", [False, True])
def test_lid_mapping_returns_re_and_gr(oracle_mod, nee):
    O = oracle_mod
    rng = np.random.default_rng(11 + nee)
    checked = 0
    for d in _draws(21 + nee, 40):
        Re, Gr, U0 = 10 ** rng.uniform(1, 3), 10 ** rng.uniform(2, 5), rng.uniform(0.05, 0.15)
        try:
            p = O.derive_lid(d["nx"], d["ny"], Re, Gr, d["Da"], d["eps"], d["Pr"], d["Le"], d["N"],
                             d["J"], d["sigma"], U0, d["varpi"], nee=nee)
        except ValueError:
            continue
        if not all(0 < s < 2 for s in list(p.s) + list(p.zeta) + list(p.eta)):
            continue
        L = d["nx"] - 1 if nee else d["nx"]
        _check_common(p, d, L)
        _close(L * U0 / p.nu, Re, "Re")
        _close(p.gbT * L ** 3 / p.nu ** 2, Gr, "Gr")
        _close(p.uw[3][0], U0, "lid velocity")
        checked += 1
    assert checked >= 10, checked
