"""Pins of the oracle's steady-state residual.

The steady runs of Sec. 4 (Tables 1-5) are stopped when the fields stop changing; the
paper does not state its test, and the reading taken is the relative change of the four
fields over the last k steps,

    r = max over phi in {u_x, u_y, T, C} of max|phi_now - phi_prev| / max|phi_now|

with T and C the absolute values of Eq. 26.  The pins fix it without restating it:

* hand-made fields whose r follows from arithmetic alone: one node changed in one field
  at a time (each of the four fields must count), the larger of two changes wins, the
  denominator is the current field's maximum (not the earlier one's, not the change's),
  zero fields, a sign-independent change, a non-finite value;
* a state of the oracle: a sine of T and C diffusing at rest on a periodic grid decays at
  alpha_e k^2 / sigma and D_e k^2 / eps (Eq. 3-4 with Eq. 29; the decay itself is pinned in
  test_oracle_physics.py), so r between two calls follows in closed form; the first call
  gives +inf, a second call with no step in between gives 0, and the exact steady
  conduction profile gives r at round-off.
"""
import numpy as np
import pytest


def _fields(ny=3, nx=5, T=0.5, C=0.5):
    a = np.zeros((4, ny, nx))
    a[2] = T
    a[3] = C
    return a


def test_identical_fields_give_zero(oracle_mod):
    O = oracle_mod
    a = _fields()
    a[0] = 0.01
    r, bad = O.residual_fields(a, a.copy())
    assert r == 0.0 and not bad


@pytest.mark.parametrize("q", [0, 1, 2, 3])
def test_each_field_counts(oracle_mod, q):
    """A change of one node in field q alone: r = |change| / max|phi_q now|.  For T and C
    the maximum is of the absolute value (0.5 + change here), which a denominator in
    deviations T - T0 would turn into 1."""
    O = oracle_mod
    prev = _fields()
    prev[0] = 0.02      # a flow field that does not change
    prev[1] = -0.03
    now = prev.copy()
    d = 0.125
    now[q, 1, 2] += d
    r, bad = O.residual_fields(now, prev)
    assert not bad
    expect = d / np.abs(now[q]).max()
    assert r == pytest.approx(expect, rel=1e-15), (q, r, expect)


def test_largest_relative_change_wins_and_sign_does_not_matter(oracle_mod):
    O = oracle_mod
    prev = _fields(T=1.0, C=2.0)
    prev[0] = 0.5
    prev[1] = 0.25
    now = prev.copy()
    now[0, 0, 0] -= 0.05        # u_x: 0.05 / 0.5  = 0.1
    now[1, 2, 4] += 0.05        # u_y: 0.05 / 0.30 = 1/6 (max|u_y| is the changed node)
    now[2, 1, 1] -= 0.25        # T:   0.25 / 1.0  = 0.25
    now[3, 0, 3] += 0.2         # C:   0.2 / 2.2
    r, _ = O.residual_fields(now, prev)
    assert r == pytest.approx(0.25, rel=1e-15)
    now[2] = prev[2]            # without the change of T, u_y's 1/6 is the largest
    r, _ = O.residual_fields(now, prev)
    assert r == pytest.approx(0.05 / 0.3, rel=1e-14)


def test_denominator_is_the_current_maximum(oracle_mod):
    """prev had a larger peak than now: the ratio is taken against now's maximum."""
    O = oracle_mod
    prev = _fields()
    now = prev.copy()
    prev[2, 1, 2] = 1.0         # T fell from 1.0 to 0.5 at one node
    r, _ = O.residual_fields(now, prev)
    assert r == pytest.approx(0.5 / 0.5, rel=1e-15)


def test_zero_fields(oracle_mod):
    """u = 0 now and before contributes nothing; u = 0 now after a flow gives +inf."""
    O = oracle_mod
    prev = _fields()
    now = prev.copy()
    r, _ = O.residual_fields(now, prev)
    assert r == 0.0
    prev[0, 1, 1] = 1e-9
    r, _ = O.residual_fields(now, prev)
    assert r == np.inf


def test_non_finite_value_is_reported(oracle_mod):
    O = oracle_mod
    prev = _fields()
    now = prev.copy()
    now[3, 2, 0] = np.nan
    _, bad = O.residual_fields(now, prev)
    assert bad
    now[3, 2, 0] = 0.5
    now[0, 0, 0] = np.inf
    _, bad = O.residual_fields(now, prev)
    assert bad


def _diffusing_sine(O, cap, eps, A=0.1, nx=64):
    """T = C = T0 + A sin(k x) at rest on a periodic nx x 3 grid with no force."""
    ny = 3
    p = O.derive(nx, ny, 1e4, 1e-2, eps, 1, 1, 0, sigma=cap)
    p.periodic_x = p.periodic_y = 1
    p.gbT = p.gbC = 0.0
    p.K = 1e300
    za, ed = 1.0, 1.4
    p.zeta[1] = p.zeta[2] = za
    p.eta[1] = p.eta[2] = ed
    x = np.arange(nx) + 0.5
    kw = 2 * np.pi / nx
    T0f = np.broadcast_to(0.5 + A * np.sin(kw * x), (ny, nx)).copy()
    o = O.Oracle(p, seed=1, noise=0.0, T_init=T0f, C_init=T0f)
    lamT = p.csT2 * (1 / za - 0.5) * kw ** 2 / cap       # Eq. 29: alpha_e, then / sigma
    lamC = p.csT2 * (1 / ed - 0.5) * kw ** 2 / eps       # D_e / eps
    smax = np.abs(np.sin(kw * x)).max()
    return o, lamT, lamC, A * smax


def test_residual_of_a_diffusing_sine(oracle_mod):
    """Between calls at t1 and t2 the amplitude of T falls from a e^(-lam t1) to
    a e^(-lam t2): r_T = a (e^(-lam t1) - e^(-lam t2)) / (1/2 + a e^(-lam t2)), likewise
    r_C; u = 0 throughout contributes nothing.  sigma and eps are chosen so that T decays
    faster than C: r = r_T, and r_T and r_C differ by more than the tolerance."""
    O = oracle_mod
    o, lamT, lamC, a = _diffusing_sine(O, cap=0.5, eps=0.8)
    r0, bad = o.residual()
    assert r0 == np.inf and not bad
    r, _ = o.residual()                     # no step since the last call
    assert r == 0.0
    t1 = 0
    for t2 in (150, 400, 900):
        o.step(t2 - t1)
        r, bad = o.residual()
        rT = a * (np.exp(-lamT * t1) - np.exp(-lamT * t2)) / (0.5 + a * np.exp(-lamT * t2))
        rC = a * (np.exp(-lamC * t1) - np.exp(-lamC * t2)) / (0.5 + a * np.exp(-lamC * t2))
        assert rT > 1.1 * rC
        assert not bad
        assert r == pytest.approx(rT, rel=5e-3), (t2, r, rT, rC)
        t1 = t2


def test_residual_matches_the_fields_of_the_two_calls(oracle_mod):
    """The snapshot the state keeps is the fields of the previous call: r equals the
    residual of the two sets of fields read out at those times."""
    O = oracle_mod
    p = O.derive(20, 14, 1e5, 1e-2, 0.6, 1, 2, 1)
    o = O.Oracle(p, seed=3, noise=0.05)
    o.step(50)
    f1 = o.fields()
    o.residual()
    o.step(37)
    f2 = o.fields()
    r, _ = o.residual()
    stack = lambda f: np.stack([f["ux"], f["uy"], f["T"], f["C"]])
    r_ref, _ = O.residual_fields(stack(f2), stack(f1))
    assert r == r_ref and 0 < r < 1


def test_steady_conduction_has_round_off_residual(oracle_mod):
    """Ra = 0 between Dirichlet walls: the linear profile is an exact steady state of
    the lattice scheme, so r stays at round-off from step to step."""
    O = oracle_mod
    nx, ny = 16, 5
    p = O.derive(nx, ny, 1e4, 1e-2, 0.6, 1, 1, 0)
    p.gbT = p.gbC = 0.0
    x = (np.arange(nx) + 0.5) / nx
    Tl = np.broadcast_to(1.0 - x, (ny, nx)).copy()
    o = O.Oracle(p, seed=1, noise=0.0, T_init=Tl, C_init=Tl)
    o.step(20000)
    o.residual()
    o.step(100)
    r, _ = o.residual()
    assert r < 1e-13
