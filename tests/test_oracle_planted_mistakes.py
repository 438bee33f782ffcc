"""The pins catch plausible mistakes in the oracle.

Each case plants one mistake in a copy of oracle/lbm_oracle.c (a dropped term, a wrong
sign, coefficient or index, a transposed operand), compiles the copy, and runs the pin
tests that should notice it against that copy (LBM_ORACLE_LIB): they must fail.  The
oracle itself is never altered; its unaltered pins run in the rest of the suite.

If the oracle's source is rewritten so that a planted expression no longer appears
verbatim, the case fails and names it, so that the list follows the source.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")
COLL = "tests/test_oracle_collision.py"
PHYS = "tests/test_oracle_physics.py"
WALLS = "tests/test_oracle_walls.py"
FIELD = "tests/test_oracle_porous_field.py"
NEE = "tests/test_oracle_nee.py"
DERIVE = "tests/test_oracle_derive.py"
MODEL_A = "tests/test_model_a.py"
RESID = "tests/test_oracle_residual.py"

# (what is planted, the correct expression, the mistaken one, the pins that must fail)
MISTAKES = [
    ("sign of S_7 in the forcing moments (Eq. 15)",
     "2.0 * rho0 * (ux * Fx - uy * Fy) / eps,", "-2.0 * rho0 * (ux * Fx - uy * Fy) / eps,", [COLL]),
    ("alpha_2 = -2 instead of -3 (Eq. 14, Sec. 3.1)",
     "double a1 = 1.0, a2 = -3.0;", "double a1 = 1.0, a2 = -2.0;", [COLL]),
    ("sign of the explicit d(T u)/dt (Eq. 27, Sec. 3.2)",
     "double XTx = Tux - hist[0], XTy = Tuy - hist[1];",
     "double XTx = hist[0] - Tux, XTy = hist[1] - Tuy;", [COLL]),
    ("model A's equilibrium (Eq. 30) in place of Eq. 24",
     ": -4.0 * cap * Phi + 5.0 * varpi * Phi;", ": (-4.0 + 5.0 * varpi) * cap * Phi;", [COLL]),
    ("eps dropped from the buoyancy half-force of v (Eq. 19)",
     "double vy = jy / p->rho0 + 0.5 * eps * Gy;", "double vy = jy / p->rho0 + 0.5 * Gy;", [COLL]),
    ("sign of the anti-bounce-back of a Dirichlet wall",
     "s->g2[opp[q] * n + x] = -gs[q] + 2.0 * wt_axis * kg * p->Tw[side];",
     "s->g2[opp[q] * n + x] = gs[q] + 2.0 * wt_axis * kg * p->Tw[side];", [WALLS]),
    ("source term dropped from the D2Q5 collision (Eqs. 21-22, 27)",
     "ns[k] = n[k] - rates[k] * (n[k] - neq[k]) + (1.0 - 0.5 * rates[k]) * S[k];",
     "ns[k] = n[k] - rates[k] * (n[k] - neq[k]);", [COLL]),
    ("eps dropped from l_0 (Eq. 19)",
     "double l0 = 0.5 * (1.0 + eps * 0.5 * p->nu / p->K);",
     "double l0 = 0.5 * (1.0 + 0.5 * p->nu / p->K);", [COLL]),
    ("eps dropped from the Forchheimer force (Eq. 5)",
     "- eps * p->Feps / sqrt(p->K) * umag * ux", "- p->Feps / sqrt(p->K) * umag * ux", [COLL]),
    ("eps dropped from the Darcy force (Eq. 5)",
     "double Fx = -eps * p->nu / p->K * ux", "double Fx = -p->nu / p->K * ux", [COLL]),
    ("Nu length scale nx - 1 with halfway walls (Eq. 38)",
     "nuL += -nx * dTdx_L / dT;", "nuL += -(nx - 1) * dTdx_L / dT;", [PHYS]),
    ("M^-1 transposed in the back-transform",
     "fs[i] += M9inv[i][k] * ms[k];", "fs[i] += M9inv[k][i] * ms[k];", [COLL]),
    ("N transposed in the D2Q5 source moments (Eq. 27)",
     "for (int i = 0; i < 5; ++i) S[k] += N5[k][i] * St[i];",
     "for (int i = 0; i < 5; ++i) S[k] += N5[i][k] * St[i];", [COLL]),
    ("C from sigma instead of eps (Eq. 26)",
     "double C = sh / p->eps;", "double C = sh / p->sigma;", [COLL]),
    ("eps^2 instead of eps^3 in F_eps (Eq. 7)",
     "p->Feps = 1.75 / sqrt(150.0 * p->eps * p->eps * p->eps);",
     "p->Feps = 1.75 / sqrt(150.0 * p->eps * p->eps);", [FIELD]),
    ("wrong rate with the forcing moments (Eq. 10)",
     "ms[k] = m[k] - p->s[k] * (m[k] - meq[k]) + (1.0 - 0.5 * p->s[k]) * S[k];",
     "ms[k] = m[k] - p->s[k] * (m[k] - meq[k]) + (1.0 - 0.5 * p->s[8 - k]) * S[k];", [COLL]),
    ("non-equilibrium part dropped at wall nodes (Eq. 33)",
     "F[q * n + xb] = eb + ff[q] - ef;", "F[q * n + xb] = eb;", [NEE + "::test_nee_couette_exact"]),
    ("sign of the convective wall term (Eq. 39)",
     "return (4.0 * Phi_f - Phi_ff + 2.0 * b) / (3.0 + 2.0 * a);",
     "return (4.0 * Phi_f - Phi_ff - 2.0 * b) / (3.0 - 2.0 * a);", [NEE + "::test_convective_right_wall_exact"]),
    ("weights of the one-sided gradient (Eqs. 36-37)",
     "(4.0 * Phi_f - Phi_ff + 2.0 * b)", "(4.0 * Phi_f - 2.0 * Phi_ff + 2.0 * b)",
     [NEE + "::test_convective_right_wall_exact"]),
    ("Nu length scale nx with wall nodes",
     "        const double L = (double)(nx - 1);", "        const double L = (double)nx;",
     [NEE + "::test_nee_dirichlet_conduction_exact"]),
    ("J dropped from s_nu (Sec. 4.1)",
     "double inv_snu = 0.5 + p->Ma * p->J * L * sqrt(p->Pr) / (sqrt(p->cs2) * sqrt(p->Ra));",
     "double inv_snu = 0.5 + p->Ma * L * sqrt(p->Pr) / (sqrt(p->cs2) * sqrt(p->Ra));", [DERIVE]),
    ("Pr for sqrt(Pr) in s_nu (Sec. 4.1)",
     "double inv_snu = 0.5 + p->Ma * p->J * L * sqrt(p->Pr) / (sqrt(p->cs2) * sqrt(p->Ra));",
     "double inv_snu = 0.5 + p->Ma * p->J * L * p->Pr / (sqrt(p->cs2) * sqrt(p->Ra));", [DERIVE]),
    ("length scale nx with wall nodes in the mapping",
     "double L = p->nee ? (double)(p->nx - 1) : (double)p->nx;", "double L = (double)p->nx;", [DERIVE]),
    ("c_sT^2 = varpi / 3",
     "p->csT2 = p->varpi / 2.0;", "p->csT2 = p->varpi / 3.0;", [DERIVE]),
    ("D_e = alpha_e Le",
     "p->D_e = p->alpha_e / p->Le;", "p->D_e = p->alpha_e * p->Le;", [DERIVE]),
    ("nu = nu_e J",
     "p->nu = p->nu_e / p->J;", "p->nu = p->nu_e * p->J;", [DERIVE]),
    ("g beta_T dT = U^2 / L^2",
     "p->gbT = p->U * p->U / L;", "p->gbT = p->U * p->U / (L * L);", [DERIVE]),
    ("sign of the moving-wall term of the bounce-back",
     "s->f2[opp[q] * n + x] = fs[q] - 2.0 * W9[q] * p->rho0 * eu / p->cs2;",
     "s->f2[opp[q] * n + x] = fs[q] + 2.0 * W9[q] * p->rho0 * eu / p->cs2;", [WALLS]),
    ("stream function without the half cell below the first node",
     "double acc = p->nee ? 0.0 : 0.25 * ux[i];", "double acc = 0.0;", [WALLS + "::test_couette_exact"]),
    ("stream function with rectangles for trapezoids",
     "acc += 0.5 * (ux[(size_t)(j - 1) * nx + i] + ux[(size_t)j * nx + i]);",
     "acc += ux[(size_t)j * nx + i];", [NEE + "::test_nee_couette_exact"]),
    ("model A's Dirichlet wall without its capacity factor",
     "double kg = p->model_a ? p->sigma : 1.0, kh = p->model_a ? px.eps : 1.0;",
     "double kg = 1.0, kh = 1.0;", [MODEL_A]),
    ("model A's n_eq,3 without the capacity (Eqs. 30-31)",
     "neq[3] = p->model_a ? (-4.0 + 5.0 * varpi) * cap * Phi", "neq[3] = p->model_a ? (-4.0 + 5.0 * varpi) * Phi",
     [MODEL_A]),
    ("model A's initial g_0 without sigma",
     "s->g[x] = (1.0 - varpi) * p->sigma * T;", "s->g[x] = (1.0 - varpi) * T;",
     [PHYS + "::test_initial_state_holds_the_given_fields"]),
    ("initial h_0 with the scalar porosity in a porosity field",
     "s->h[x] = eps_x * C - varpi * C;", "s->h[x] = p->eps * C - varpi * C;",
     [PHYS + "::test_initial_state_holds_the_given_fields"]),
    ("Nu length scale nx - 1 on the bottom wall (halfway walls)",
     "nuB += ny * (-8.0 * p->Tw[2] + 9.0 * T0 - T1) / 3.0 / dT;",
     "nuB += (ny - 1) * (-8.0 * p->Tw[2] + 9.0 * T0 - T1) / 3.0 / dT;", [WALLS + "::test_top_bottom_conduction_exact"]),
    ("F_eps of the scalar porosity in a porosity field (Eq. 7)",
     "        q.Feps = 1.75 / sqrt(150.0 * q.eps * q.eps * q.eps);   /* Eq. 7 */\n", "", [FIELD]),
    ("permeability field ignored",
     "if (s->K) q.K = s->K[x];", "if (0) q.K = s->K[x];", [FIELD]),
    ("sign in the top-wall gradient with wall nodes",
     "nuT += wi * L * (3.0 * t0[top] - 4.0 * t0[top - r] + t0[top - 2 * r]) / 2.0 / dT;",
     "nuT += wi * L * (3.0 * t0[top] - 4.0 * t0[top - r] - t0[top - 2 * r]) / 2.0 / dT;",
     [NEE + "::test_nee_top_bottom_conduction_exact"]),
    ("corner nodes take the side wall's velocity",
     "const int sv = dj ? (dj > 0 ? 2 : 3) : (di > 0 ? 0 : 1);",
     "const int sv = di ? (di > 0 ? 0 : 1) : (dj > 0 ? 2 : 3);",
     [NEE + "::test_nee_initial_wall_state_is_the_wall_equilibrium"]),
    ("wall-node equilibrium at the interior node's porosity (Eq. 33)",
     "meq9(&pb, of.rho, uwx, uwy, mb);", "meq9(&pf, of.rho, uwx, uwy, mb);",
     [NEE + "::test_nee_initial_wall_state_is_the_wall_equilibrium"]),
    ("C's anti-bounce-back with T's wall value",
     "s->h2[opp[q] * n + x] = -hs[q] + 2.0 * wt_axis * kh * p->Cw[side];",
     "s->h2[opp[q] * n + x] = -hs[q] + 2.0 * wt_axis * kh * p->Tw[side];",
     [PHYS + "::test_linear_conduction_with_distinct_wall_values"]),
    ("T's wall value taken from the opposite wall",
     "s->g2[opp[q] * n + x] = -gs[q] + 2.0 * wt_axis * kg * p->Tw[side];",
     "s->g2[opp[q] * n + x] = -gs[q] + 2.0 * wt_axis * kg * p->Tw[side ^ 1];", [PHYS]),
    ("C's initial noise drawn at T's keys",
     "p->C0 + noise * (2.0 * or_uniform(seed, n + x) - 1.0);",
     "p->C0 + noise * (2.0 * or_uniform(seed, x) - 1.0);", [COLL + "::test_splitmix64_definition"]),
    ("N^-1 transposed in the D2Q5 back-transform",
     "for (int k = 0; k < 5; ++k) ds[i] += N5inv[i][k] * ns[k];",
     "for (int k = 0; k < 5; ++k) ds[i] += N5inv[k][i] * ns[k];", [COLL]),
    ("D2Q5 axis weights varpi / 5",
     "double wt[5] = {1.0 - varpi, varpi / 4, varpi / 4, varpi / 4, varpi / 4};",
     "double wt[5] = {1.0 - varpi, varpi / 5, varpi / 5, varpi / 5, varpi / 5};", [COLL]),
    ("factor 2 under the root of Eq. 18",
     "double den = l0 + sqrt(l0 * l0 + l1 * vmag);", "double den = l0 + sqrt(l0 * l0 + 2.0 * l1 * vmag);", [COLL]),
    ("|v| for |u| in the Forchheimer force (Eq. 5)",
     "double Fx = -eps * p->nu / p->K * ux - eps * p->Feps / sqrt(p->K) * umag * ux + eps * Gx;",
     "double Fx = -eps * p->nu / p->K * ux - eps * p->Feps / sqrt(p->K) * vmag * ux + eps * Gx;", [COLL]),
    ("sign of the solutal buoyancy (Eq. 6)",
     "double Gy = p->gbT * (T - p->T0) + p->gbC * (C - p->C0);",
     "double Gy = p->gbT * (T - p->T0) - p->gbC * (C - p->C0);", [COLL]),
    ("eps dropped from m_eq,1 (Eq. 14)",
     "meq[1] = -2.0 * rho + 3.0 * rho0 * u2 / eps;", "meq[1] = -2.0 * rho + 3.0 * rho0 * u2;", [COLL]),
    ("eps dropped from m_eq,8 (Eq. 14)",
     "meq[8] = rho0 * ux * uy / eps;", "meq[8] = rho0 * ux * uy;", [COLL]),
    ("eps put into n_eq,1 (Eq. 24)",
     "neq[1] = ux * Phi;", "neq[1] = ux * Phi / p->eps;", [COLL]),
    ("C's source term from T's history",
     "double XCx = Cux - hist[2], XCy = Cuy - hist[3];",
     "double XCx = Cux - hist[0], XCy = Cuy - hist[1];", [COLL]),
    ("zeta for eta in the concentration collision",
     "collide_d2q5(p, p->eta, eps, o->C, ux, uy, XCx, XCy, h, hs);",
     "collide_d2q5(p, p->zeta, eps, o->C, ux, uy, XCx, XCy, h, hs);", [COLL]),
    ("C at x_ff through sigma (Eq. 26)",
     "const double Tff = sgff / pff.sigma, Cff = shff / pff.eps;",
     "const double Tff = sgff / pff.sigma, Cff = shff / pff.sigma;", [NEE + "::test_nee_dirichlet_conduction_exact"]),
    ("x_ff = x_f in the gradient extrapolation",
     "const size_t xff = (size_t)(j + 2 * dj) * nx + (i + 2 * di);",
     "const size_t xff = (size_t)(j + dj) * nx + (i + di);", [NEE + "::test_convective_right_wall_exact"]),
    ("a convective wall treated as Dirichlet",
     "if (!(Bi[sd] > 0.0) && kind == OR_DIRICHLET) return W[sd];",
     "if (kind == OR_DIRICHLET) return W[sd];", [NEE + "::test_convective_right_wall_exact"]),
    ("sign in the right-wall gradient (halfway walls)",
     "double dTdx_R = (8.0 * p->Tw[1] - 9.0 * Tr[nx - 1] + Tr[nx - 2]) / 3.0;",
     "double dTdx_R = (8.0 * p->Tw[1] - 9.0 * Tr[nx - 1] - Tr[nx - 2]) / 3.0;", [PHYS]),
    ("adiabatic wall reflecting h with a sign flip",
     "s->h2[opp[q] * n + x] = hs[q];", "s->h2[opp[q] * n + x] = -hs[q];",
     [PHYS + "::test_scalar_content_changes_by_the_wall_link_fluxes"]),
    ("adiabatic wall reflecting g into the same direction",
     "s->g2[opp[q] * n + x] = gs[q];", "s->g2[q * n + x] = gs[q];",
     [PHYS + "::test_scalar_content_changes_by_the_wall_link_fluxes"]),
    ("residual against the earlier field's maximum",
     "if (fabs(a[x]) > amax) amax = fabs(a[x]);", "if (fabs(b[x]) > amax) amax = fabs(b[x]);",
     [RESID]),
    ("residual without the concentration field",
     "    for (int q = 0; q < 4; ++q) {\n        const double* a = now + (size_t)q * n;",
     "    for (int q = 0; q < 3; ++q) {\n        const double* a = now + (size_t)q * n;", [RESID]),
    ("absolute instead of relative change in the residual",
     "            rq = dmax / amax;", "            rq = dmax;", [RESID]),
    ("residual snapshot not replaced by the current fields",
     "    memcpy(snap, now, 4 * n * sizeof(double));\n    free(now);",
     "    if (!have_snap) memcpy(snap, now, 4 * n * sizeof(double));\n    free(now);", [RESID]),
    ("residual of the first call taken against an empty snapshot",
     "    if (!have_snap) *r = INFINITY;\n", "", [RESID]),
    ("residual against the change's own maximum (deviations from the earlier field)",
     "            if (fabs(a[x]) > amax) amax = fabs(a[x]);",
     "            if (d > amax) amax = d;", [RESID]),
    ("plain mean for the trapezoidal mean with wall nodes",
     "const double wj = (j == 0 || j == ny - 1) ? 0.5 : 1.0;", "const double wj = 1.0;",
     [NEE + "::test_nee_dirichlet_conduction_exact"]),
]


def _build(tmp, k, src):
    c = os.path.join(tmp, f"planted_{k}.c")
    so = os.path.join(tmp, f"planted_{k}.so")
    with open(c, "w") as f:
        f.write(src)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-I", ORACLE,
                    "-o", so, c, "-lm"], check=True, capture_output=True)
    return so


def _pins_fail(so, targets):
    env = dict(os.environ, LBM_ORACLE_LIB=so, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", *targets, "-x", "-q", "-m", "not gpu",
                        "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    return r.returncode, r.stdout[-800:]


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc is needed to build the altered copies")
def test_every_planted_mistake_fails_a_pin(tmp_path):
    with open(os.path.join(ORACLE, "lbm_oracle.c")) as f:
        src = f.read()
    for what, good, _, _ in MISTAKES:
        assert src.count(good) == 1, f"'{what}': the expression is not in the oracle exactly once"
    sos = [_build(str(tmp_path), k, src.replace(good, bad)) for k, (_, good, bad, _) in enumerate(MISTAKES)]
    workers = max(1, min(8, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        results = list(ex.map(lambda a: _pins_fail(*a), [(so, m[3]) for so, m in zip(sos, MISTAKES)]))
    missed = [(m[0], out) for m, (rc, out) in zip(MISTAKES, results) if rc != 1]
    assert not missed, "planted mistakes not caught (pytest exit code != 1):\n" + "\n".join(
        f"- {w}:\n{o}" for w, o in missed)
