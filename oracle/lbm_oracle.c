/*
 * FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY (see lbm_oracle.h for scope,
 * citations and readings).  Plain loops in the paper's order: per node,
 * macroscopic quantities -> moments -> relaxation -> back to velocity space,
 * then push-streaming with the wall rules.  No blocking, fusion or reordering.
 */
#include "lbm_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- lattice definitions ------------------------------------------------ */

/* Eq. 8: D2Q9 velocities, c = 1.  The first five are the D2Q5 set (Sec. 3.2). */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
/* Eq. 20: D2Q9 weights */
static const double W9[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                             1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

/* Eq. 13: transformation matrix M (rows: rho, e, eps, jx, qx, jy, qy, pxx, pxy) */
static const double M9[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},
    {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},
    {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},
    {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},
    {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1}};

/* Eq. 23: D2Q5 transformation matrix N */
static const double N5[5][5] = {
    {1, 1, 1, 1, 1},
    {0, 1, 0, -1, 0},
    {0, 0, 1, 0, -1},
    {-4, 1, 1, 1, 1},
    {0, 1, -1, 1, -1}};

static double M9inv[9][9];
static double N5inv[5][5];
static int inverses_ready = 0;

/* index of the opposite velocity */
static int opposite(int q)
{
    for (int k = 0; k < 9; ++k)
        if (EX[k] == -EX[q] && EY[k] == -EY[q]) return k;
    return -1;
}

/* Gauss-Jordan inversion with partial pivoting (n <= 9). The paper defines
 * f* = M^-1 m* (Eq. 11); the inverse is computed, not written down. */
static void invert(int n, const double* a, double* inv)
{
    double w[9][18];
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < 2 * n; ++c)
            w[r][c] = c < n ? a[r * n + c] : (c - n == r ? 1.0 : 0.0);
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(w[r][col]) > fabs(w[piv][col])) piv = r;
        if (piv != col)
            for (int c = 0; c < 2 * n; ++c) {
                double t = w[col][c];
                w[col][c] = w[piv][c];
                w[piv][c] = t;
            }
        double d = w[col][col];
        for (int c = 0; c < 2 * n; ++c) w[col][c] /= d;
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            double m = w[r][col];
            if (m == 0.0) continue;
            for (int c = 0; c < 2 * n; ++c) w[r][c] -= m * w[col][c];
        }
    }
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) inv[r * n + c] = w[r][n + c];
}

static void ensure_inverses(void)
{
    if (inverses_ready) return;
    invert(9, &M9[0][0], &M9inv[0][0]);
    invert(5, &N5[0][0], &N5inv[0][0]);
    inverses_ready = 1;
}

/* ---- parameters (Sec. 4, Sec. 4.1, Eqs. 7, 14, 29) ------------------------- */

int or_derive(or_params* p)
{
    if (p->nx < 3 || p->ny < 3) return 1;
    if (p->nee && (p->nx < 5 || p->ny < 5)) return 1;   /* x_ff must be an interior node */
    if (!(p->eps > 0.0 && p->eps <= 1.0) || !(p->Da > 0.0) || !(p->Ra > 0.0) || !(p->Pr > 0.0) ||
        !(p->Le > 0.0) || !(p->J > 0.0) || !(p->sigma > 0.0))
        return 1;
    if (p->Ma <= 0.0) p->Ma = 0.1;          /* Sec. 4.1: Ma = 0.1 */
    if (p->varpi <= 0.0) p->varpi = 0.4;    /* Sec. 4: varpi = 2/5 */
    /* Sec. 4.1: L = N_x in lattice units; with nodes on the walls the N_x lattice
     * spacings between the walls take N_x + 1 nodes */
    double L = p->nee ? (double)(p->nx - 1) : (double)p->nx;
    p->rho0 = 1.0;
    p->cs2 = 1.0 / 3.0;                     /* c_s = c / sqrt(3) */
    p->U = p->Ma * sqrt(p->cs2);            /* Ma = U / c_s */
    /* 1/s_nu = 1/2 + Ma J L sqrt(Pr) / (c_s sqrt(Ra)), i.e. nu_e = J U L sqrt(Pr/Ra) */
    double inv_snu = 0.5 + p->Ma * p->J * L * sqrt(p->Pr) / (sqrt(p->cs2) * sqrt(p->Ra));
    p->nu_e = p->cs2 * (inv_snu - 0.5);     /* nu_e = c_s^2 (1/s_nu - 1/2) */
    p->nu = p->nu_e / p->J;                 /* J = nu_e / nu */
    p->alpha_e = p->nu / p->Pr;             /* Pr = nu / alpha_e */
    p->D_e = p->alpha_e / p->Le;            /* Le = alpha_e / D_e */
    p->csT2 = p->varpi / 2.0;               /* c_sT^2 = varpi / 2 */
    p->K = p->Da * L * L;                   /* Da = K / L^2 */
    p->Feps = 1.75 / sqrt(150.0 * p->eps * p->eps * p->eps); /* Eq. 7 */
    p->gbT = p->U * p->U / L;               /* U = sqrt(g beta_T dT L), dT = 1 */
    p->gbC = p->N * p->gbT;                 /* N = beta_C dC / (beta_T dT), dC = dT = 1 */
    p->T0 = 0.5;                            /* T0 = (T_h + T_l)/2 with T_h = 1, T_l = 0 */
    p->C0 = 0.5;
    /* Sec. 4: s0 = s3 = s5 = 1, s1 = s2 = 1.1, s4 = s6 = 1.2; s7 = s8 = s_nu */
    double snu = 1.0 / inv_snu;
    double rates[9] = {1.0, 1.1, 1.1, 1.0, 1.2, 1.0, 1.2, snu, snu};
    memcpy(p->s, rates, sizeof rates);
    /* Eq. 29: alpha_e = c_sT^2 (1/zeta_a - 1/2), D_e = c_sT^2 (1/eta_D - 1/2) */
    double za = 1.0 / (0.5 + p->alpha_e / p->csT2);
    double eD = 1.0 / (0.5 + p->D_e / p->csT2);
    double z[5] = {1.0, za, za, 1.5, 1.5};  /* zeta_0 = 1, zeta_3 = zeta_4 = 1.5 */
    double e[5] = {1.0, eD, eD, 1.5, 1.5};  /* eta_0 = 1, eta_3 = eta_4 = 1.5 */
    memcpy(p->zeta, z, sizeof z);
    memcpy(p->eta, e, sizeof e);
    p->scalar_lr = OR_DIRICHLET;
    p->scalar_tb = OR_ADIABATIC;
    p->Tw[0] = 1.0; p->Tw[1] = 0.0; p->Tw[2] = 0.5; p->Tw[3] = 0.5;
    p->Cw[0] = 1.0; p->Cw[1] = 0.0; p->Cw[2] = 0.5; p->Cw[3] = 0.5;
    memset(p->uw, 0, sizeof p->uw);
    memset(p->BiT, 0, sizeof p->BiT);
    memset(p->BiC, 0, sizeof p->BiC);
    p->Gx = 0.0;
    p->model_a = 0;
    for (int k = 0; k < 9; ++k) if (!(p->s[k] > 0.0 && p->s[k] < 2.0)) return 2;
    for (int k = 0; k < 5; ++k)
        if (!(p->zeta[k] > 0.0 && p->zeta[k] < 2.0) || !(p->eta[k] > 0.0 && p->eta[k] < 2.0))
            return 2;
    return 0;
}

/* ---- state ---------------------------------------------------------------- */

struct or_state {
    or_params p;
    long t;
    size_t n;
    double *f, *g, *h, *hist;   /* pre-collision distributions at time t */
    double *f2, *g2, *h2;       /* streaming targets */
    double *eps, *K;            /* optional per-node porosity / permeability */
};

/* The parameters at node x: the uniform ones, or with that node's eps, K, F_eps. */
static or_params node_params(const or_state* s, size_t x)
{
    or_params q = s->p;
    if (s->eps) {
        q.eps = s->eps[x];
        q.Feps = 1.75 / sqrt(150.0 * q.eps * q.eps * q.eps);   /* Eq. 7 */
    }
    if (s->K) q.K = s->K[x];
    return q;
}

long or_time(const or_state* s) { return s->t; }

/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the state advances by the
 * golden-ratio increment and each output is the mix of the state.  The k-th
 * output of a generator seeded with `seed` is mix(seed + (k+1)*gamma). */
static uint64_t splitmix64_at(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + (k + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double or_uniform(uint64_t seed, uint64_t k)
{
    return (double)(splitmix64_at(seed, k) >> 11) * (1.0 / 9007199254740992.0); /* 2^-53 */
}

/* ---- per-node method -------------------------------------------------------- */

typedef struct {
    double rho, jx, jy, T, C, Gx, Gy, ux, uy, Fx, Fy;
} or_macro;

/* Eqs. 16, 26, 6, 19, 18, 5 in that order. */
static void macro(const or_params* p, const double f[9], const double g[5], const double h[5],
                  or_macro* o)
{
    double rho = 0, jx = 0, jy = 0;
    for (int i = 0; i < 9; ++i) {
        rho += f[i];                               /* Eq. 16 */
        jx += EX[i] * f[i];                        /* sum e_i f_i */
        jy += EY[i] * f[i];
    }
    double sg = 0, sh = 0;
    for (int i = 0; i < 5; ++i) { sg += g[i]; sh += h[i]; }
    double T = sg / p->sigma;                      /* Eq. 26: sigma T = sum g */
    double C = sh / p->eps;                        /* Eq. 26: eps C = sum h */
    double Gx = p->Gx;                             /* external, test-only */
    double Gy = p->gbT * (T - p->T0) + p->gbC * (C - p->C0);   /* Eq. 6 */
    double eps = p->eps;
    /* Eq. 19 (delta_t = 1) */
    double vx = jx / p->rho0 + 0.5 * eps * Gx;
    double vy = jy / p->rho0 + 0.5 * eps * Gy;
    double l0 = 0.5 * (1.0 + eps * 0.5 * p->nu / p->K);
    double l1 = eps * 0.5 * p->Feps / sqrt(p->K);
    double vmag = sqrt(vx * vx + vy * vy);
    /* Eq. 18 */
    double den = l0 + sqrt(l0 * l0 + l1 * vmag);
    double ux = vx / den, uy = vy / den;
    /* Eq. 5 */
    double umag = sqrt(ux * ux + uy * uy);
    double Fx = -eps * p->nu / p->K * ux - eps * p->Feps / sqrt(p->K) * umag * ux + eps * Gx;
    double Fy = -eps * p->nu / p->K * uy - eps * p->Feps / sqrt(p->K) * umag * uy + eps * Gy;
    o->rho = rho; o->jx = jx; o->jy = jy; o->T = T; o->C = C; o->Gx = Gx; o->Gy = Gy;
    o->ux = ux; o->uy = uy; o->Fx = Fx; o->Fy = Fy;
}

/* Eq. 14 with alpha_1 = 1, alpha_2 = -3 (Sec. 3.1): equilibrium moments of f. */
static void meq9(const or_params* p, double rho, double ux, double uy, double meq[9])
{
    double rho0 = p->rho0, eps = p->eps;
    double u2 = ux * ux + uy * uy;
    double a1 = 1.0, a2 = -3.0;
    meq[0] = rho;
    meq[1] = -2.0 * rho + 3.0 * rho0 * u2 / eps;
    meq[2] = a1 * rho + a2 * rho0 * u2 / eps;
    meq[3] = rho0 * ux;
    meq[4] = -rho0 * ux;
    meq[5] = rho0 * uy;
    meq[6] = -rho0 * uy;
    meq[7] = rho0 * (ux * ux - uy * uy) / eps;
    meq[8] = rho0 * ux * uy / eps;
}

/* Eqs. 24/25 (model A: Eqs. 30/31): equilibrium moments of the D2Q5 lattice of a
 * scalar Phi whose zeroth moment carries the factor cap (sigma for T, eps for C). */
static void neq5(const or_params* p, double cap, double Phi, double ux, double uy, double neq[5])
{
    double varpi = p->varpi;
    neq[0] = cap * Phi;
    neq[1] = ux * Phi;
    neq[2] = uy * Phi;
    neq[3] = p->model_a ? (-4.0 + 5.0 * varpi) * cap * Phi : -4.0 * cap * Phi + 5.0 * varpi * Phi;
    neq[4] = 0.0;
}

/* D2Q5 collision (Eqs. 21/22 with Eqs. 24/25 and 27) for a scalar Phi whose
 * zeroth moment carries the factor `cap` (sigma for T, eps for C). */
static void collide_d2q5(const or_params* p, const double rates[5], double cap, double Phi,
                         double ux, double uy, double Xx, double Xy, const double d[5],
                         double ds[5])
{
    double varpi = p->varpi;
    double wt[5] = {1.0 - varpi, varpi / 4, varpi / 4, varpi / 4, varpi / 4};
    /* Eq. 27: S~_i = w~_i e_i . d(Phi u)/dt / c_sT^2, then S = N S~ */
    double St[5], S[5];
    for (int i = 0; i < 5; ++i) St[i] = wt[i] * (EX[i] * Xx + EY[i] * Xy) / p->csT2;
    for (int k = 0; k < 5; ++k) {
        S[k] = 0;
        for (int i = 0; i < 5; ++i) S[k] += N5[k][i] * St[i];
    }
    /* n = N d */
    double n[5];
    for (int k = 0; k < 5; ++k) {
        n[k] = 0;
        for (int i = 0; i < 5; ++i) n[k] += N5[k][i] * d[i];
    }
    /* Eqs. 24/25: modified equilibrium moments; model A: Eqs. 30/31 */
    double neq[5];
    neq5(p, cap, Phi, ux, uy, neq);
    /* n* = n - Theta (n - n_eq) + (I - Theta/2) S */
    double ns[5];
    for (int k = 0; k < 5; ++k)
        ns[k] = n[k] - rates[k] * (n[k] - neq[k]) + (1.0 - 0.5 * rates[k]) * S[k];
    for (int i = 0; i < 5; ++i) {
        ds[i] = 0;
        for (int k = 0; k < 5; ++k) ds[i] += N5inv[i][k] * ns[k];
    }
}

static void collide(const or_params* p, const double f[9], const double g[5], const double h[5],
                    double hist[4], double fs[9], double gs[5], double hs[5], or_macro* o)
{
    macro(p, f, g, h, o);
    double rho0 = p->rho0, eps = p->eps;
    double ux = o->ux, uy = o->uy, Fx = o->Fx, Fy = o->Fy, rho = o->rho;
    /* Eqs. 12-13: m = M f */
    double m[9];
    for (int k = 0; k < 9; ++k) {
        m[k] = 0;
        for (int i = 0; i < 9; ++i) m[k] += M9[k][i] * f[i];
    }
    /* Eq. 14 */
    double meq[9];
    meq9(p, rho, ux, uy, meq);
    /* Eq. 15 */
    double uF = ux * Fx + uy * Fy;
    double S[9] = {0.0,
                   6.0 * rho0 * uF / eps,
                   -6.0 * rho0 * uF / eps,
                   rho0 * Fx,
                   -rho0 * Fx,
                   rho0 * Fy,
                   -rho0 * Fy,
                   2.0 * rho0 * (ux * Fx - uy * Fy) / eps,
                   rho0 * (ux * Fy + uy * Fx) / eps};
    /* Eq. 10 (delta_t = 1) */
    double ms[9];
    for (int k = 0; k < 9; ++k)
        ms[k] = m[k] - p->s[k] * (m[k] - meq[k]) + (1.0 - 0.5 * p->s[k]) * S[k];
    /* f* = M^-1 m* */
    for (int i = 0; i < 9; ++i) {
        fs[i] = 0;
        for (int k = 0; k < 9; ++k) fs[i] += M9inv[i][k] * ms[k];
    }
    /* Eq. 27 with the explicit difference d(Tu)/dt = (Tu)|t - (Tu)|t-1 (Sec. 3.2) */
    double Tux = o->T * ux, Tuy = o->T * uy, Cux = o->C * ux, Cuy = o->C * uy;
    double XTx = Tux - hist[0], XTy = Tuy - hist[1];
    double XCx = Cux - hist[2], XCy = Cuy - hist[3];
    hist[0] = Tux; hist[1] = Tuy; hist[2] = Cux; hist[3] = Cuy;
    collide_d2q5(p, p->zeta, p->sigma, o->T, ux, uy, XTx, XTy, g, gs);   /* Eq. 21, 24 */
    collide_d2q5(p, p->eta, eps, o->C, ux, uy, XCx, XCy, h, hs);         /* Eq. 22, 25 */
}

void or_collide_node(const or_params* p, const double f[9], const double g[5],
                     const double h[5], double hist[4], double fs[9], double gs[5],
                     double hs[5], double mac[7])
{
    ensure_inverses();
    or_macro o;
    collide(p, f, g, h, hist, fs, gs, hs, &o);
    mac[0] = o.rho; mac[1] = o.ux; mac[2] = o.uy; mac[3] = o.T; mac[4] = o.C;
    mac[5] = o.Fx; mac[6] = o.Fy;
}

/* ---- walls with nodes on them (Sec. 3.3) -------------------------------------------- */

/* Value of the scalar Phi (T or C) at a boundary node whose inward link to the
 * nearest interior node is (di, dj), from Phi_f at x_f = x_b + (di, dj) and Phi_ff
 * at x_ff = x_b + 2 (di, dj).  A Dirichlet wall at the node gives its value (the
 * left / right wall first at a corner).  Otherwise every wall at the node is of
 * gradient type and Eq. 36/37 applies along (di, dj):
 *   Phi_b = (4 Phi_f - Phi_ff - 2 dx . grad Phi_b) / 3,
 * where each wall contributes its inward derivative, dx . grad Phi = sum over the
 * walls of (Bi / L)(Phi_b - Phi_w) (Eq. 39 as a convective condition, Bi = 0 for
 * an adiabatic wall); solved for Phi_b. */
static double nee_scalar(const or_params* p, int di, int dj, const double W[4], const double Bi[4],
                         double Phi_f, double Phi_ff)
{
    const double L = (double)(p->nx - 1);
    int sides[2], ns = 0;
    if (di) sides[ns++] = di > 0 ? 0 : 1;
    if (dj) sides[ns++] = dj > 0 ? 2 : 3;
    for (int k = 0; k < ns; ++k) {
        int sd = sides[k];
        int kind = sd < 2 ? p->scalar_lr : p->scalar_tb;
        if (!(Bi[sd] > 0.0) && kind == OR_DIRICHLET) return W[sd];
    }
    double a = 0.0, b = 0.0;   /* sum of Bi / L and of (Bi / L) Phi_w */
    for (int k = 0; k < ns; ++k) {
        int sd = sides[k];
        if (Bi[sd] > 0.0) {
            a += Bi[sd] / L;
            b += Bi[sd] / L * W[sd];
        }
    }
    return (4.0 * Phi_f - Phi_ff + 2.0 * b) / (3.0 + 2.0 * a);
}

/* Eqs. 33-35 at every boundary node of the arrays F, G, H (layout [q][ny][nx]),
 * from the post-streaming values at interior nodes.  x_f is the nearest interior
 * node along the inward wall normal (the diagonal one at a corner), x_ff the next
 * one along the same link.  The full sets f, g, h of the boundary node are
 * replaced:
 *   f_i(x_b) = f_i^eq(rho(x_f), u_w) + f_i(x_f) - f_i^eq(rho(x_f), u(x_f))     (Eq. 33)
 *   g_i(x_b) = g_i^eq(T_b, u_w) + g_i(x_f) - g_i^eq(T(x_f), u(x_f))            (Eq. 34)
 *   h_i(x_b) = h_i^eq(C_b, u_w) + h_i(x_f) - h_i^eq(C(x_f), u(x_f))            (Eq. 35)
 * with the equilibria f^eq = M^-1 m^eq (Eq. 14) and g^eq = N^-1 n^eq (Eqs. 24/25),
 * each at its own node's porosity, u(x_f) from Eq. 18, T_b / C_b from the wall's
 * Dirichlet value or Eqs. 36/37, and u_w the velocity of the wall (the bottom /
 * top wall's at a corner).  Only interior nodes are read, so the order of the
 * boundary nodes does not matter. */
static void nee_apply(const or_state* s, double* F, double* G, double* H)
{
    const or_params* p = &s->p;
    const int nx = p->nx, ny = p->ny;
    const size_t n = s->n;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int di = 0, dj = 0;
            if (!p->periodic_x) di = i == 0 ? 1 : (i == nx - 1 ? -1 : 0);
            if (!p->periodic_y) dj = j == 0 ? 1 : (j == ny - 1 ? -1 : 0);
            if (!di && !dj) continue;
            const size_t xb = (size_t)j * nx + i;
            const size_t xf = (size_t)(j + dj) * nx + (i + di);
            const size_t xff = (size_t)(j + 2 * dj) * nx + (i + 2 * di);
            double ff[9], gf[5], hf[5];
            for (int q = 0; q < 9; ++q) ff[q] = F[q * n + xf];
            for (int q = 0; q < 5; ++q) { gf[q] = G[q * n + xf]; hf[q] = H[q * n + xf]; }
            const or_params pb = node_params(s, xb), pf = node_params(s, xf), pff = node_params(s, xff);
            or_macro of;
            macro(&pf, ff, gf, hf, &of);
            double sgff = 0, shff = 0;
            for (int q = 0; q < 5; ++q) { sgff += G[q * n + xff]; shff += H[q * n + xff]; }
            const double Tff = sgff / pff.sigma, Cff = shff / pff.eps;   /* Eq. 26 */
            const int sv = dj ? (dj > 0 ? 2 : 3) : (di > 0 ? 0 : 1);
            const double uwx = p->uw[sv][0], uwy = p->uw[sv][1];
            /* Eq. 33 */
            double mb[9], mf[9];
            meq9(&pb, of.rho, uwx, uwy, mb);
            meq9(&pf, of.rho, of.ux, of.uy, mf);
            for (int q = 0; q < 9; ++q) {
                double eb = 0, ef = 0;
                for (int k = 0; k < 9; ++k) { eb += M9inv[q][k] * mb[k]; ef += M9inv[q][k] * mf[k]; }
                F[q * n + xb] = eb + ff[q] - ef;
            }
            /* Eqs. 34-37 */
            const double Tb = nee_scalar(p, di, dj, p->Tw, p->BiT, of.T, Tff);
            const double Cb = nee_scalar(p, di, dj, p->Cw, p->BiC, of.C, Cff);
            double nb[5], nf[5], kb[5], kf[5];
            neq5(&pb, pb.sigma, Tb, uwx, uwy, nb);
            neq5(&pf, pf.sigma, of.T, of.ux, of.uy, nf);
            neq5(&pb, pb.eps, Cb, uwx, uwy, kb);
            neq5(&pf, pf.eps, of.C, of.ux, of.uy, kf);
            for (int q = 0; q < 5; ++q) {
                double gb = 0, gff = 0, hb = 0, hff = 0;
                for (int k = 0; k < 5; ++k) {
                    gb += N5inv[q][k] * nb[k];
                    gff += N5inv[q][k] * nf[k];
                    hb += N5inv[q][k] * kb[k];
                    hff += N5inv[q][k] * kf[k];
                }
                G[q * n + xb] = gb + gf[q] - gff;
                H[q * n + xb] = hb + hf[q] - hff;
            }
        }
}

/* ---- creation ---------------------------------------------------------------- */

or_state* or_create(const or_params* p, uint64_t seed, double noise, const double* T_init,
                    const double* C_init)
{
    return or_create_field(p, seed, noise, T_init, C_init, NULL, NULL);
}

or_state* or_create_field(const or_params* p, uint64_t seed, double noise, const double* T_init,
                          const double* C_init, const double* eps_field, const double* K_field)
{
    ensure_inverses();
    or_state* s = (or_state*)calloc(1, sizeof(or_state));
    if (!s) return NULL;
    s->p = *p;
    s->n = (size_t)p->nx * (size_t)p->ny;
    size_t n = s->n;
    s->f = (double*)calloc(9 * n, sizeof(double));
    s->g = (double*)calloc(5 * n, sizeof(double));
    s->h = (double*)calloc(5 * n, sizeof(double));
    s->hist = (double*)calloc(4 * n, sizeof(double));
    s->f2 = (double*)calloc(9 * n, sizeof(double));
    s->g2 = (double*)calloc(5 * n, sizeof(double));
    s->h2 = (double*)calloc(5 * n, sizeof(double));
    if (!s->f || !s->g || !s->h || !s->hist || !s->f2 || !s->g2 || !s->h2) {
        or_destroy(s);
        return NULL;
    }
    if (eps_field) {
        s->eps = (double*)malloc(n * sizeof(double));
        if (!s->eps) { or_destroy(s); return NULL; }
        memcpy(s->eps, eps_field, n * sizeof(double));
    }
    if (K_field) {
        s->K = (double*)malloc(n * sizeof(double));
        if (!s->K) { or_destroy(s); return NULL; }
        memcpy(s->K, K_field, n * sizeof(double));
    }
    double varpi = p->varpi;
    for (int j = 0; j < p->ny; ++j)
        for (int i = 0; i < p->nx; ++i) {
            size_t x = (size_t)j * p->nx + i;
            const double eps_x = s->eps ? s->eps[x] : p->eps;
            /* noise key: (field * ny + j) * nx + i, field 0 = T, 1 = C */
            double T = T_init ? T_init[x]
                              : p->T0 + noise * (2.0 * or_uniform(seed, x) - 1.0);
            double C = C_init ? C_init[x]
                              : p->C0 + noise * (2.0 * or_uniform(seed, n + x) - 1.0);
            /* Eq. 20 at rho = rho0, u = 0 */
            for (int q = 0; q < 9; ++q) s->f[q * n + x] = W9[q] * p->rho0;
            /* Eq. 28 at u = 0; model A: g_i^eq = w~_i T (sigma + e_i.u / c_sT^2) at u = 0 */
            if (!p->model_a) {
                s->g[x] = p->sigma * T - varpi * T;
                s->h[x] = eps_x * C - varpi * C;
                for (int q = 1; q < 5; ++q) {
                    s->g[q * n + x] = varpi / 4 * T;
                    s->h[q * n + x] = varpi / 4 * C;
                }
            } else {
                s->g[x] = (1.0 - varpi) * p->sigma * T;
                s->h[x] = (1.0 - varpi) * eps_x * C;
                for (int q = 1; q < 5; ++q) {
                    s->g[q * n + x] = varpi / 4 * p->sigma * T;
                    s->h[q * n + x] = varpi / 4 * eps_x * C;
                }
            }
        }
    /* with nodes on the walls the state at t = 0 obeys the wall rules too */
    if (p->nee) nee_apply(s, s->f, s->g, s->h);
    /* history = (T u, C u) of the initial state */
    for (size_t x = 0; x < n; ++x) {
        double fl[9], gl[5], hl[5];
        for (int q = 0; q < 9; ++q) fl[q] = s->f[q * n + x];
        for (int q = 0; q < 5; ++q) { gl[q] = s->g[q * n + x]; hl[q] = s->h[q * n + x]; }
        or_macro o;
        or_params px = node_params(s, x);
        macro(&px, fl, gl, hl, &o);
        s->hist[0 * n + x] = o.T * o.ux;
        s->hist[1 * n + x] = o.T * o.uy;
        s->hist[2 * n + x] = o.C * o.ux;
        s->hist[3 * n + x] = o.C * o.uy;
    }
    return s;
}

void or_destroy(or_state* s)
{
    if (!s) return;
    free(s->f); free(s->g); free(s->h); free(s->hist);
    free(s->f2); free(s->g2); free(s->h2);
    free(s->eps); free(s->K);
    free(s);
}

/* The initial T and C (reading r8: 1/2 plus noise * (2U - 1), U the SplitMix64 output
 * with key (field * ny + j) * nx + i) of the window [x0, x0 + w) x [y0, y0 + h) of an
 * nx x ny cavity, into T[h][w], C[h][w].  A window run of the oracle started from these
 * reproduces the whole cavity's run within its dependence cone. */
void or_noise_window(uint64_t seed, double noise, int nx, int ny, int x0, int y0, int w, int h,
                     double* T, double* C)
{
    const uint64_t n = (uint64_t)nx * (uint64_t)ny;
    for (int j = 0; j < h; ++j)
        for (int i = 0; i < w; ++i) {
            const uint64_t k = (uint64_t)(y0 + j) * (uint64_t)nx + (uint64_t)(x0 + i);
            T[(size_t)j * w + i] = 0.5 + noise * (2.0 * or_uniform(seed, k) - 1.0);
            C[(size_t)j * w + i] = 0.5 + noise * (2.0 * or_uniform(seed, n + k) - 1.0);
        }
}

/* ---- one time step ------------------------------------------------------------- */

void or_step(or_state* s, long nsteps)
{
    const or_params* p = &s->p;
    const int nx = p->nx, ny = p->ny;
    const size_t n = s->n;
    int opp[9];
    for (int q = 0; q < 9; ++q) opp[q] = opposite(q);
    const double wt_axis = p->varpi / 4;  /* w~_1..4 */
    for (long step = 0; step < nsteps; ++step) {
#pragma omp parallel for schedule(static)
        for (int j = 0; j < ny; ++j) {
            for (int i = 0; i < nx; ++i) {
                size_t x = (size_t)j * nx + i;
                double f[9], g[5], h[5], hist[4], fs[9], gs[5], hs[5];
                for (int q = 0; q < 9; ++q) f[q] = s->f[q * n + x];
                for (int q = 0; q < 5; ++q) { g[q] = s->g[q * n + x]; h[q] = s->h[q * n + x]; }
                for (int k = 0; k < 4; ++k) hist[k] = s->hist[k * n + x];
                or_macro o;
                const or_params px = node_params(s, x);
                collide(&px, f, g, h, hist, fs, gs, hs, &o);
                for (int k = 0; k < 4; ++k) s->hist[k * n + x] = hist[k];
                /* Eq. 11: push f*_q to x + e_q; links that leave the cavity are
                 * reflected at the halfway wall back into the opposite slot of x. */
                for (int q = 0; q < 9; ++q) {
                    int ti = i + EX[q], tj = j + EY[q];
                    if (p->periodic_x) ti = (ti + nx) % nx;
                    if (p->periodic_y) tj = (tj + ny) % ny;
                    if (ti >= 0 && ti < nx && tj >= 0 && tj < ny) {
                        s->f2[q * n + (size_t)tj * nx + ti] = fs[q];
                    } else if (p->nee) {
                        /* leaves through a wall node: the wall rule rebuilds what enters */
                    } else {
                        /* halfway bounce-back off a wall moving with u_w (a resting wall:
                         * no-slip): f_opp(x) = f*_q(x) - 2 w_q rho0 (e_q . u_w) / c_s^2.
                         * A link through a corner takes the bottom / top wall. */
                        int side = (tj < 0 || tj >= ny) ? (tj < 0 ? 2 : 3) : (ti < 0 ? 0 : 1);
                        double eu = EX[q] * p->uw[side][0] + EY[q] * p->uw[side][1];
                        s->f2[opp[q] * n + x] = fs[q] - 2.0 * W9[q] * p->rho0 * eu / p->cs2;
                    }
                }
                for (int q = 0; q < 5; ++q) {
                    int ti = i + EX[q], tj = j + EY[q];
                    if (p->periodic_x) ti = (ti + nx) % nx;
                    if (p->periodic_y) tj = (tj + ny) % ny;
                    if (ti >= 0 && ti < nx && tj >= 0 && tj < ny) {
                        s->g2[q * n + (size_t)tj * nx + ti] = gs[q];
                        s->h2[q * n + (size_t)tj * nx + ti] = hs[q];
                        continue;
                    }
                    if (p->nee) continue;
                    int lr = (ti < 0 || ti >= nx);           /* left/right wall link */
                    int type = lr ? p->scalar_lr : p->scalar_tb;
                    if (type == OR_DIRICHLET) {
                        /* anti-bounce-back: g_opp(x) = -g*_q(x) + g_q^eq(T_w) + g_opp^eq(T_w),
                         * = 2 w~ T_w (Eq. 28), = 2 w~ sigma T_w (model A) */
                        int side = lr ? (ti < 0 ? 0 : 1) : (tj < 0 ? 2 : 3);
                        double kg = p->model_a ? p->sigma : 1.0, kh = p->model_a ? px.eps : 1.0;
                        s->g2[opp[q] * n + x] = -gs[q] + 2.0 * wt_axis * kg * p->Tw[side];
                        s->h2[opp[q] * n + x] = -hs[q] + 2.0 * wt_axis * kh * p->Cw[side];
                    } else {
                        /* adiabatic / impermeable: plain bounce-back */
                        s->g2[opp[q] * n + x] = gs[q];
                        s->h2[opp[q] * n + x] = hs[q];
                    }
                }
            }
        }
        /* Sec. 3.3: boundary nodes from the post-streaming interior */
        if (p->nee) nee_apply(s, s->f2, s->g2, s->h2);
        double* t;
        t = s->f; s->f = s->f2; s->f2 = t;
        t = s->g; s->g = s->g2; s->g2 = t;
        t = s->h; s->h = s->h2; s->h2 = t;
        s->t += 1;
    }
}

/* ---- read-out ---------------------------------------------------------------- */

void or_fields(const or_state* s, double* ux, double* uy, double* T, double* C, double* rho)
{
    size_t n = s->n;
    for (size_t x = 0; x < n; ++x) {
        double f[9], g[5], h[5];
        for (int q = 0; q < 9; ++q) f[q] = s->f[q * n + x];
        for (int q = 0; q < 5; ++q) { g[q] = s->g[q * n + x]; h[q] = s->h[q * n + x]; }
        or_macro o;
        const or_params px = node_params(s, x);
        macro(&px, f, g, h, &o);
        if (ux) ux[x] = o.ux;
        if (uy) uy[x] = o.uy;
        if (T) T[x] = o.T;
        if (C) C[x] = o.C;
        if (rho) rho[x] = o.rho;
    }
}

/* Eq. 38 with a second-order one-sided wall gradient through the wall value and
 * the first two nodes (at distances 1/2 and 3/2 from the halfway wall):
 *   dPhi/dx|wall = (-8 Phi_w + 9 Phi_0 - Phi_1) / 3  (left), mirrored on the right.
 * Nu(y) = -L dT/dx / dT with L = nx; the mean is the midpoint rule over the ny rows. */
void or_nusselt_sherwood(const or_state* s, double out[4])
{
    const or_params* p = &s->p;
    int nx = p->nx, ny = p->ny;
    size_t n = s->n;
    double* T = (double*)malloc(n * sizeof(double));
    double* C = (double*)malloc(n * sizeof(double));
    or_fields(s, NULL, NULL, T, C, NULL);
    double dT = p->Tw[0] - p->Tw[1], dC = p->Cw[0] - p->Cw[1];
    double nuL = 0, shL = 0, nuR = 0, shR = 0;
    if (p->nee) {
        /* nodes on the walls: dPhi/dx|wall = (-3 Phi_0 + 4 Phi_1 - Phi_2) / 2 (left),
         * mirrored on the right; L = nx - 1; trapezoidal mean over y in [0, ny - 1] */
        const double L = (double)(nx - 1);
        for (int j = 0; j < ny; ++j) {
            const double* Tr = T + (size_t)j * nx;
            const double* Cr = C + (size_t)j * nx;
            const double wj = (j == 0 || j == ny - 1) ? 0.5 : 1.0;
            nuL += wj * -L * (-3.0 * Tr[0] + 4.0 * Tr[1] - Tr[2]) / 2.0 / dT;
            shL += wj * -L * (-3.0 * Cr[0] + 4.0 * Cr[1] - Cr[2]) / 2.0 / dC;
            nuR += wj * -L * (3.0 * Tr[nx - 1] - 4.0 * Tr[nx - 2] + Tr[nx - 3]) / 2.0 / dT;
            shR += wj * -L * (3.0 * Cr[nx - 1] - 4.0 * Cr[nx - 2] + Cr[nx - 3]) / 2.0 / dC;
        }
        out[0] = nuL / (ny - 1); out[1] = shL / (ny - 1);
        out[2] = nuR / (ny - 1); out[3] = shR / (ny - 1);
        free(T);
        free(C);
        return;
    }
    for (int j = 0; j < ny; ++j) {
        const double* Tr = T + (size_t)j * nx;
        const double* Cr = C + (size_t)j * nx;
        double dTdx_L = (-8.0 * p->Tw[0] + 9.0 * Tr[0] - Tr[1]) / 3.0;
        double dCdx_L = (-8.0 * p->Cw[0] + 9.0 * Cr[0] - Cr[1]) / 3.0;
        double dTdx_R = (8.0 * p->Tw[1] - 9.0 * Tr[nx - 1] + Tr[nx - 2]) / 3.0;
        double dCdx_R = (8.0 * p->Cw[1] - 9.0 * Cr[nx - 1] + Cr[nx - 2]) / 3.0;
        nuL += -nx * dTdx_L / dT;
        shL += -nx * dCdx_L / dC;
        nuR += -nx * dTdx_R / dT;
        shR += -nx * dCdx_R / dC;
    }
    out[0] = nuL / ny; out[1] = shL / ny; out[2] = nuR / ny; out[3] = shR / ny;
    free(T);
    free(C);
}

void or_nusselt_sherwood_tb(const or_state* s, double out[4])
{
    const or_params* p = &s->p;
    int nx = p->nx, ny = p->ny;
    size_t n = s->n;
    double* T = (double*)malloc(n * sizeof(double));
    double* C = (double*)malloc(n * sizeof(double));
    or_fields(s, NULL, NULL, T, C, NULL);
    double dT = p->Tw[3] - p->Tw[2], dC = p->Cw[3] - p->Cw[2];
    double nuB = 0, shB = 0, nuT = 0, shT = 0;
    if (p->nee) {
        /* as the left / right walls, transposed: L = ny - 1, trapezoidal mean over x */
        const double L = (double)(ny - 1);
        for (int i = 0; i < nx; ++i) {
            const double wi = (i == 0 || i == nx - 1) ? 0.5 : 1.0;
            const double* t0 = T + i;
            const double* c0 = C + i;
            const size_t r = (size_t)nx, top = (size_t)(ny - 1) * nx;
            nuB += wi * L * (-3.0 * t0[0] + 4.0 * t0[r] - t0[2 * r]) / 2.0 / dT;
            shB += wi * L * (-3.0 * c0[0] + 4.0 * c0[r] - c0[2 * r]) / 2.0 / dC;
            nuT += wi * L * (3.0 * t0[top] - 4.0 * t0[top - r] + t0[top - 2 * r]) / 2.0 / dT;
            shT += wi * L * (3.0 * c0[top] - 4.0 * c0[top - r] + c0[top - 2 * r]) / 2.0 / dC;
        }
        out[0] = nuB / (nx - 1); out[1] = shB / (nx - 1);
        out[2] = nuT / (nx - 1); out[3] = shT / (nx - 1);
        free(T);
        free(C);
        return;
    }
    for (int i = 0; i < nx; ++i) {
        double T0 = T[i], T1 = T[(size_t)nx + i];
        double C0 = C[i], C1 = C[(size_t)nx + i];
        double Tn = T[(size_t)(ny - 1) * nx + i], Tm = T[(size_t)(ny - 2) * nx + i];
        double Cn = C[(size_t)(ny - 1) * nx + i], Cm = C[(size_t)(ny - 2) * nx + i];
        nuB += ny * (-8.0 * p->Tw[2] + 9.0 * T0 - T1) / 3.0 / dT;
        shB += ny * (-8.0 * p->Cw[2] + 9.0 * C0 - C1) / 3.0 / dC;
        nuT += ny * (8.0 * p->Tw[3] - 9.0 * Tn + Tm) / 3.0 / dT;
        shT += ny * (8.0 * p->Cw[3] - 9.0 * Cn + Cm) / 3.0 / dC;
    }
    out[0] = nuB / nx; out[1] = shB / nx; out[2] = nuT / nx; out[3] = shT / nx;
    free(T);
    free(C);
}

void or_stream_function(const or_state* s, double* psi)
{
    const or_params* p = &s->p;
    const int nx = p->nx, ny = p->ny;
    double* ux = (double*)malloc(s->n * sizeof(double));
    or_fields(s, ux, NULL, NULL, NULL, NULL);
    for (int i = 0; i < nx; ++i) {
        /* from the wall node (psi = 0), or from the halfway wall at distance 1/2 below
         * node 0 where u = 0: the trapezoid over that half spacing is u_0 / 4 */
        double acc = p->nee ? 0.0 : 0.25 * ux[i];
        psi[i] = acc;
        for (int j = 1; j < ny; ++j) {
            acc += 0.5 * (ux[(size_t)(j - 1) * nx + i] + ux[(size_t)j * nx + i]);
            psi[(size_t)j * nx + i] = acc;
        }
    }
    free(ux);
}

/* ---- steady-state residual ---------------------------------------------------------
 * The steady runs of Sec. 4 (Tables 1-5) stop when the fields no longer change.  The
 * paper does not state its test; the reading taken is the relative change of the
 * four fields over the last k steps,
 *   r = max over phi in {u_x, u_y, T, C} of  max_x |phi_now(x) - phi_prev(x)| / max_x |phi_now(x)|,
 * with T and C the absolute values of Eq. 26 and u from Eq. 18.  A field that is zero
 * everywhere now contributes 0 if it did not change and +inf if it did.
 * now, prev: planes [4][n] holding (u_x, u_y, T, C).  Returns 1 if a value of now is
 * not finite (the run has diverged), else 0. */
int or_residual_fields(long n, const double* now, const double* prev, double* r)
{
    int bad = 0;
    double res = 0.0;
    for (int q = 0; q < 4; ++q) {
        const double* a = now + (size_t)q * n;
        const double* b = prev + (size_t)q * n;
        double dmax = 0.0, amax = 0.0;
        for (long x = 0; x < n; ++x) {
            if (!isfinite(a[x])) bad = 1;
            const double d = fabs(a[x] - b[x]);
            if (d > dmax) dmax = d;
            if (fabs(a[x]) > amax) amax = fabs(a[x]);
        }
        double rq;
        if (amax > 0.0)
            rq = dmax / amax;
        else
            rq = dmax > 0.0 ? INFINITY : 0.0;
        if (rq > res) res = rq;
    }
    *r = res;
    return bad;
}

/* The residual of the current state against the fields an earlier call left in snap
 * ([4][ny][nx]: u_x, u_y, T, C), which is then overwritten with the current fields.
 * have_snap = 0: snap holds nothing yet and r = +inf.  Returns 1 if a current field
 * value is not finite, else 0. */
int or_residual(const or_state* s, double* snap, int have_snap, double* r)
{
    const size_t n = s->n;
    double* now = (double*)malloc(4 * n * sizeof(double));
    or_fields(s, now, now + n, now + 2 * n, now + 3 * n, NULL);
    int bad = or_residual_fields((long)n, now, snap, r);
    if (!have_snap) *r = INFINITY;
    memcpy(snap, now, 4 * n * sizeof(double));
    free(now);
    return bad;
}

void or_get(const or_state* s, double* f, double* g, double* h, double* hist)
{
    size_t n = s->n;
    if (f) memcpy(f, s->f, 9 * n * sizeof(double));
    if (g) memcpy(g, s->g, 5 * n * sizeof(double));
    if (h) memcpy(h, s->h, 5 * n * sizeof(double));
    if (hist) memcpy(hist, s->hist, 4 * n * sizeof(double));
}

void or_set(or_state* s, const double* f, const double* g, const double* h, const double* hist)
{
    size_t n = s->n;
    if (f) memcpy(s->f, f, 9 * n * sizeof(double));
    if (g) memcpy(s->g, g, 5 * n * sizeof(double));
    if (h) memcpy(s->h, h, 5 * n * sizeof(double));
    if (hist) memcpy(s->hist, hist, 4 * n * sizeof(double));
}

void or_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

int or_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
