/*
 * FP64 CPU oracle for the REV-scale MRT lattice Boltzmann model of
 * double-diffusive convection in porous media (Liu & He, arXiv:1708.07525).
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the plain, slow, obviously correct
 * statement of what one time step computes; it exists so that the CUDA path
 * can be checked against it.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant with the GPU library, and never includes anything from
 * it.
 *
 * What it follows (section / equation of the paper):
 *   - D2Q9 flow lattice, MRT collision in moment space        Sec. 3.1, Eqs. 8-15
 *   - density and velocity, explicit velocity closed form      Eqs. 16-19
 *   - Brinkman-Forchheimer total force and buoyancy            Sec. 2, Eqs. 5-7
 *   - D2Q5 temperature / concentration MRT collisions with the
 *     modified equilibrium moments and source terms            Sec. 3.2, Eqs. 21-27
 *   - optionally the coupled "model A" equilibria (negative
 *     control of Sec. 3.2)                                     Eqs. 30-32
 *   - streaming in velocity space                              Eq. 11
 *   - optional walls with nodes on them: non-equilibrium
 *     extrapolation and gradient extrapolation                Sec. 3.3, Eqs. 33-37
 *   - convective (Robin) walls                                 Sec. 4.2, Eq. 39
 *   - Nusselt / Sherwood numbers                               Sec. 4.1, Eq. 38
 *   - steady-state residual (stopping test of the steady runs)  Sec. 4 (reading below)
 *   - parameter mapping from Ra, Pr, Le, Da, Ma                Sec. 4 and 4.1
 * Readings where the paper is silent (all stated again beside the code):
 *   - walls (default): no-slip halfway bounce-back for f; anti-bounce-back
 *     (Dirichlet) and bounce-back (adiabatic) for g, h.  The cavity workloads
 *     specify halfway walls.
 *   - walls (nee = 1): the paper's own scheme (Sec. 3.3) with nodes on the
 *     walls.  Each step streams, then rebuilds the full sets f, g, h of every
 *     wall node by Eqs. 33-35 from the nearest interior node along the inward
 *     normal (the diagonal one at a corner); the rebuilt node then collides
 *     like any other.  Wall T / C: the Dirichlet value, else Eqs. 36-37 along
 *     the same link, where a convective wall (Eq. 39) enters as
 *     dPhi/dn = -(Bi / L)(Phi - Phi_ambient) along the outward normal (the sign
 *     the paper leaves implicit: heat leaves through the wall); at a corner the
 *     Dirichlet wall wins, else both walls' gradients enter.  The state at
 *     t = 0 is rebuilt the same way.
 *   - Robin / convective wall, Eq. 39: Bi = h L / alpha_e with L the cavity
 *     width nx - 1 on every side.
 *   - the time derivative of T*u in Eq. 27 is the explicit backward
 *     difference the paper suggests (Sec. 3.2), with the history initialised
 *     to T*u of the initial state, so the source vanishes at the first step.
 *   - initial noise: SplitMix64 (Steele, Lea & Flood 2014), see or_uniform().
 *   - steady state: the paper states no test; the relative change of u_x, u_y,
 *     T, C over the last k steps is taken (or_residual).
 *
 * Parity status: every function here is pinned by tests under tests/
 * (identities between the paper's moment- and velocity-space forms,
 * conservation, exact conduction profiles, Brinkman channels, Tables 1-4;
 * for nee: exact Dirichlet and convective conduction profiles, the channel's
 * second-order convergence, Sec. 3.2's T = C at Le = 1 and Tables 2-3).
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_DIRICHLET = 0, OR_ADIABATIC = 1 };

typedef struct {
    /* grid (nodes); walls sit half a spacing outside the outermost nodes */
    int nx, ny;
    /* physical inputs (Sec. 2, dimensionless groups) */
    double Ra, Da, eps, Pr, Le, N, J, sigma, Ma, varpi;
    /* derived lattice quantities (filled by or_derive, may be edited by tests) */
    double rho0, cs2, U, nu, nu_e, alpha_e, D_e, csT2, K, Feps, gbT, gbC, T0, C0;
    double s[9];      /* Lambda = diag(s_rho, s_e, s_eps, s_j, s_q, s_j, s_q, s_nu, s_nu) */
    double zeta[5];   /* Theta  = diag(zeta_0, zeta_a, zeta_a, zeta_e, zeta_eps) */
    double eta[5];    /* Q      = diag(eta_0, eta_D, eta_D, eta_e, eta_eps) */
    /* boundary and test knobs */
    int periodic_x, periodic_y;
    int scalar_lr, scalar_tb;   /* OR_DIRICHLET / OR_ADIABATIC for g and h */
    double Tw[4], Cw[4];        /* Dirichlet values by side: [0] left (x = 0), [1] right (x = nx),
                                   [2] bottom (y = 0), [3] top (y = ny) */
    double uw[4][2];            /* wall velocity (x, y) by side; 0 for resting walls */
    double Gx;                  /* constant external body force along x (enters as eps*G) */
    int model_a;                /* 1: the coupled equilibria of Eqs. 30-31 ("model A"), whose
                                   diffusivities follow Eq. 32; 0: Eqs. 24-25 (the paper's model) */
    int nee;                    /* 0: halfway walls (half a spacing outside the outermost nodes);
                                   1: the outermost nodes lie on the walls, which follow the
                                   non-equilibrium extrapolation of Sec. 3.3 (Eqs. 33-37); the
                                   cavity width is then L = nx - 1 (an input of or_derive) */
    double BiT[4], BiC[4];      /* nee only: a side with Bi > 0 is a convective (Robin) wall,
                                   Eq. 39: dPhi/dn = -(Bi / L) (Phi - Phi_w) along the outward
                                   normal n, Phi_w = Tw / Cw of that side the ambient value;
                                   Bi = 0 keeps the side's Dirichlet / adiabatic kind */
} or_params;

typedef struct or_state or_state;

/* Fill the derived fields of p from nx, Ra, Da, eps, Pr, Le, N, J, sigma, Ma, varpi
 * and nee (L = nx, or nx - 1 when nee).  The wall knobs are reset (BiT = BiC = 0).
 * Returns 0 on success, nonzero if a relaxation rate leaves (0,2) or an input is invalid. */
int or_derive(or_params* p);

/* Create a state at t = 0: f = f_eq(rho0, u=0), g = g_eq(T, 0), h = h_eq(C, 0), where
 * T = T0 + noise*(2U-1), C = C0 + noise*(2U'-1) from SplitMix64(seed), unless T_init /
 * C_init (row-major [ny][nx]) are given.  History = (T u, C u) at t = 0. */
or_state* or_create(const or_params* p, uint64_t seed, double noise,
                    const double* T_init, const double* C_init);
/* The same with a porosity field eps[ny][nx] and a permeability field K[ny][nx]
 * (either may be NULL: then p->eps / p->K everywhere).  At every node the model of
 * Sec. 2-3 is applied with that node's eps, K and F_eps = 1.75 / sqrt(150 eps^3)
 * (Eq. 7), i.e. the REV model with spatially varying porous properties. */
or_state* or_create_field(const or_params* p, uint64_t seed, double noise, const double* T_init,
                          const double* C_init, const double* eps, const double* K);
void or_destroy(or_state* s);

/* n time steps: collide (Eqs. 10, 21, 22), stream (Eq. 11), wall rules. */
void or_step(or_state* s, long n);
long or_time(const or_state* s);

/* Macroscopic fields at the current time level (pre-collision), row-major [ny][nx].
 * Any pointer may be NULL. u is from Eq. 18, T and C from Eq. 26, rho from Eq. 16. */
void or_fields(const or_state* s, double* ux, double* uy, double* T, double* C, double* rho);

/* Mean Nu and Sh on the left and right walls (Eq. 38), out = {Nu_L, Sh_L, Nu_R, Sh_R};
 * dT = Tw[0] - Tw[1] (hot wall minus cold wall, or minus the ambient of a convective wall). */
void or_nusselt_sherwood(const or_state* s, double out[4]);
/* Mean Nu and Sh on the bottom and top walls, out = {Nu_B, Sh_B, Nu_T, Sh_T}: the wall-normal
 * gradient times L = ny over (Phi_top - Phi_bottom), averaged over the nx columns. */
void or_nusselt_sherwood_tb(const or_state* s, double out[4]);

/* Stream function psi[ny][nx] with u_x = d psi / dy, psi = 0 on the bottom wall:
 * the trapezoidal rule up each column (from the wall node when nee, else from the
 * halfway wall half a spacing below the first node, where u = 0). */
void or_stream_function(const or_state* s, double* psi);

/* Steady-state residual (the stopping test of the steady runs of Sec. 4; the paper states
 * none, the reading taken is): r = max over phi in {u_x, u_y, T, C} of
 * max_x |phi_now - phi_prev| / max_x |phi_now| (absolute T and C; a field that is zero
 * everywhere contributes 0 if unchanged, +inf otherwise).  now / prev are planes [4][n]
 * of (u_x, u_y, T, C).  Returns 1 if a value of now is not finite, else 0. */
int or_residual_fields(long n, const double* now, const double* prev, double* r);
/* The same for the current state against snap ([4][ny][nx], the fields of an earlier
 * call), which is replaced by the current fields; have_snap = 0 gives r = +inf. */
int or_residual(const or_state* s, double* snap, int have_snap, double* r);

/* Copy the distributions out / in, layout [q][ny][nx]; hist is [4][ny][nx] =
 * (T u_x, T u_y, C u_x, C u_y) at the previous collision. */
void or_get(const or_state* s, double* f, double* g, double* h, double* hist);
void or_set(or_state* s, const double* f, const double* g, const double* h, const double* hist);

/* One node's collision, for brute-force checks.  hist is read and updated.
 * mac = {rho, ux, uy, T, C, Fx, Fy}. */
void or_collide_node(const or_params* p, const double f[9], const double g[5],
                     const double h[5], double hist[4], double fs[9], double gs[5],
                     double hs[5], double mac[7]);

/* The k-th SplitMix64 output of a generator seeded with `seed`, as a double in [0,1). */
double or_uniform(uint64_t seed, uint64_t k);

/* Initial T and C (1/2 + noise (2U - 1), U = or_uniform with key (field ny + j) nx + i)
 * of the window [x0, x0 + w) x [y0, y0 + h) of an nx x ny cavity, into [h][w] arrays. */
void or_noise_window(uint64_t seed, double noise, int nx, int ny, int x0, int y0, int w, int h,
                     double* T, double* C);

void or_set_threads(int n);
int or_get_threads(void);

#ifdef __cplusplus
}
#endif
#endif
