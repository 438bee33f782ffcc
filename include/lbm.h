/*
 * liblbm -- C ABI of the GB300 (sm_103a) implementation of the REV-scale
 * multiple-relaxation-time lattice Boltzmann model for double-diffusive
 * convection in fluid-saturated porous media (Liu & He, arXiv:1708.07525).
 *
 * One cavity ("context") holds three lattices on the device:
 *   f  D2Q9 flow distributions           (Sec. 3.1, Eqs. 8-20)
 *   g  D2Q5 temperature distributions    (Sec. 3.2, Eqs. 21, 23, 24, 26-28)
 *   h  D2Q5 concentration distributions  (Sec. 3.2, Eqs. 22, 23, 25-28)
 * plus four history values per node (T u, C u at the previous step) for the
 * explicit time derivative in the source terms of Eq. 27.
 *
 * One time step = one fused pass over the nodes (one kernel launch, or two
 * where the outermost ring of nodes has a launch of its own): pull-streaming
 * (Eq. 11) with the wall rules, macroscopic fields (Eqs. 16, 18-19, 26), total
 * force (Eqs. 5-6), the D2Q9 collision in moment space (Eq. 10 with Eqs.
 * 12-15) and the two D2Q5 collisions (Eqs. 21-22 with Eqs. 24-25, 27).
 *
 * Cavity (default walls): nodes (i, j), 0 <= i < nx, 0 <= j < ny, at positions
 * (i+1/2, j+1/2); walls at x = 0, x = nx, y = 0, y = ny, halfway between the
 * outermost nodes and their missing neighbours.  Left wall T = C = 1, right
 * wall T = C = 0, top and bottom adiabatic and impermeable, all walls no-slip:
 * halfway bounce-back (f), anti-bounce-back (Dirichlet g, h) and bounce-back
 * (adiabatic g, h).  With lbm_params.nee = 1 the outermost nodes lie on the
 * walls instead and follow the paper's own scheme (Sec. 3.3, Eqs. 33-37),
 * with convective walls (Eq. 39) available.
 *
 * Conventions for every entry point:
 *   - Returns an lbm_status; never aborts, exits or traps.  The message of the
 *     last failure is available from lbm_last_error().
 *   - Host arrays are caller-owned, row-major [ny][nx] doubles unless stated.
 *   - Device memory is owned by the library (through the caller's allocator
 *     hooks when given) and released by lbm_destroy().
 *   - Work is enqueued on the context's stream; calls that return host data
 *     synchronise that stream.
 *   - A context must not be used from two host threads at once.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
    LBM_OK = 0,
    LBM_ERR_INVALID = 1,      /* bad argument or parameter set */
    LBM_ERR_NOMEM = 2,        /* device or host allocation failed */
    LBM_ERR_CUDA = 3,         /* a CUDA runtime call failed; see lbm_last_error() */
    LBM_ERR_DIVERGED = 4,     /* NaN / Inf found by a reduction */
    LBM_ERR_TIMEOUT = 5,      /* a bounded device-side wait gave up */
    LBM_ERR_UNCONVERGED = 6   /* step cap reached before the residual tolerance */
} lbm_status;

/* Storage precision of the 19 distributions.  F64 computes in FP64; the
 * others compute in FP32.  All store deviations from the rest equilibria
 * f_i - f_i^eq(rho0, 0), g_i - g_i^eq(T0, 0), h_i - h_i^eq(C0, 0) (Eqs. 20, 28). */
enum { LBM_F64 = 0, LBM_F32 = 1, LBM_BF16 = 2, LBM_F16 = 3 };
/* Memory pattern: two buffers with pull streaming, or one buffer in place (AA). */
enum { LBM_AB_PULL = 0, LBM_AA = 1 };
/* Wall type of the scalar fields g, h on a pair of walls. */
enum { LBM_WALL_DIRICHLET = 0, LBM_WALL_ADIABATIC = 1 };

typedef struct {
    int nx, ny;                 /* lattice nodes; both >= 3 */
} lbm_grid;

/* Device allocator hooks: alloc(bytes, user, stream) returns a device pointer
 * aligned to at least 256 bytes, or NULL; free(ptr, user, stream). */
typedef void* (*lbm_alloc_fn)(size_t bytes, void* user, void* stream);
typedef void (*lbm_free_fn)(void* ptr, void* user, void* stream);

/* Options; a zero-initialised struct (or NULL) selects the paper's defaults. */
typedef struct {
    int precision;              /* LBM_F64 (default) | LBM_F32 | LBM_BF16 | LBM_F16 */
    int layout;                 /* LBM_AB_PULL (default) | LBM_AA */
    double Ma;                  /* Mach number U / c_s, 0 -> 0.1 (Sec. 4.1) */
    double varpi;               /* D2Q5 weight parameter, 0 -> 2/5 (Sec. 4) */
    uint64_t seed;              /* initial-noise seed (SplitMix64) */
    double noise;               /* amplitude of the uniform initial noise on T and C;
                                   negative -> 0, zero -> default 1e-3 */
    const double* T_init;       /* optional host [ny][nx] initial T (overrides noise) */
    const double* C_init;       /* optional host [ny][nx] initial C */
    void* stream;               /* cudaStream_t; NULL -> the library creates its own */
    lbm_alloc_fn alloc;         /* NULL -> cudaMalloc / cudaFree */
    lbm_free_fn free;
    void* alloc_user;
    int block_x, block_y;       /* launch tile of the step kernel: block_x a multiple of 32,
                                   block_x * block_y <= 256; 0 -> tuned default */
    int graph_chunk;            /* steps per captured CUDA graph; 0 -> default, <0 -> off */
    const double* eps_field;    /* optional host [ny][nx] porosity field: the REV model with
                                   spatially varying eps (Sec. 2-3 applied per node, F_eps of
                                   Eq. 7 per node); values in (0, 1]; NULL -> uniform eps */
    const double* K_field;      /* optional host [ny][nx] permeability field (> 0); NULL ->
                                   uniform K.  Not with model_a.  Copied at create. */
    int round_nearest;          /* 16-bit storage: 0 (default) -> stochastic rounding of every
                                   stored population (unbiased; random bits hashed from the
                                   node index and its pre-collision state, so runs are
                                   reproducible); 1 -> round to nearest even */
} lbm_options;

/* Derived lattice constants (Sec. 4 / 4.1 mapping).  Filled by
 * lbm_derive_params() from the dimensionless groups, or by the caller for
 * lbm_create_raw().  Units: lattice (delta_x = delta_t = 1, rho0 = 1). */
typedef struct {
    int nx, ny;
    double eps;                 /* porosity phi of Eqs. 2-5 */
    double sigma;               /* heat capacity ratio of Eq. 3 */
    double varpi;               /* D2Q5 model parameter (Eq. 24), c_sT^2 = varpi / 2 */
    double nu;                  /* fluid viscosity in the Darcy term of Eq. 5 */
    double K;                   /* permeability, K = Da L^2 */
    double Feps;                /* Forchheimer coefficient, Eq. 7 */
    double gbT, gbC;            /* g beta_T dT and g beta_C dC of Eq. 6 */
    double Gx;                  /* extra constant body force along x (0 for cavities) */
    double T0, C0;              /* reference values of Eq. 6 and of the storage shift */
    double s[9];                /* Lambda of Eq. 9 */
    double zeta[5];             /* Theta of Eq. 21 */
    double eta[5];              /* Q of Eq. 22 */
    double Tw[4], Cw[4];        /* Dirichlet wall values by side: [0] left (x = 0),
                                   [1] right (x = nx), [2] bottom (y = 0), [3] top (y = ny) */
    int wall_lr, wall_tb;       /* LBM_WALL_* for g and h on left/right, bottom/top */
    double uw[4][2];            /* velocity (x, y) of each wall side (same order as Tw);
                                   0 = resting no-slip wall; a moving lid bounces populations
                                   back with the momentum 2 w_i rho0 (e_i . u_w) / c_s^2 */
    int model_a;                /* 0: the paper's equilibria (Eqs. 24-25); 1: the coupled
                                   "model A" equilibria of Eqs. 30-31 (a negative control; with
                                   it, Eq. 32 relates zeta, eta to the diffusivities) */
    int nee;                    /* 0: halfway walls half a spacing outside the outermost nodes
                                   (the rules of wall_lr / wall_tb / uw above); 1: the outermost
                                   nodes lie on the walls and follow the paper's own scheme
                                   (Sec. 3.3): after streaming, each wall node's f, g, h are
                                   rebuilt by the non-equilibrium extrapolation of Eqs. 33-35
                                   from the nearest interior node along the inward normal (the
                                   diagonal one at a corner), with the wall velocity uw, and T / C
                                   from the Dirichlet value or the gradient extrapolation of
                                   Eqs. 36-37.  The cavity width is then L = nx - 1.  Needs
                                   nx, ny >= 5 and the two-buffer layout. */
    double BiT[4], BiC[4];      /* nee only: Biot numbers of convective (Robin) walls, Eq. 39.
                                   A side with Bi > 0 takes dPhi/dn = -(Bi / L)(Phi - Phi_w)
                                   along its outward normal n, Phi_w = Tw / Cw of that side as
                                   the ambient value, L = nx - 1; at a corner a Dirichlet wall
                                   wins, else both walls' gradients enter Eq. 36 along the
                                   diagonal.  0: the side keeps its wall_lr / wall_tb kind. */
} lbm_params;

/* Parameter mapping of Sec. 4 and 4.1 (L = nx, c_s^2 = 1/3, U = Ma c_s,
 * nu_e = J U L sqrt(Pr / Ra), alpha_e = nu / Pr, D_e = alpha_e / Le,
 * s_nu, zeta_a, eta_D from Eq. 29 and the nu_e relation of Sec. 3.1,
 * g beta_T = U^2 / L, g beta_C = N g beta_T, K = Da L^2, F_eps of Eq. 7,
 * fixed rates of Sec. 4).  Ma <= 0 -> 0.1, varpi <= 0 -> 0.4.
 * Returns LBM_ERR_INVALID if nx or ny < 3, eps is outside (0, 1], Da, Ra, Pr,
 * Le, J or sigma is not positive, or a relaxation rate leaves (0, 2). */
lbm_status lbm_derive_params(lbm_grid grid, double Ra, double Da, double eps, double Pr,
                             double Le, double N, double J, double sigma, double Ma,
                             double varpi, lbm_params* out);

/* The mapping of lbm_derive_params() for walls with nodes on them (nee = 1):
 * L = nx - 1 (the nx - 1 spacings between the wall nodes), nx, ny >= 5. */
lbm_status lbm_derive_params_nee(lbm_grid grid, double Ra, double Da, double eps, double Pr,
                                 double Le, double N, double J, double sigma, double Ma,
                                 double varpi, lbm_params* out);

/* The porous cavity with a freely convective wall of Sec. 4.2: Nx lattice spacings
 * per side ((Nx + 1) x (Nx + 1) nodes on walls, nee = 1), left wall T = C = 1,
 * right wall convective (Eq. 39) to the ambient T = C = 0 with Biot numbers
 * BiT, BiC, top and bottom adiabatic and impermeable; other groups as in
 * lbm_derive_params() with L = Nx. */
lbm_status lbm_derive_params_convective(int Nx, double Ra, double Da, double eps, double Pr,
                                        double Le, double N, double BiT, double BiC, double J,
                                        double sigma, double Ma, double varpi, lbm_params* out);

/* Parameter mapping of the lid-driven porous cavity of Sec. 4.3: top wall moving
 * with U0 along +x, top T = C = 1 and bottom T = C = 0 (Dirichlet), left and right
 * walls adiabatic; Re = L U0 / nu with 1/s_nu = 1/2 + J L U0 / (c_s^2 Re);
 * Gr = g beta_T dT L^3 / nu^2; Pr, Le, N, Da, eps, sigma as in lbm_derive_params;
 * L = nx.  U0 <= 0 -> 0.1, varpi <= 0 -> 0.4. */
lbm_status lbm_derive_params_lid(lbm_grid grid, double Re, double Gr, double Da, double eps,
                                 double Pr, double Le, double N, double J, double sigma,
                                 double U0, double varpi, lbm_params* out);

/* The lid-driven mapping of lbm_derive_params_lid() for walls with nodes on them
 * (nee = 1, Sec. 3.3): L = nx - 1, nx, ny >= 5; corner nodes of the top wall move
 * with the lid. */
lbm_status lbm_derive_params_lid_nee(lbm_grid grid, double Re, double Gr, double Da, double eps,
                                     double Pr, double Le, double N, double J, double sigma,
                                     double U0, double varpi, lbm_params* out);

/* Switch parameters from lbm_derive_params() to the coupled "model A" equilibria
 * (Eqs. 30-31) with the same effective diffusivities: by Eq. 32,
 * 1/zeta_a = 1/2 + alpha_e / (sigma c_sT^2), 1/eta_D = 1/2 + D_e / (eps c_sT^2).
 * A negative control: the paper's model (Eqs. 24-25, 29) keeps these independent
 * of sigma and eps.  LBM_ERR_INVALID if a rate leaves (0, 2) or p is NULL. */
lbm_status lbm_params_model_a(lbm_params* p);

/* Create a cavity at t = 0: u = 0, rho = rho0, T = C = 1/2 plus uniform noise
 * of amplitude opt->noise drawn by SplitMix64 (Steele, Lea & Flood 2014) with
 * key (field * ny + j) * nx + i (field 0 = T, 1 = C), f = f^eq (Eq. 20),
 * g, h = equilibria of Eq. 28, history = (T u, C u) of that state, so the
 * source of Eq. 27 vanishes at the first step.  On success *out owns the
 * device state.  Errors: LBM_ERR_INVALID (see lbm_derive_params, or out is
 * NULL), LBM_ERR_NOMEM, LBM_ERR_CUDA. */
lbm_status lbm_create(lbm_grid grid, double Ra, double Da, double eps, double Pr, double Le,
                      double N, double J, double sigma, const lbm_options* opt,
                      lbm_ctx** out);

/* Same, from explicit lattice constants (used for analytic test cases). */
lbm_status lbm_create_raw(const lbm_params* params, const lbm_options* opt, lbm_ctx** out);

/* Re-initialise the cavity at t = 0 as lbm_create does, from caller-owned host
 * [ny][nx] initial fields T_init and C_init (both or neither; pinned host memory
 * makes the copy faster), or from the SplitMix64 noise with the given seed and
 * amplitude (noise < 0 -> none, 0 -> 1e-3).  The first call with fields
 * allocates a device staging buffer of 16 nx ny bytes, kept until destroy.
 * Asynchronous on the context's stream; the host arrays must stay valid until
 * the stream has passed this point. */
lbm_status lbm_reset(lbm_ctx* ctx, const double* T_init, const double* C_init, uint64_t seed,
                     double noise);

/* Advance n >= 0 time steps (asynchronous on the context's stream).  On a stream other
 * than the legacy default stream the steps are replayed from CUDA graphs in chunks, and
 * a step that is one kernel goes out as a programmatic dependent launch: its blocks may
 * be placed while the kernel before it on the stream drains, but each waits for that
 * kernel to complete before it touches the state, so work of the caller's on the same
 * stream, before or after, is ordered as in plain stream order. */
lbm_status lbm_step(lbm_ctx* ctx, int64_t n);

/* Number of time steps taken since creation (or since the loaded checkpoint). */
int64_t lbm_time(const lbm_ctx* ctx);

/* Macroscopic fields at the current time level, before collision:
 * u from Eq. 18, T and C from Eq. 26, rho from Eq. 16.  Caller-owned host
 * arrays [ny][nx]; any pointer may be NULL.  Synchronises the stream. */
lbm_status lbm_fields(lbm_ctx* ctx, double* ux, double* uy, double* T, double* C,
                      double* rho);

/* The same fields over the window of nodes [x0, x0 + w) x [y0, y0 + h) only, into
 * caller-owned host arrays [h][w] (for grids too large to copy whole).
 * LBM_ERR_INVALID if the window leaves the grid or h > 65535. */
lbm_status lbm_fields_window(lbm_ctx* ctx, int x0, int y0, int w, int h, double* ux, double* uy,
                             double* T, double* C, double* rho);

/* Mean Nusselt and Sherwood numbers on the left and right walls (Eq. 38),
 * out = {Nu_L, Sh_L, Nu_R, Sh_R}, reduced in FP64.  The wall gradient is the
 * second-order one-sided difference through the wall value and the two
 * nearest nodes, (-8 T_w + 9 T_0 - T_1) / 3 on the left, mirrored on the
 * right; Nu(y) = -L dT/dx / dT with L = nx; the mean is over the ny rows.
 * Synchronises the stream.  LBM_ERR_DIVERGED if a result is not finite. */
lbm_status lbm_nusselt_sherwood(lbm_ctx* ctx, double out[4]);

/* Mean Nu and Sh on the bottom and top walls: the wall-normal gradient (same
 * one-sided stencil) times L = ny over (top value - bottom value), averaged over
 * the nx columns; out = {Nu_B, Sh_B, Nu_T, Sh_T}, FP64.  Synchronises. */
lbm_status lbm_nusselt_sherwood_tb(lbm_ctx* ctx, double out[4]);

/* Steady-state residual: r = max over phi in {u_x, u_y, T, C} of
 * max|phi_now - phi_snap| / max|phi_now|, where phi_snap is the snapshot of
 * the previous call (r = +inf on the first call); the snapshot is then
 * replaced by phi_now.  Per node the differences are taken in the compute
 * precision (FP64 for FP64 storage, else FP32) on u_x, u_y, T - T0 and C - C0,
 * so that the difference of two close values is exact; the maxima and the
 * ratio are reduced in FP64.  Synchronises the stream.
 * LBM_ERR_DIVERGED if a field value is not finite. */
lbm_status lbm_residual(lbm_ctx* ctx, double* r);

/* The maxima behind lbm_residual(), for combining several contexts (the slabs of
 * one cavity): parts[q] = max |phi_now - phi_snap| and parts[4 + q] = max |phi_now|
 * for phi = u_x, u_y, T, C (q = 0..3) over this context's rows; parts[0..3] = +inf
 * on the first call.  The residual of the whole cavity is
 * max over q of (max over slabs of parts[q]) / (max over slabs of parts[4 + q]).
 * Replaces the snapshot as lbm_residual() does.  Synchronises the stream.
 * LBM_ERR_DIVERGED if a field value is not finite. */
lbm_status lbm_residual_parts(lbm_ctx* ctx, double parts[8]);

/* Checkpoint of the full state (distributions, history, time, parameters).
 * lbm_save with buf == NULL stores the size needed in *len.  lbm_load
 * requires a checkpoint of a context with the same grid and layout; a
 * checkpoint of another storage precision is converted on the host: each
 * stored deviation (f_i - f_i^eq(rho0, 0) etc., Eqs. 20, 28) and history value
 * is taken to FP64 and stored in this context's precision (exact when
 * widening, e.g. an FP32 state polished further in FP64; rounded to nearest
 * when narrowing).  Both synchronise the stream. */
lbm_status lbm_save(lbm_ctx* ctx, void* buf, size_t* len);
lbm_status lbm_load(lbm_ctx* ctx, const void* buf, size_t len);

/* ---- A cavity split along y into slabs ---------------------------------------
 * One cavity of params->nx x params->ny nodes may be cut into slabs of whole rows,
 * e.g. one per GPU.  Streaming (Eq. 11) pulls the populations with e_y = +1
 * (f2, f5, f6, g2, h2) across a cut from the row below it and those with e_y = -1
 * (f4, f7, f8, g4, h4) from the row above, so after every time step each slab sends
 * those five values per column of its outermost rows to its neighbours, which
 * store them in a ghost row beside the cut; the collision and everything else is
 * local to a node.  With those exchanges after every step the slabs reproduce the
 * undivided cavity's run bit for bit.  Slabs take halfway walls, the two-buffer
 * layout and a uniform porous medium; any storage precision.
 *
 * lbm_create_slab: the slab of rows [y0, y0 + h) of the cavity described by params
 * (the whole cavity's constants, e.g. from lbm_derive_params(); walls only where the
 * slab meets the cavity's walls).  The initial noise takes the values those rows have
 * in the whole cavity; T_init / C_init of opt are [h][nx].  Row j of lbm_fields(),
 * lbm_fields_window() is the cavity's row y0 + j; lbm_nusselt_sherwood() gives the
 * means over the slab's rows (the cavity's mean is the h-weighted mean over slabs);
 * lbm_nusselt_sherwood_tb() is not defined on a slab (LBM_ERR_INVALID); for the
 * residual of the whole cavity combine lbm_residual_parts() of all slabs.
 * LBM_ERR_INVALID for rows outside the cavity, walls with nodes on them, the in-place
 * layout or porous fields. */
lbm_status lbm_create_slab(const lbm_params* params, int y0, int h, const lbm_options* opt,
                           lbm_ctx** out);

/* Bytes of one face: the five crossing populations of each of the nx columns, in the
 * storage precision (5 * nx * element size), laid out [5][nx]. */
lbm_status lbm_halo_bytes(const lbm_ctx* ctx, size_t* bytes);

/* side 0: the cut below the slab, 1: the cut above it.  lbm_halo_export copies the
 * populations of the slab's outermost row on that side that cross the cut (the
 * post-collision values of the last step) into the caller-owned device buffer face;
 * lbm_halo_import copies the neighbour's face (its export toward this slab) into the
 * ghost row on that side.  Both are asynchronous on the context's stream (order them
 * after the neighbour's export with events, or synchronise).  Call them between steps:
 * after lbm_step(ctx, 1) on every slab, export on every slab, then import on every slab.
 * LBM_ERR_INVALID if that side of the slab is a wall of the cavity. */
lbm_status lbm_halo_export(lbm_ctx* ctx, int side, void* face);
lbm_status lbm_halo_import(lbm_ctx* ctx, int side, const void* face);

/* Parameters in use, and bytes of device memory the context holds. */
lbm_status lbm_get_params(const lbm_ctx* ctx, lbm_params* out);
size_t lbm_device_bytes(const lbm_ctx* ctx);

/* ---- Many cavities in one launch ------------------------------------------
 * A batch holds cavities of different sizes and parameters in one device arena
 * and advances all of them with one fused launch per time step (the same
 * per-node work as lbm_step: Sec. 3, Eqs. 5-27), tiled per cavity and captured
 * in CUDA graphs.  All cavities of a batch share the storage precision and the
 * memory pattern given in lbm_options; the per-cavity noise seed and amplitude
 * come from the descriptors.  Results of a cavity do not depend on the other
 * members of the batch (bitwise).  Cavities with wall nodes (lbm_params.nee,
 * Sec. 3.3, convective walls included) may join two-buffer batches; moving
 * walls and porosity fields are single-cavity features. */
typedef struct lbm_batch lbm_batch;

typedef struct {
    lbm_params params;          /* from lbm_derive_params() or written by the caller */
    uint64_t seed;              /* initial-noise seed of this cavity */
    double noise;               /* noise amplitude (<0 none, 0 -> 1e-3) */
} lbm_instance;

/* Create a batch with room for `capacity` cavities in a device arena of
 * `arena_bytes` (0 -> exactly what the `count` initial cavities need; then
 * nothing more can be added).  The first `count` cavities of `inst` (may be 0)
 * are added at t = 0.  Errors: LBM_ERR_INVALID, LBM_ERR_NOMEM, LBM_ERR_CUDA. */
lbm_status lbm_batch_create(const lbm_instance* inst, int count, int capacity,
                            size_t arena_bytes, const lbm_options* opt, lbm_batch** out);

/* Bytes of arena one cavity of this grid needs in a batch with these options. */
size_t lbm_batch_instance_bytes(lbm_grid grid, const lbm_options* opt);

/* Add one cavity at the batch's current time; *slot receives its index.
 * LBM_ERR_NOMEM if no free slot or no arena block is large enough (the arena is
 * the admission budget). */
lbm_status lbm_batch_add(lbm_batch* b, const lbm_instance* inst, int* slot);

/* Remove a cavity and return its arena block; its slot becomes free. */
lbm_status lbm_batch_remove(lbm_batch* b, int slot);

/* Advance every cavity of the batch by n time steps (asynchronous). */
lbm_status lbm_batch_step(lbm_batch* b, int64_t n);

/* Steps taken by the cavity in `slot` since it was added (-1 if the slot is free). */
int64_t lbm_batch_time(const lbm_batch* b, int slot);

/* Mean Nu/Sh (Eq. 38) of every slot: out[4 * slot + k] as in lbm_nusselt_sherwood
 * (zeros for free slots); out has 4 * capacity doubles.  Synchronises. */
lbm_status lbm_batch_nusselt_sherwood(lbm_batch* b, double* out);

/* Residual (as lbm_residual) of every slot against its previous call: r has
 * `capacity` doubles (+inf on a cavity's first call, 0 for free slots);
 * diverged[slot] (may be NULL) is set to 1 for cavities with non-finite values.
 * Synchronises. */
lbm_status lbm_batch_residual(lbm_batch* b, double* r, int* diverged);

/* Fields of one cavity, as lbm_fields.  Synchronises. */
lbm_status lbm_batch_fields(lbm_batch* b, int slot, double* ux, double* uy, double* T, double* C,
                            double* rho);

/* Choose the tile shape of every grid size present in the batch by timing
 * candidate shapes (128-node tiles 32, 64 or 128 wide) over `trial_steps` steps on
 * scratch cavities of that size (the batch's own state is not touched), and
 * apply them.  The choice is cached per (nx, ny, precision, layout) for the
 * process and used by later batches.  report (may be NULL, `cap` chars)
 * receives one line per size: "nx ny tile_w tile_h us_per_step". */
lbm_status lbm_batch_autotune(lbm_batch* b, int trial_steps, char* report, size_t cap);

/* Set the tile shape of one cavity by hand (tile_w a power of two in 32..256,
 * tile_h >= 1, tile_w * tile_h <= 4096).  Results do not depend on it. */
lbm_status lbm_batch_set_tile(lbm_batch* b, int slot, int tile_w, int tile_h);

/* L2 temporal blocking: cavities are grouped so that the per-step working sets
 * of the two groups in flight stay within l2_bytes (each group's within half of
 * it; 0 -> keep; default 3/8 of the L2), and each group is advanced `steps` steps
 * (default 64) at a time, so that its state is read from L2 rather than HBM on
 * all but the first of them.  The groups are dealt alternately to the batch's
 * stream and a second stream the batch owns (forked from and joined back to
 * the batch's stream, also inside its CUDA graphs), so that one group's launches
 * fill the gaps of the other's.  steps = 1 turns blocking off (one launch over
 * all tiles per step).  Results do not depend on it. */
lbm_status lbm_batch_set_blocking(lbm_batch* b, int steps, size_t l2_bytes);

/* Number of slots, slots in use, and the arena size / bytes in use. */
lbm_status lbm_batch_info(const lbm_batch* b, int* capacity, int* used, size_t* arena_bytes,
                          size_t* arena_used);

void lbm_batch_destroy(lbm_batch* b);
const char* lbm_batch_last_error(const lbm_batch* b);

/* ---- Serving: cavity solves as requests ------------------------------------
 * A server keeps a batch whose arena is the device-memory budget.  Submitted
 * requests wait in a FIFO queue; every tick admits the queued requests whose
 * storage fits in the arena (later requests may fill space an earlier, larger
 * one cannot use), advances every admitted cavity by `check_every` steps with
 * the batch's fused launch, computes each one's residual (lbm_residual), and
 * retires those below their tolerance (status LBM_OK), past their step cap
 * (LBM_ERR_UNCONVERGED) or non-finite (LBM_ERR_DIVERGED), freeing their
 * storage for the next admissions.  Because a cavity's work does not depend
 * on the rest of the batch and checks fall every `check_every` steps after
 * admission, a request's result is the same whatever it was served with. */
typedef struct lbm_server lbm_server;

typedef struct {
    int64_t id;                 /* the caller's request id */
    int status;                 /* LBM_OK, LBM_ERR_UNCONVERGED or LBM_ERR_DIVERGED */
    int64_t steps;              /* time steps taken */
    double residual;            /* last residual */
    double nush[4];             /* Nu_L, Sh_L, Nu_R, Sh_R at the end (Eq. 38) */
    double t_submit, t_admit, t_done;   /* seconds on the server clock */
} lbm_result;

/* budget_bytes: device arena for the cavities' storage; max_slots: cavities in
 * flight at most; check_every: steps per tick (even, >= 2).  Precision, memory
 * pattern, stream and allocator come from opt (FP32, BF16 or FP16 storage). */
lbm_status lbm_server_create(size_t budget_bytes, int max_slots, int check_every,
                             const lbm_options* opt, lbm_server** out);
/* Queue one solve.  It is steady (status LBM_OK) at the first check where the
 * residual over the last check_every steps is below tol (tol > 0), or where every
 * one of Nu_L, Sh_L, Nu_R, Sh_R changed by less than nush_tol relative to its
 * value since the previous check (nush_tol > 0; the Nu/Sh rule averages over a
 * wall and so tolerates the rounding noise of 16-bit storage, which keeps the
 * field residual near 1e-3); else it stops after max_steps steps. */
lbm_status lbm_server_submit(lbm_server* s, const lbm_instance* inst, double tol,
                             double nush_tol, int64_t max_steps, int64_t id);
/* One tick (admit, step, check, retire); *active receives the cavities in flight
 * afterwards (may be NULL).  Synchronises the stream. */
lbm_status lbm_server_tick(lbm_server* s, int* active);
/* Move up to cap finished results to out; *n receives how many. */
lbm_status lbm_server_poll(lbm_server* s, lbm_result* out, int cap, int* n);
/* Seconds since the server was created (the clock of lbm_result). */
double lbm_server_clock(const lbm_server* s);
/* Queue length, cavities in flight, results not yet polled, arena bytes in use. */
lbm_status lbm_server_info(const lbm_server* s, int* queued, int* active, int* done,
                           size_t* arena_used);
void lbm_server_destroy(lbm_server* s);
const char* lbm_server_last_error(const lbm_server* s);

/* Slots of 9 doubles in the fixed scratch of lbm_residual_noalloc(). */
#define LBM_NOALLOC_MAX_BLOCKS 4096

/* The steady-state residual of lbm_residual(), for callers that cannot let the
 * library allocate device memory when they ask for it: code embedded in a host
 * framework that has already reserved the device memory for its own pool, and
 * loops that must not stall, since cudaMalloc and cudaFree can synchronise
 * the whole device.  The paper has no counterpart; this is plumbing.
 *   snapshot       caller-owned device buffer of 4 * nx * ny doubles, planes
 *                  (u_x, u_y, T - T0, C - C0) of [ny][nx] (values of the compute
 *                  precision); read as the previous snapshot and overwritten
 *                  with the current fields.
 *   have_snapshot  0 if snapshot holds no earlier fields (then *r = +inf).
 *   r              host output, defined as in lbm_residual().
 * Allocates nothing: the per-block maxima are folded into one file-scope
 * device array of LBM_NOALLOC_MAX_BLOCKS * 9 + 16 doubles (about 288 KiB), which
 * every GPU that loads the library holds until the process exits; any grid fits
 * (the blocks of the first pass share its slots).  The first call on each
 * device looks up the array's device address and keeps it for the life of the
 * process (a device reset, which unloads the library's device code, makes it
 * stale); make that first call before any stream capture.  The call runs on the
 * context's device whatever device the calling thread has current.  All calls
 * share the array: each call clears it, then folds
 * into it; calls whose work overlaps on the GPU, from any context or stream,
 * race on it.  Synchronises the context's stream.  Errors as for
 * lbm_residual(), plus LBM_ERR_INVALID for NULL arguments. */
lbm_status lbm_residual_noalloc(lbm_ctx* ctx, double* snapshot, int have_snapshot, double* r);

/* Releases everything the context owns.  NULL is ignored. */
void lbm_destroy(lbm_ctx* ctx);

/* Message of the last failure on ctx, or of the calling thread's last
 * failed call that had no context (ctx == NULL).  Never NULL. */
const char* lbm_last_error(const lbm_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
