// C ABI of liblbm (declared in include/lbm.h): context management, parameter
// mapping, stepping with CUDA-graph replay, read-outs, checkpoints.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_launch.h"

using namespace lbm;

namespace {

thread_local std::string g_last_error = "";

void set_global_error(const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

size_t storage_size(int prec) {
    switch (prec) {
        case LBM_F64: return 8;
        case LBM_F32: return 4;
        default: return 2;
    }
}


}  // namespace

namespace lbm {
template <typename R>
Coef<R> make_coef(const lbm_params& P) {
    Coef<R> c;
    std::memset(&c, 0, sizeof c);
    const double eps = P.eps;
    c.T0 = (R)P.T0;
    c.C0 = (R)P.C0;
    c.inv_sigma = (R)(1.0 / P.sigma);
    c.inv_eps = (R)(1.0 / eps);
    c.eps = (R)eps;
    c.half_eps = (R)(0.5 * eps);
    c.inv_eps_f = (R)(1.0 / eps);
    c.gbT = (R)P.gbT;
    c.gbC = (R)P.gbC;
    c.Gx = (R)P.Gx;
    // Eq. 19 with delta_t = 1
    const double l0 = 0.5 * (1.0 + eps * 0.5 * P.nu / P.K);
    const double l1 = eps * 0.5 * P.Feps / std::sqrt(P.K);
    c.l0 = (R)l0;
    c.l0sq = (R)(l0 * l0);
    c.l1 = (R)l1;
    c.drag_lin = (R)(eps * P.nu / P.K);                     // Eq. 5
    c.drag_quad = (R)(eps * P.Feps / std::sqrt(P.K));
    c.s1 = (R)P.s[1]; c.s2 = (R)P.s[2]; c.s3 = (R)P.s[3]; c.s4 = (R)P.s[4];
    c.s5 = (R)P.s[5]; c.s6 = (R)P.s[6]; c.s7 = (R)P.s[7]; c.s8 = (R)P.s[8];
    c.za1 = (R)P.zeta[1]; c.za2 = (R)P.zeta[2]; c.za3 = (R)P.zeta[3]; c.za4 = (R)P.zeta[4];
    c.ed1 = (R)P.eta[1]; c.ed2 = (R)P.eta[2]; c.ed3 = (R)P.eta[3]; c.ed4 = (R)P.eta[4];
    // 1 - s/2 factors of the forcing / source terms (Eqs. 10, 21, 22), in the compute precision
    c.h1 = (R)(1.0 - 0.5 * P.s[1]); c.h2 = (R)(1.0 - 0.5 * P.s[2]);
    c.h3 = (R)(1.0 - 0.5 * P.s[3]); c.h4 = (R)(1.0 - 0.5 * P.s[4]);
    c.h5 = (R)(1.0 - 0.5 * P.s[5]); c.h6 = (R)(1.0 - 0.5 * P.s[6]);
    c.h7 = (R)(1.0 - 0.5 * P.s[7]); c.h8 = (R)(1.0 - 0.5 * P.s[8]);
    c.hz1 = (R)(1.0 - 0.5 * P.zeta[1]); c.hz2 = (R)(1.0 - 0.5 * P.zeta[2]);
    c.he1 = (R)(1.0 - 0.5 * P.eta[1]); c.he2 = (R)(1.0 - 0.5 * P.eta[2]);
    // Eqs. 24 / 25 (model A: Eqs. 30 / 31): n_eq,3 = c3 Phi
    c.c3T = (R)(P.model_a ? (5.0 * P.varpi - 4.0) * P.sigma : 5.0 * P.varpi - 4.0 * P.sigma);
    c.c3C = (R)(P.model_a ? (5.0 * P.varpi - 4.0) * eps : 5.0 * P.varpi - 4.0 * eps);
    const double w = 0.25 * P.varpi;                        // w~_1..4 (Sec. 3.2)
    // anti-bounce-back constant g_q^eq + g_opp^eq at the wall value: 2 w~ Phi_w (Eq. 28),
    // 2 w~ sigma T_w / 2 w~ eps C_w for model A; in deviations from Phi0
    const double kg = P.model_a ? P.sigma : 1.0, kh = P.model_a ? eps : 1.0;
    for (int s = 0; s < 4; ++s) {
        c.wallT[s] = (R)(2.0 * w * kg * (P.Tw[s] - P.T0));
        c.wallC[s] = (R)(2.0 * w * kh * (P.Cw[s] - P.C0));
    }
    c.dirichlet_mask = (P.wall_lr == LBM_WALL_DIRICHLET ? 3 : 0) |
                       (P.wall_tb == LBM_WALL_DIRICHLET ? 12 : 0);
    c.sr = 1;
    c.poro = nullptr;
    c.nu = (R)P.nu;
    c.varpi5 = (R)(5.0 * P.varpi);
    c.moving = 0;
    for (int s = 0; s < 4; ++s)
        for (int d = 0; d < 2; ++d) {
            c.wmom[s][d] = (R)(2.0 * 1.0 * P.uw[s][d] / (1.0 / 3.0));   // 2 rho0 u_w / c_s^2
            if (P.uw[s][d] != 0.0) c.moving = 1;
        }
    // walls with nodes on them (Sec. 3.3)
    c.nee = P.nee;
    const double L = P.nx - 1.0;
    for (int s = 0; s < 4; ++s) {
        c.TwP[s] = (R)(P.Tw[s] - P.T0);
        c.CwP[s] = (R)(P.Cw[s] - P.C0);
        c.bT[s] = (R)(P.nee ? P.BiT[s] / L : 0.0);
        c.bC[s] = (R)(P.nee ? P.BiC[s] / L : 0.0);
        c.uwall[s][0] = (R)P.uw[s][0];
        c.uwall[s][1] = (R)P.uw[s][1];
    }
    const double c3T = P.model_a ? (5.0 * P.varpi - 4.0) * P.sigma : 5.0 * P.varpi - 4.0 * P.sigma;
    const double c3C = P.model_a ? (5.0 * P.varpi - 4.0) * eps : 5.0 * P.varpi - 4.0 * eps;
    c.aT0 = (R)((P.sigma - c3T) / 5.0);
    c.aT1 = (R)(P.sigma / 5.0 + c3T / 20.0);
    c.aC0 = (R)((eps - c3C) / 5.0);
    c.aC1 = (R)(eps / 5.0 + c3C / 20.0);
    return c;
}
template Coef<float> make_coef<float>(const lbm_params&);
template Coef<double> make_coef<double>(const lbm_params&);
template Coef<f2> make_coef<f2>(const lbm_params&);
}  // namespace lbm

namespace {

bool rate_ok(double s) { return s > 0.0 && s < 2.0; }

const char* check_params(const lbm_params& P) {
    if (P.nx < 3 || P.ny < 3) return "nx and ny must be >= 3";
    if (!(P.eps > 0.0 && P.eps <= 1.0)) return "porosity eps must lie in (0, 1]";
    if (!(P.sigma > 0.0)) return "sigma must be positive";
    if (!(P.varpi > 0.0 && P.varpi < 1.0)) return "varpi must lie in (0, 1)";
    if (!(P.K > 0.0)) return "permeability K must be positive";
    if (!(P.nu >= 0.0) || !(P.Feps >= 0.0)) return "nu and F_eps must be non-negative";
    for (int k = 0; k < 9; ++k)
        if (!rate_ok(P.s[k])) return "a flow relaxation rate lies outside (0, 2)";
    for (int k = 0; k < 5; ++k)
        if (!rate_ok(P.zeta[k]) || !rate_ok(P.eta[k]))
            return "a scalar relaxation rate lies outside (0, 2)";
    if (P.wall_lr != LBM_WALL_DIRICHLET && P.wall_lr != LBM_WALL_ADIABATIC) return "bad wall_lr";
    if (P.wall_tb != LBM_WALL_DIRICHLET && P.wall_tb != LBM_WALL_ADIABATIC) return "bad wall_tb";
    if (P.model_a != 0 && P.model_a != 1) return "model_a must be 0 or 1";
    if (P.nee != 0 && P.nee != 1) return "nee must be 0 or 1";
    if (P.nee && (P.nx < 5 || P.ny < 5)) return "walls with nodes on them need nx, ny >= 5";
    for (int k = 0; k < 4; ++k) {
        if (!(P.BiT[k] >= 0.0) || !(P.BiC[k] >= 0.0) || !std::isfinite(P.BiT[k]) ||
            !std::isfinite(P.BiC[k]))
            return "Biot numbers must be finite and >= 0";
        if (!P.nee && (P.BiT[k] > 0.0 || P.BiC[k] > 0.0))
            return "convective (Robin) walls need walls with nodes on them (nee = 1)";
    }
    if ((double)P.nx * (double)P.ny > 4.0e9) return "grid too large";
    return nullptr;
}

}  // namespace

struct lbm_ctx {
    lbm_params P;
    int prec = LBM_F64, layout = LBM_AB_PULL;
    Geom G{};
    size_t esz = 8, rsz = 8;
    void* buf[2] = {nullptr, nullptr};
    void* hist = nullptr;
    double* d_out = nullptr;        // 16 doubles: Nu/Sh and residual results
    double* d_fields = nullptr;     // lazily allocated [5][h][w] read-out window
    size_t fields_cap = 0;          // nodes d_fields holds
    void* d_snap = nullptr;         // lazily allocated [4][ny][nx] in the compute precision
    double* d_partial = nullptr;    // lazily allocated residual partials
    double* d_stage = nullptr;      // lazily allocated [2][ny][nx] initial-field staging
    void* poro = nullptr;           // optional [2][ny][pitch] (eps, K) in the compute precision
    bool snap_valid = false;
    int cur = 0;                    // two-buffer layout: buffer holding the state
    int64_t t = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t aux = nullptr;           // second stream for the ring launches of split steps
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int device = 0;
    int slab_y0 = 0;                // global row of the first updated row (0 for a cavity)
    bool slab = false;              // a slab of a cavity split along y (lbm_create_slab)
    Coef<double> cd{};
    Coef<float> cf{};
    Coef<f2> cp{};                  // 16-bit storage: cf as pairs (two nodes per thread)
    LaunchCfg L{};
    int graph_chunk = 0;
    bool round_nearest = false;     // 16-bit storage: nearest-even instead of stochastic
    cudaGraphExec_t graph = nullptr;
    lbm_alloc_fn alloc = nullptr;
    lbm_free_fn free_fn = nullptr;
    void* alloc_user = nullptr;
    size_t bytes = 0;
    std::string err;

    lbm_status fail(lbm_status s, const char* fmt, ...) {
        char b[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(b, sizeof b, fmt, ap);
        va_end(ap);
        err = b;
        g_last_error = b;
        return s;
    }
    lbm_status cuda_fail(cudaError_t e, const char* where) {
        return fail(LBM_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
    }

    void* dalloc(size_t n) {
        void* p = nullptr;
        if (alloc) {
            p = alloc(n, alloc_user, (void*)stream);
            if (p && ((uintptr_t)p & 255u)) {   // the kernels assume 256-byte alignment
                free_fn(p, alloc_user, (void*)stream);
                p = nullptr;
            }
        } else if (cudaMalloc(&p, n) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        if (p) bytes += n;
        return p;
    }
    void dfree(void* p, size_t n) {
        if (!p) return;
        if (alloc)
            free_fn(p, alloc_user, (void*)stream);
        else
            cudaFree(p);
        bytes -= n;
    }

    size_t state_bytes() const { return (size_t)NQ * G.plane * esz; }
    size_t hist_bytes() const { return (size_t)4 * G.plane * rsz; }
    size_t nodes() const { return (size_t)G.nx * G.ny; }
    int read_mode() const {
        if (layout == LBM_AB_PULL) return P.nee ? GATHER_NEE_AB : GATHER_PULL_AB;
        return (t & 1) ? GATHER_PULL_AA : GATHER_LOCAL;
    }
};

namespace {

inline const Coef<double>& coef_of(const lbm_ctx* c, double*) { return c->cd; }
inline const Coef<float>& coef_of(const lbm_ctx* c, float*) { return c->cf; }

template <typename S>
cudaError_t dispatch_step(lbm_ctx* c) {
    using R = typename Real<S>::type;
    const Coef<R>& k = coef_of(c, (R*)nullptr);
    if (c->layout == LBM_AB_PULL) {
        cudaError_t e = launch_step_ab<S>(c->buf[c->cur], c->buf[c->cur ^ 1], c->hist, c->G, k, c->L);
        c->cur ^= 1;
        return e;
    }
    return launch_step_aa<S>(c->buf[0], c->hist, c->G, k, (c->t & 1) != 0, c->L);
}

cudaError_t one_step(lbm_ctx* c) {
    cudaError_t e;
    switch (c->prec) {
        case LBM_F64: e = dispatch_step<double>(c); break;
        case LBM_F32: e = dispatch_step<float>(c); break;
        case LBM_BF16: e = dispatch_step<__nv_bfloat16>(c); break;
        default: e = dispatch_step<__half>(c); break;
    }
    c->t += 1;
    return e;
}

#define LBM_DISPATCH(c, CALL_D, CALL_F, CALL_B, CALL_H) \
    ((c)->prec == LBM_F64 ? (CALL_D) : (c)->prec == LBM_F32 ? (CALL_F) : (c)->prec == LBM_BF16 ? (CALL_B) : (CALL_H))

cudaError_t run_init(lbm_ctx* c, const InitSpec& I) {
    const bool pull = c->layout == LBM_AB_PULL;
    return LBM_DISPATCH(c, launch_init<double>(c->buf[0], c->hist, c->G, c->cd, I, pull, c->stream),
                        launch_init<float>(c->buf[0], c->hist, c->G, c->cf, I, pull, c->stream),
                        launch_init<__nv_bfloat16>(c->buf[0], c->hist, c->G, c->cf, I, pull, c->stream),
                        launch_init<__half>(c->buf[0], c->hist, c->G, c->cf, I, pull, c->stream));
}

const void* cur_buf(const lbm_ctx* c) { return c->layout == LBM_AB_PULL ? c->buf[c->cur] : c->buf[0]; }

// (Re)initialise the state at t = 0 from host T / C fields or from the noise.
lbm_status do_init(lbm_ctx* c, const double* T_host, const double* C_host, uint64_t seed,
                   double noise) {
    InitSpec I;
    std::memset(&I, 0, sizeof I);
    I.seed = seed;
    I.noise = noise < 0 ? 0.0 : (noise == 0 ? 1e-3 : noise);
    I.T0 = c->P.T0;
    I.C0 = c->P.C0;
    I.sigma = c->P.sigma;
    I.eps = c->P.eps;
    I.varpi = c->P.varpi;
    I.model_a = c->P.model_a;
    // noise keys of the whole cavity: a slab draws the values its rows have in it
    I.key_ny = c->P.ny;
    I.key_j0 = c->slab_y0 - c->G.jb;
    const size_t n = (size_t)c->G.nx * step_rows(c->G);
    cudaError_t e = cudaSuccess;
    if (T_host) {
        if (!c->d_stage) {
            c->d_stage = (double*)c->dalloc(2 * c->nodes() * sizeof(double));
            if (!c->d_stage) return c->fail(LBM_ERR_NOMEM, "no device memory for initial fields");
        }
        e = cudaMemcpyAsync(c->d_stage, T_host, n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->d_stage + n, C_host, n * sizeof(double), cudaMemcpyHostToDevice,
                                c->stream);
        I.T_init = c->d_stage;
        I.C_init = c->d_stage + n;
    }
    if (e == cudaSuccess) e = run_init(c, I);
    if (e != cudaSuccess) return c->cuda_fail(e, "init");
    c->t = 0;
    c->cur = 0;
    c->snap_valid = false;
    return LBM_OK;
}

}  // namespace

bool lbm_ctx_view(const lbm_ctx* c, CtxView* v) {
    if (!c || !v) return false;
    v->prec = c->prec;
    v->buf = cur_buf(c);
    v->G = c->G;
    v->cd = &c->cd;
    v->cf = &c->cf;
    v->mode = c->read_mode();
    v->stream = c->stream;
    v->device = c->device;
    return true;
}

void lbm_set_error(lbm_ctx* c, const char* msg) {
    if (c) c->err = msg;
    g_last_error = msg;
}

extern "C" {

namespace {

// The mapping of Sec. 4 / 4.1 for a characteristic length of N_x spacings
// (L = nx for halfway walls, nx - 1 with nodes on the walls).
lbm_status derive_core(lbm_grid grid, int nee, double Ra, double Da, double eps, double Pr,
                       double Le, double N, double J, double sigma, double Ma, double varpi,
                       lbm_params* out) {
    if (!out) {
        set_global_error("lbm_derive_params: out is NULL");
        return LBM_ERR_INVALID;
    }
    if (grid.nx < 3 || grid.ny < 3) {
        set_global_error("lbm_derive_params: nx and ny must be >= 3 (got %d x %d)", grid.nx, grid.ny);
        return LBM_ERR_INVALID;
    }
    if (!(eps > 0.0 && eps <= 1.0) || !(Da > 0.0) || !(Ra > 0.0) || !(Pr > 0.0) || !(Le > 0.0) ||
        !(J > 0.0) || !(sigma > 0.0) || !std::isfinite(N)) {
        set_global_error("lbm_derive_params: need eps in (0,1], Da, Ra, Pr, Le, J, sigma > 0");
        return LBM_ERR_INVALID;
    }
    if (!(Ma > 0.0)) Ma = 0.1;
    if (!(varpi > 0.0)) varpi = 0.4;
    lbm_params P;
    std::memset(&P, 0, sizeof P);
    P.nx = grid.nx;
    P.ny = grid.ny;
    P.nee = nee;
    // characteristic length = N_x spacings (Sec. 4.1): nx halfway cells, or the nx - 1
    // spacings between wall nodes
    const double L = nee ? grid.nx - 1.0 : (double)grid.nx;
    const double cs2 = 1.0 / 3.0, cs = std::sqrt(cs2);
    const double U = Ma * cs;                       // Ma = U / c_s
    const double nu_e = J * U * L * std::sqrt(Pr / Ra);
    const double nu = nu_e / J;
    const double alpha_e = nu / Pr;
    const double D_e = alpha_e / Le;
    const double csT2 = 0.5 * varpi;
    const double s_nu = 1.0 / (0.5 + nu_e / cs2);   // nu_e = c_s^2 (1/s_nu - 1/2)
    const double za = 1.0 / (0.5 + alpha_e / csT2); // Eq. 29
    const double eD = 1.0 / (0.5 + D_e / csT2);
    P.eps = eps;
    P.sigma = sigma;
    P.varpi = varpi;
    P.nu = nu;
    P.K = Da * L * L;                               // Da = K / L^2
    P.Feps = 1.75 / std::sqrt(150.0 * eps * eps * eps);   // Eq. 7
    P.gbT = U * U / L;                              // U^2 = g beta_T dT L with dT = 1
    P.gbC = N * P.gbT;                              // N = beta_C dC / (beta_T dT)
    P.Gx = 0.0;
    P.T0 = 0.5;
    P.C0 = 0.5;
    const double s[9] = {1.0, 1.1, 1.1, 1.0, 1.2, 1.0, 1.2, s_nu, s_nu};   // Sec. 4
    const double z[5] = {1.0, za, za, 1.5, 1.5};
    const double e[5] = {1.0, eD, eD, 1.5, 1.5};
    std::memcpy(P.s, s, sizeof s);
    std::memcpy(P.zeta, z, sizeof z);
    std::memcpy(P.eta, e, sizeof e);
    const double Tw[4] = {1.0, 0.0, 0.5, 0.5};
    std::memcpy(P.Tw, Tw, sizeof Tw);
    std::memcpy(P.Cw, Tw, sizeof Tw);
    P.wall_lr = LBM_WALL_DIRICHLET;
    P.wall_tb = LBM_WALL_ADIABATIC;
    const char* bad = check_params(P);
    if (bad) {
        set_global_error("lbm_derive_params: %s (s_nu=%g zeta_a=%g eta_D=%g)", bad, s_nu, za, eD);
        return LBM_ERR_INVALID;
    }
    *out = P;
    return LBM_OK;
}

}  // namespace

lbm_status lbm_derive_params(lbm_grid grid, double Ra, double Da, double eps, double Pr,
                             double Le, double N, double J, double sigma, double Ma,
                             double varpi, lbm_params* out) {
    return derive_core(grid, 0, Ra, Da, eps, Pr, Le, N, J, sigma, Ma, varpi, out);
}

lbm_status lbm_derive_params_nee(lbm_grid grid, double Ra, double Da, double eps, double Pr,
                                 double Le, double N, double J, double sigma, double Ma,
                                 double varpi, lbm_params* out) {
    return derive_core(grid, 1, Ra, Da, eps, Pr, Le, N, J, sigma, Ma, varpi, out);
}

lbm_status lbm_derive_params_convective(int Nx, double Ra, double Da, double eps, double Pr,
                                        double Le, double N, double BiT, double BiC, double J,
                                        double sigma, double Ma, double varpi, lbm_params* out) {
    if (!(BiT >= 0.0) || !(BiC >= 0.0) || !std::isfinite(BiT) || !std::isfinite(BiC) || Nx < 4) {
        set_global_error("lbm_derive_params_convective: need Nx >= 4 and finite Bi >= 0");
        return LBM_ERR_INVALID;
    }
    lbm_grid g;
    g.nx = g.ny = Nx + 1;
    lbm_status st = derive_core(g, 1, Ra, Da, eps, Pr, Le, N, J, sigma, Ma, varpi, out);
    if (st != LBM_OK) return st;
    out->BiT[1] = BiT;                  // the right wall: ambient T = C = 0 (Tw[1], Cw[1])
    out->BiC[1] = BiC;
    return LBM_OK;
}

namespace {

lbm_status derive_lid_core(lbm_grid grid, int nee, double Re, double Gr, double Da, double eps,
                           double Pr, double Le, double N, double J, double sigma, double U0,
                           double varpi, lbm_params* out) {
    if (!out || grid.nx < 3 || grid.ny < 3 || !(Re > 0.0) || !(Gr >= 0.0) || !(Da > 0.0) ||
        !(eps > 0.0 && eps <= 1.0) || !(Pr > 0.0) || !(Le > 0.0) || !(J > 0.0) || !(sigma > 0.0)) {
        set_global_error("lbm_derive_params_lid: invalid arguments");
        return LBM_ERR_INVALID;
    }
    if (!(U0 > 0.0)) U0 = 0.1;
    if (!(varpi > 0.0)) varpi = 0.4;
    // reuse the cavity mapping for everything but the flow scales, then set those (Sec. 4.3)
    lbm_status st = derive_core(grid, nee, 1e4, Da, eps, Pr, Le, N, J, sigma, 0.1, varpi, out);
    if (st != LBM_OK) return st;
    lbm_params P = *out;
    const double L = nee ? grid.nx - 1.0 : (double)grid.nx, cs2 = 1.0 / 3.0, csT2 = 0.5 * varpi;
    const double nu_e = J * L * U0 / Re;             // 1/s_nu = 1/2 + J L U0 / (c_s^2 Re)
    const double nu = nu_e / J;
    const double alpha_e = nu / Pr, D_e = alpha_e / Le;
    const double s_nu = 1.0 / (0.5 + nu_e / cs2);
    P.nu = nu;
    P.s[7] = P.s[8] = s_nu;
    P.zeta[1] = P.zeta[2] = 1.0 / (0.5 + alpha_e / csT2);   // Eq. 29
    P.eta[1] = P.eta[2] = 1.0 / (0.5 + D_e / csT2);
    P.gbT = Gr * nu * nu / (L * L * L);                       // Gr = g beta_T dT L^3 / nu^2
    P.gbC = N * P.gbT;
    const double Tw[4] = {0.5, 0.5, 0.0, 1.0};               // bottom cold, top hot
    std::memcpy(P.Tw, Tw, sizeof Tw);
    std::memcpy(P.Cw, Tw, sizeof Tw);
    P.wall_lr = LBM_WALL_ADIABATIC;
    P.wall_tb = LBM_WALL_DIRICHLET;
    std::memset(P.uw, 0, sizeof P.uw);
    P.uw[3][0] = U0;                                          // the lid
    const char* bad = check_params(P);
    if (bad) {
        set_global_error("lbm_derive_params_lid: %s", bad);
        return LBM_ERR_INVALID;
    }
    *out = P;
    return LBM_OK;
}

}  // namespace

lbm_status lbm_derive_params_lid(lbm_grid grid, double Re, double Gr, double Da, double eps,
                                 double Pr, double Le, double N, double J, double sigma,
                                 double U0, double varpi, lbm_params* out) {
    return derive_lid_core(grid, 0, Re, Gr, Da, eps, Pr, Le, N, J, sigma, U0, varpi, out);
}

lbm_status lbm_derive_params_lid_nee(lbm_grid grid, double Re, double Gr, double Da, double eps,
                                     double Pr, double Le, double N, double J, double sigma,
                                     double U0, double varpi, lbm_params* out) {
    return derive_lid_core(grid, 1, Re, Gr, Da, eps, Pr, Le, N, J, sigma, U0, varpi, out);
}

lbm_status lbm_params_model_a(lbm_params* p) {
    if (!p || p->model_a) {
        set_global_error("lbm_params_model_a: NULL parameters, or already model A");
        return LBM_ERR_INVALID;
    }
    // Eq. 29 -> alpha_e, D_e; Eq. 32 -> the model-A rates
    const double csT2 = 0.5 * p->varpi;
    const double alpha_e = csT2 * (1.0 / p->zeta[1] - 0.5);
    const double D_e = csT2 * (1.0 / p->eta[1] - 0.5);
    lbm_params q = *p;
    q.zeta[1] = q.zeta[2] = 1.0 / (0.5 + alpha_e / (p->sigma * csT2));
    q.eta[1] = q.eta[2] = 1.0 / (0.5 + D_e / (p->eps * csT2));
    q.model_a = 1;
    const char* bad = check_params(q);
    if (bad) {
        set_global_error("lbm_params_model_a: %s", bad);
        return LBM_ERR_INVALID;
    }
    *p = q;
    return LBM_OK;
}

namespace {

// A cavity (slab_h = 0), or the slab of rows [slab_y0, slab_y0 + slab_h) of it.
lbm_status create_core(const lbm_params* params, const lbm_options* opt, int slab_y0, int slab_h,
                       lbm_ctx** out) {
    if (!params || !out) {
        set_global_error("lbm_create_raw: params and out must be non-NULL");
        return LBM_ERR_INVALID;
    }
    *out = nullptr;
    const char* bad = check_params(*params);
    if (bad) {
        set_global_error("lbm_create_raw: %s", bad);
        return LBM_ERR_INVALID;
    }
    const bool slab = slab_h > 0;
    if (slab) {
        if (slab_y0 < 0 || slab_y0 + slab_h > params->ny) {
            set_global_error("lbm_create_slab: rows [%d, %d) outside the %d rows of the cavity",
                             slab_y0, slab_y0 + slab_h, params->ny);
            return LBM_ERR_INVALID;
        }
        if (params->nee || (opt && (opt->layout != LBM_AB_PULL || opt->eps_field || opt->K_field))) {
            set_global_error("lbm_create_slab: slabs take halfway walls, the two-buffer layout "
                             "and a uniform porous medium");
            return LBM_ERR_INVALID;
        }
    }
    lbm_options O;
    std::memset(&O, 0, sizeof O);
    if (opt) O = *opt;
    if (O.precision < LBM_F64 || O.precision > LBM_F16) {
        set_global_error("lbm_create: unknown precision %d", O.precision);
        return LBM_ERR_INVALID;
    }
    if (O.layout != LBM_AB_PULL && O.layout != LBM_AA) {
        set_global_error("lbm_create: unknown layout %d", O.layout);
        return LBM_ERR_INVALID;
    }
    if ((O.alloc == nullptr) != (O.free == nullptr)) {
        set_global_error("lbm_create: alloc and free hooks must be given together");
        return LBM_ERR_INVALID;
    }
    if (params->nee && O.layout != LBM_AB_PULL) {
        set_global_error("lbm_create: walls with nodes on them (nee) need the two-buffer layout");
        return LBM_ERR_INVALID;
    }
    // the step kernels are compiled for blocks of at most 256 threads; the shape after
    // the defaults below (block_x 0 -> 128 or 32, block_y 0 -> 128 / block_x) must fit
    if (O.block_x < 0 || O.block_y < 0 || O.block_x > 256 || O.block_y > 256 ||
        (O.block_x && O.block_x % 32) ||
        (O.block_x ? O.block_x : (params->nx >= 128 ? 128 : 32)) *
                (O.block_y ? O.block_y : 1) > 256) {
        set_global_error("lbm_create: block_x must be a multiple of 32 and block_x*block_y <= 256");
        return LBM_ERR_INVALID;
    }
    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) {
        set_global_error("lbm_create: out of host memory");
        return LBM_ERR_NOMEM;
    }
    c->P = *params;
    c->prec = O.precision;
    c->layout = O.layout;
    c->esz = storage_size(c->prec);
    c->rsz = c->prec == LBM_F64 ? 8 : 4;
    c->alloc = O.alloc;
    c->free_fn = O.free;
    c->alloc_user = O.alloc_user;
    cudaGetDevice(&c->device);
    if (O.stream) {
        c->stream = (cudaStream_t)O.stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            lbm_status s = c->cuda_fail(e, "cudaStreamCreate");
            delete c;
            return s;
        }
        c->own_stream = true;
    }
    const int nx = params->nx;
    // a slab holds a ghost row beside each side that is a cut rather than a wall
    const int glo = slab && slab_y0 > 0 ? 1 : 0;
    const int ghi = slab && slab_y0 + slab_h < params->ny ? 1 : 0;
    const int rows = slab ? slab_h : params->ny;
    const int ny = rows + glo + ghi;
    const int per128 = (int)(128 / c->esz);
    c->slab = slab;
    c->slab_y0 = slab ? slab_y0 : 0;
    c->G.nx = nx;
    c->G.ny = ny;
    c->G.jb = glo;
    c->G.je = glo + rows;
    c->G.pitch = (nx + per128 - 1) / per128 * per128;
    c->G.plane = (size_t)ny * c->G.pitch;
    c->cd = make_coef<double>(c->P);
    c->cf = make_coef<float>(c->P);
    c->round_nearest = O.round_nearest != 0;
    c->cf.sr = c->round_nearest ? 0 : 1;
    c->cp = make_coef<f2>(c->P);
    c->cp.sr = c->cf.sr;
    // rounding streams keyed by the node's index in the undivided cavity
    c->cf.seed_off = (long long)(c->slab_y0 - c->G.jb) * c->G.pitch;
    int bx = O.block_x, by = O.block_y;
    if (bx == 0) bx = nx >= 128 ? 128 : 32;
    if (by == 0) by = bx >= 128 ? 1 : 128 / bx;
    if ((ny + by - 1) / by > 65535) {   // the launch grid's y extent
        lbm_status s = c->fail(LBM_ERR_INVALID, "lbm_create: ny = %d needs block_y >= %d", ny,
                               (ny + 65534) / 65535);
        g_last_error = c->err;
        lbm_destroy(c);
        return s;
    }
    c->L.bx = bx;
    c->L.by = by;
    c->L.stream = c->stream;
    c->L.aux = nullptr;
    // 16-bit storage takes the two-nodes-per-thread kernels, except on slabs, whose rows
    // all run the one-node kernel (the same arithmetic as a one-node whole cavity)
    c->L.pair = (c->prec == LBM_BF16 || c->prec == LBM_F16) && !slab ? &c->cp : nullptr;
    // a second stream lets the small ring launch of a split step run beside the inner one;
    // without it both go to the context's stream
    if (cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking) == cudaSuccess &&
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) == cudaSuccess) {
        c->L.aux = c->aux;
        c->L.fork = c->ev_fork;
        c->L.join = c->ev_join;
    } else {
        cudaGetLastError();
    }
    c->graph_chunk = O.graph_chunk == 0 ? 64 : (O.graph_chunk < 0 ? 0 : O.graph_chunk);
    if (c->graph_chunk & 1) c->graph_chunk += 1;   // a chunk must return to the same parity
    if (c->stream == nullptr || c->stream == cudaStreamLegacy || c->stream == cudaStreamPerThread)
        c->graph_chunk = 0;                        // the legacy stream cannot be captured

    c->buf[0] = c->dalloc(c->state_bytes());
    if (c->layout == LBM_AB_PULL) c->buf[1] = c->dalloc(c->state_bytes());
    c->hist = c->dalloc(c->hist_bytes());
    c->d_out = (double*)c->dalloc(64 * sizeof(double));
    if (O.eps_field || O.K_field) {
        if (c->P.model_a) {
            lbm_status s = c->fail(LBM_ERR_INVALID, "lbm_create: porous fields are not supported with model_a");
            g_last_error = c->err;
            lbm_destroy(c);
            return s;
        }
        // both planes in the compute precision, row pitch of the state
        const size_t plane = c->G.plane, n2 = 2 * plane;
        std::vector<double> hv(n2, 0.0);
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const size_t k = (size_t)j * nx + i, d = (size_t)j * c->G.pitch + i;
                const double e = O.eps_field ? O.eps_field[k] : c->P.eps;
                const double K = O.K_field ? O.K_field[k] : c->P.K;
                if (!(e > 0.0 && e <= 1.0) || !(K > 0.0)) {
                    lbm_status s = c->fail(LBM_ERR_INVALID,
                                           "lbm_create: porous field at (%d, %d): eps %g, K %g", i, j, e, K);
                    g_last_error = c->err;
                    lbm_destroy(c);
                    return s;
                }
                hv[d] = e;
                hv[plane + d] = K;
            }
        // padding columns: copies of a valid value, never read by the kernels
        for (size_t d = 0; d < n2; ++d)
            if (hv[d] == 0.0) hv[d] = d < plane ? c->P.eps : c->P.K;
        c->poro = c->dalloc(n2 * c->rsz);
        if (!c->poro) {
            lbm_status s = c->fail(LBM_ERR_NOMEM, "lbm_create: no device memory for the porous field");
            g_last_error = c->err;
            lbm_destroy(c);
            return s;
        }
        cudaError_t e;
        if (c->rsz == 8) {
            e = cudaMemcpy(c->poro, hv.data(), n2 * 8, cudaMemcpyHostToDevice);
        } else {
            std::vector<float> hf(hv.begin(), hv.end());
            e = cudaMemcpy(c->poro, hf.data(), n2 * 4, cudaMemcpyHostToDevice);
        }
        if (e != cudaSuccess) {
            lbm_status s = c->cuda_fail(e, "lbm_create: porous field upload");
            g_last_error = c->err;
            lbm_destroy(c);
            return s;
        }
        c->cd.poro = c->rsz == 8 ? (const double*)c->poro : nullptr;
        c->cf.poro = c->rsz == 4 ? (const float*)c->poro : nullptr;
    }
    if (!c->buf[0] || (c->layout == LBM_AB_PULL && !c->buf[1]) || !c->hist || !c->d_out) {
        lbm_status s = c->fail(LBM_ERR_NOMEM, "lbm_create: device allocation of %.3f GB failed",
                               (2.0 * c->state_bytes() + c->hist_bytes()) / 1e9);
        lbm_destroy(c);
        return s;
    }
    // padding columns are never read, but keep them defined
    cudaMemsetAsync(c->buf[0], 0, c->state_bytes(), c->stream);
    if (c->buf[1]) cudaMemsetAsync(c->buf[1], 0, c->state_bytes(), c->stream);
    cudaMemsetAsync(c->hist, 0, c->hist_bytes(), c->stream);

    if ((O.T_init == nullptr) != (O.C_init == nullptr)) {
        lbm_status s = c->fail(LBM_ERR_INVALID, "lbm_create: give both T_init and C_init");
        lbm_destroy(c);
        return s;
    }
    lbm_status s = do_init(c, O.T_init, O.C_init, O.seed, O.noise);
    if (s == LBM_OK) {   // the caller may release T_init / C_init once create returns
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) s = c->cuda_fail(e, "lbm_create: init");
    }
    if (s != LBM_OK) {
        g_last_error = c->err;
        lbm_destroy(c);
        return s;
    }
    *out = c;
    return LBM_OK;
}

}  // namespace

lbm_status lbm_create_raw(const lbm_params* params, const lbm_options* opt, lbm_ctx** out) {
    return create_core(params, opt, 0, 0, out);
}

lbm_status lbm_create_slab(const lbm_params* params, int y0, int h, const lbm_options* opt,
                           lbm_ctx** out) {
    if (h < 1) {
        if (out) *out = nullptr;
        set_global_error("lbm_create_slab: a slab needs at least one row");
        return LBM_ERR_INVALID;
    }
    return create_core(params, opt, y0, h, out);
}

lbm_status lbm_create(lbm_grid grid, double Ra, double Da, double eps, double Pr, double Le,
                      double N, double J, double sigma, const lbm_options* opt, lbm_ctx** out) {
    lbm_params P;
    const double Ma = opt ? opt->Ma : 0.0, varpi = opt ? opt->varpi : 0.0;
    lbm_status s = lbm_derive_params(grid, Ra, Da, eps, Pr, Le, N, J, sigma, Ma, varpi, &P);
    if (s != LBM_OK) return s;
    return lbm_create_raw(&P, opt, out);
}

lbm_status lbm_reset(lbm_ctx* c, const double* T_init, const double* C_init, uint64_t seed,
                     double noise) {
    if (!c || ((T_init == nullptr) != (C_init == nullptr))) {
        set_global_error("lbm_reset: NULL context, or only one of T_init / C_init given");
        return LBM_ERR_INVALID;
    }
    DeviceGuard dg(c->device);
    return do_init(c, T_init, C_init, seed, noise);
}

lbm_status lbm_step(lbm_ctx* c, int64_t n) {
    if (!c || n < 0) {
        set_global_error("lbm_step: invalid context or negative step count");
        return LBM_ERR_INVALID;
    }
    DeviceGuard dg(c->device);
    cudaError_t e = cudaSuccess;
    // Graph replay needs the even-parity state the graph was captured from.
    while (n > 0 && (c->t & 1) && e == cudaSuccess) {
        e = one_step(c);
        --n;
    }
    if (c->graph_chunk > 0 && n >= c->graph_chunk && e == cudaSuccess) {
        if (!c->graph) {
            cudaGraph_t g = nullptr;
            e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                const int64_t t0 = c->t;
                const int cur0 = c->cur;
                cudaError_t le = cudaSuccess;
                for (int k = 0; k < c->graph_chunk && le == cudaSuccess; ++k) le = one_step(c);
                c->t = t0;   // capture records, it does not run
                c->cur = cur0;
                e = cudaStreamEndCapture(c->stream, &g);
                if (le != cudaSuccess) e = le;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph, g, 0);
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                c->graph = nullptr;
                return c->cuda_fail(e, "lbm_step: graph capture");
            }
        }
        while (n >= c->graph_chunk && e == cudaSuccess) {
            e = cudaGraphLaunch(c->graph, c->stream);
            c->t += c->graph_chunk;   // even chunk: buffer parity unchanged
            n -= c->graph_chunk;
        }
    }
    while (n > 0 && e == cudaSuccess) {
        e = one_step(c);
        --n;
    }
    if (e != cudaSuccess) return c->cuda_fail(e, "lbm_step");
    return LBM_OK;
}

int64_t lbm_time(const lbm_ctx* c) { return c ? c->t : -1; }

lbm_status lbm_fields_window(lbm_ctx* c, int x0, int y0, int w, int h, double* ux, double* uy,
                             double* T, double* C, double* rho) {
    if (!c) {
        set_global_error("lbm_fields_window: NULL context");
        return LBM_ERR_INVALID;
    }
    const int rows = step_rows(c->G);
    if (x0 < 0 || y0 < 0 || w < 1 || h < 1 || x0 + w > c->G.nx || y0 + h > rows || h > 65535)
        return c->fail(LBM_ERR_INVALID, "lbm_fields_window: window (%d, %d, %d x %d) outside the %d x %d grid",
                       x0, y0, w, h, c->G.nx, rows);
    y0 += c->G.jb;   // a slab's rows start after its lower ghost row
    DeviceGuard dg(c->device);
    const size_t n = (size_t)w * h;
    if (n > c->fields_cap) {
        c->dfree(c->d_fields, 5 * c->fields_cap * sizeof(double));
        c->fields_cap = 0;
        c->d_fields = (double*)c->dalloc(5 * n * sizeof(double));
        if (!c->d_fields) return c->fail(LBM_ERR_NOMEM, "lbm_fields: no device memory for read-out");
        c->fields_cap = n;
    }
    const int mode = c->read_mode();
    const void* b = cur_buf(c);
    cudaError_t e = LBM_DISPATCH(c, launch_fields<double>(b, c->G, c->cd, mode, x0, y0, w, h, c->d_fields, c->stream),
                                 launch_fields<float>(b, c->G, c->cf, mode, x0, y0, w, h, c->d_fields, c->stream),
                                 launch_fields<__nv_bfloat16>(b, c->G, c->cf, mode, x0, y0, w, h, c->d_fields, c->stream),
                                 launch_fields<__half>(b, c->G, c->cf, mode, x0, y0, w, h, c->d_fields, c->stream));
    double* outs[5] = {ux, uy, T, C, rho};
    for (int k = 0; k < 5 && e == cudaSuccess; ++k)
        if (outs[k])
            e = cudaMemcpyAsync(outs[k], c->d_fields + k * n, n * sizeof(double),
                                cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return c->cuda_fail(e, "lbm_fields");
    return LBM_OK;
}

lbm_status lbm_fields(lbm_ctx* c, double* ux, double* uy, double* T, double* C, double* rho) {
    if (!c) {
        set_global_error("lbm_fields: NULL context");
        return LBM_ERR_INVALID;
    }
    // whole grid, in row bands of at most 65535 rows and about 2^26 nodes (2.7 GB of read-out)
    const int band = (int)std::max<size_t>(1, std::min<size_t>(65535, ((size_t)1 << 26) / c->G.nx));
    const int rows = step_rows(c->G);
    if (rows <= band) return lbm_fields_window(c, 0, 0, c->G.nx, rows, ux, uy, T, C, rho);
    for (int y0 = 0; y0 < rows; y0 += band) {
        const int h = std::min(band, rows - y0);
        const size_t off = (size_t)y0 * c->G.nx;
        lbm_status s = lbm_fields_window(c, 0, y0, c->G.nx, h, ux ? ux + off : nullptr, uy ? uy + off : nullptr,
                                         T ? T + off : nullptr, C ? C + off : nullptr, rho ? rho + off : nullptr);
        if (s != LBM_OK) return s;
    }
    return LBM_OK;
}

lbm_status lbm_nusselt_sherwood(lbm_ctx* c, double out[4]) {
    if (!c || !out) {
        set_global_error("lbm_nusselt_sherwood: NULL argument");
        return LBM_ERR_INVALID;
    }
    DeviceGuard dg(c->device);
    WallSpec W;
    W.Tw[0] = c->P.Tw[0];
    W.Tw[1] = c->P.Tw[1];
    W.Cw[0] = c->P.Cw[0];
    W.Cw[1] = c->P.Cw[1];
    W.T0 = c->P.T0;
    W.C0 = c->P.C0;
    W.dT = c->P.Tw[0] - c->P.Tw[1];
    W.dC = c->P.Cw[0] - c->P.Cw[1];
    W.nee = c->P.nee;
    W.L = c->P.nee ? c->P.nx - 1.0 : (double)c->P.nx;
    const int mode = c->read_mode();
    const void* b = cur_buf(c);
    cudaError_t e = LBM_DISPATCH(c, launch_nush<double>(b, c->G, c->cd, mode, W, c->d_out, c->stream),
                                 launch_nush<float>(b, c->G, c->cf, mode, W, c->d_out, c->stream),
                                 launch_nush<__nv_bfloat16>(b, c->G, c->cf, mode, W, c->d_out, c->stream),
                                 launch_nush<__half>(b, c->G, c->cf, mode, W, c->d_out, c->stream));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, c->d_out, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return c->cuda_fail(e, "lbm_nusselt_sherwood");
    for (int k = 0; k < 4; ++k)
        if (!std::isfinite(out[k]))
            return c->fail(LBM_ERR_DIVERGED, "lbm_nusselt_sherwood: non-finite result at t=%lld",
                           (long long)c->t);
    return LBM_OK;
}

lbm_status lbm_nusselt_sherwood_tb(lbm_ctx* c, double out[4]) {
    if (!c || !out) {
        set_global_error("lbm_nusselt_sherwood_tb: NULL argument");
        return LBM_ERR_INVALID;
    }
    if (c->slab) return c->fail(LBM_ERR_INVALID, "lbm_nusselt_sherwood_tb: not defined on a slab");
    DeviceGuard dg(c->device);
    WallSpec W;
    W.Tw[0] = c->P.Tw[2];
    W.Tw[1] = c->P.Tw[3];
    W.Cw[0] = c->P.Cw[2];
    W.Cw[1] = c->P.Cw[3];
    W.T0 = c->P.T0;
    W.C0 = c->P.C0;
    W.dT = c->P.Tw[3] - c->P.Tw[2];
    W.dC = c->P.Cw[3] - c->P.Cw[2];
    W.nee = c->P.nee;
    W.L = c->P.nee ? c->P.ny - 1.0 : (double)c->P.ny;
    const int mode = c->read_mode();
    const void* b = cur_buf(c);
    cudaError_t e = LBM_DISPATCH(c, launch_nush_tb<double>(b, c->G, c->cd, mode, W, c->d_out + 20, c->stream),
                                 launch_nush_tb<float>(b, c->G, c->cf, mode, W, c->d_out + 20, c->stream),
                                 launch_nush_tb<__nv_bfloat16>(b, c->G, c->cf, mode, W, c->d_out + 20, c->stream),
                                 launch_nush_tb<__half>(b, c->G, c->cf, mode, W, c->d_out + 20, c->stream));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, c->d_out + 20, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return c->cuda_fail(e, "lbm_nusselt_sherwood_tb");
    for (int k = 0; k < 4; ++k)
        if (!std::isfinite(out[k]))
            return c->fail(LBM_ERR_DIVERGED, "lbm_nusselt_sherwood_tb: non-finite result");
    return LBM_OK;
}

namespace {

// The residual pass over the updated rows: h[0..3] = max |phi_now - phi_snap|,
// h[4..7] = max |phi_now| (phi = u_x, u_y, T, C), h[8] != 0 if a value is not finite;
// the snapshot is replaced by phi_now.
lbm_status residual_maxima(lbm_ctx* c, const char* who, double h[9]) {
    DeviceGuard dg(c->device);
    const size_t n = c->nodes();
    if (!c->d_snap) {
        c->d_snap = c->dalloc(4 * n * c->rsz);
        c->d_partial = (double*)c->dalloc((size_t)RES_SLOTS * 9 * sizeof(double));
        if (!c->d_snap || !c->d_partial) return c->fail(LBM_ERR_NOMEM, "%s: no device memory", who);
    }
    const int mode = c->read_mode();
    const void* b = cur_buf(c);
    double* o = c->d_out + 8;
    cudaError_t e = LBM_DISPATCH(
        c, launch_residual<double>(b, c->G, c->cd, mode, c->d_snap, c->d_partial, o, c->stream),
        launch_residual<float>(b, c->G, c->cf, mode, c->d_snap, c->d_partial, o, c->stream),
        launch_residual<__nv_bfloat16>(b, c->G, c->cf, mode, c->d_snap, c->d_partial, o, c->stream),
        launch_residual<__half>(b, c->G, c->cf, mode, c->d_snap, c->d_partial, o, c->stream));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h, o, 9 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return c->cuda_fail(e, who);
    if (h[8] != 0.0) return c->fail(LBM_ERR_DIVERGED, "%s: non-finite field at t=%lld", who, (long long)c->t);
    if (!c->snap_valid)   // no earlier fields: the changes are unknown
        for (int q = 0; q < 4; ++q) h[q] = INFINITY;
    c->snap_valid = true;
    return LBM_OK;
}

}  // namespace

lbm_status lbm_residual(lbm_ctx* c, double* r) {
    if (!c || !r) {
        set_global_error("lbm_residual: NULL argument");
        return LBM_ERR_INVALID;
    }
    double h[9];
    lbm_status st = residual_maxima(c, "lbm_residual", h);
    if (st != LBM_OK) return st;
    double res = 0.0;
    for (int q = 0; q < 4; ++q) {
        double rq = h[4 + q] > 0 ? h[q] / h[4 + q] : (h[q] > 0 ? INFINITY : 0.0);
        res = rq > res ? rq : res;
    }
    *r = res;
    return LBM_OK;
}

lbm_status lbm_residual_parts(lbm_ctx* c, double parts[8]) {
    if (!c || !parts) {
        set_global_error("lbm_residual_parts: NULL argument");
        return LBM_ERR_INVALID;
    }
    double h[9];
    lbm_status st = residual_maxima(c, "lbm_residual_parts", h);
    if (st != LBM_OK) return st;
    for (int q = 0; q < 8; ++q) parts[q] = h[q];
    return LBM_OK;
}

lbm_status lbm_halo_bytes(const lbm_ctx* c, size_t* bytes) {
    if (!c || !bytes) {
        set_global_error("lbm_halo_bytes: NULL argument");
        return LBM_ERR_INVALID;
    }
    *bytes = 5 * (size_t)c->G.nx * c->esz;
    return LBM_OK;
}

namespace {

// side 0: the cut below the slab, 1: the cut above it.  Export reads the populations of
// the slab's outermost updated row that cross the cut; import writes the neighbour's into
// the ghost row on that side.
lbm_status halo_copy(lbm_ctx* c, int side, void* face, bool pack, const char* who) {
    if (!c || !face || (side != 0 && side != 1)) {
        set_global_error("%s: NULL argument or side not 0 / 1", who);
        return LBM_ERR_INVALID;
    }
    const bool cut = side == 0 ? c->G.jb > 0 : c->G.je < c->G.ny;
    if (!cut) return c->fail(LBM_ERR_INVALID, "%s: side %d of this context is a wall, not a cut", who, side);
    DeviceGuard dg(c->device);
    // export below: the bottom row's downward populations; export above: the top row's
    // upward ones; import below fills the lower ghost row with the upward populations of
    // the slab beneath, import above the upper ghost row with the downward ones
    const int row = pack ? (side == 0 ? c->G.jb : c->G.je - 1) : (side == 0 ? c->G.jb - 1 : c->G.je);
    const int up = pack ? side : 1 - side;
    void* b = c->layout == LBM_AB_PULL ? c->buf[c->cur] : c->buf[0];
    const int pk = pack ? 1 : 0;
    cudaError_t e = LBM_DISPATCH(c, launch_halo<double>(b, c->G, row, up, face, pk, c->stream),
                                 launch_halo<float>(b, c->G, row, up, face, pk, c->stream),
                                 launch_halo<__nv_bfloat16>(b, c->G, row, up, face, pk, c->stream),
                                 launch_halo<__half>(b, c->G, row, up, face, pk, c->stream));
    if (e != cudaSuccess) return c->cuda_fail(e, who);
    return LBM_OK;
}

}  // namespace

lbm_status lbm_halo_export(lbm_ctx* c, int side, void* face) {
    return halo_copy(c, side, face, true, "lbm_halo_export");
}

lbm_status lbm_halo_import(lbm_ctx* c, int side, const void* face) {
    return halo_copy(c, side, const_cast<void*>(face), false, "lbm_halo_import");
}

// Checkpoint layout: header, then the 19 state planes, then the 4 history planes.
namespace {
// A stored deviation as FP64: element k of a state array of precision prec (FP16 holds
// the deviation scaled by 2^12), and the reverse (rounded to nearest for narrower types).
double decode_value(int prec, const char* base, size_t k) {
    switch (prec) {
        case LBM_F64: return ((const double*)base)[k];
        case LBM_F32: return (double)((const float*)base)[k];
        case LBM_BF16: return (double)__bfloat162float(((const __nv_bfloat16*)base)[k]);
        default: return (double)__half2float(((const __half*)base)[k]) / 4096.0;
    }
}
void encode_value(int prec, char* base, size_t k, double v) {
    switch (prec) {
        case LBM_F64: ((double*)base)[k] = v; break;
        case LBM_F32: ((float*)base)[k] = (float)v; break;
        case LBM_BF16: ((__nv_bfloat16*)base)[k] = __float2bfloat16_rn((float)v); break;
        default: ((__half*)base)[k] = __float2half_rn((float)(v * 4096.0)); break;
    }
}
}  // namespace

namespace {
struct CkptHeader {
    char magic[8];
    int32_t version, nx, ny, prec, layout, pitch;
    int64_t t;
    lbm_params P;
};
}  // namespace

lbm_status lbm_save(lbm_ctx* c, void* buf, size_t* len) {
    if (!c || !len) {
        set_global_error("lbm_save: NULL argument");
        return LBM_ERR_INVALID;
    }
    const size_t need = sizeof(CkptHeader) + c->state_bytes() + c->hist_bytes();
    if (!buf) {
        *len = need;
        return LBM_OK;
    }
    if (*len < need) return c->fail(LBM_ERR_INVALID, "lbm_save: buffer of %zu bytes, need %zu", *len, need);
    DeviceGuard dg(c->device);
    CkptHeader h;
    std::memset(&h, 0, sizeof h);
    std::memcpy(h.magic, "LBMDDC1", 8);
    h.version = 2;   // 2: lbm_params carries the wall-node fields (nee, BiT, BiC)
    h.nx = c->G.nx;
    h.ny = c->G.ny;
    h.prec = c->prec;
    h.layout = c->layout;
    h.pitch = c->G.pitch;
    h.t = c->t;
    h.P = c->P;
    std::memcpy(buf, &h, sizeof h);
    char* p = (char*)buf + sizeof h;
    cudaError_t e = cudaMemcpyAsync(p, cur_buf(c), c->state_bytes(), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p + c->state_bytes(), c->hist, c->hist_bytes(), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return c->cuda_fail(e, "lbm_save");
    *len = need;
    return LBM_OK;
}

lbm_status lbm_load(lbm_ctx* c, const void* buf, size_t len) {
    if (!c || !buf) {
        set_global_error("lbm_load: NULL argument");
        return LBM_ERR_INVALID;
    }
    CkptHeader h;
    if (len < sizeof h) return c->fail(LBM_ERR_INVALID, "lbm_load: truncated checkpoint");
    std::memcpy(&h, buf, sizeof h);
    if (std::memcmp(h.magic, "LBMDDC1", 8) != 0 || h.version != 2)
        return c->fail(LBM_ERR_INVALID, "lbm_load: not a checkpoint of this library version");
    if (const char* bad = check_params(h.P))
        return c->fail(LBM_ERR_INVALID, "lbm_load: checkpoint parameters: %s", bad);
    if (h.P.nee && c->layout != LBM_AB_PULL)
        return c->fail(LBM_ERR_INVALID, "lbm_load: walls with nodes on them need the two-buffer layout");
    if (h.nx != c->G.nx || h.ny != c->G.ny || h.layout != c->layout)
        return c->fail(LBM_ERR_INVALID, "lbm_load: checkpoint does not match this context");
    if (h.prec < LBM_F64 || h.prec > LBM_F16)
        return c->fail(LBM_ERR_INVALID, "lbm_load: checkpoint of unknown precision %d", h.prec);
    const size_t src_esz = storage_size(h.prec), src_rsz = h.prec == LBM_F64 ? 8 : 4;
    const size_t src_plane = (size_t)h.ny * (size_t)h.pitch;
    const size_t src_state = (size_t)NQ * src_plane * src_esz, src_hist = 4 * src_plane * src_rsz;
    if (h.pitch < h.nx || len < sizeof h + src_state + src_hist)
        return c->fail(LBM_ERR_INVALID, "lbm_load: truncated checkpoint");
    DeviceGuard dg(c->device);
    // the two-buffer layout keeps the state in buffer (t mod 2), which the captured graph relies on
    const int slot = c->layout == LBM_AB_PULL ? (int)(h.t & 1) : 0;
    const char* p = (const char*)buf + sizeof h;
    cudaError_t e;
    if (h.prec == c->prec && h.pitch == c->G.pitch) {
        e = cudaMemcpyAsync(c->buf[slot], p, c->state_bytes(), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->hist, p + c->state_bytes(), c->hist_bytes(), cudaMemcpyHostToDevice,
                                c->stream);
    } else {
        // another storage precision: every stored deviation and history value is decoded
        // to FP64 and encoded in this context's precision (exact when widening, rounded to
        // nearest when narrowing), row by row into this context's row pitch
        std::vector<char> st;
        try {
            st.assign(c->state_bytes() + c->hist_bytes(), 0);
        } catch (...) {
            return c->fail(LBM_ERR_NOMEM, "lbm_load: no host memory to convert the checkpoint");
        }
        const size_t plane = c->G.plane;
        for (int q = 0; q < NQ; ++q)
            for (int j = 0; j < h.ny; ++j)
                for (int i = 0; i < h.nx; ++i) {
                    const size_t a = (size_t)q * src_plane + (size_t)j * h.pitch + i;
                    const size_t b = (size_t)q * plane + (size_t)j * c->G.pitch + i;
                    encode_value(c->prec, st.data(), b, decode_value(h.prec, p, a));
                }
        const char* ph = p + src_state;
        char* dh = st.data() + c->state_bytes();
        for (int k = 0; k < 4; ++k)
            for (int j = 0; j < h.ny; ++j)
                for (int i = 0; i < h.nx; ++i) {
                    const size_t a = (size_t)k * src_plane + (size_t)j * h.pitch + i;
                    const size_t b = (size_t)k * plane + (size_t)j * c->G.pitch + i;
                    const double v = src_rsz == 8 ? ((const double*)ph)[a] : (double)((const float*)ph)[a];
                    if (c->rsz == 8)
                        ((double*)dh)[b] = v;
                    else
                        ((float*)dh)[b] = (float)v;
                }
        e = cudaMemcpyAsync(c->buf[slot], st.data(), c->state_bytes(), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->hist, dh, c->hist_bytes(), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);   // before st is released
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return c->cuda_fail(e, "lbm_load");
    c->P = h.P;
    c->cd = make_coef<double>(c->P);
    c->cf = make_coef<float>(c->P);
    c->cf.sr = c->round_nearest ? 0 : 1;
    c->cp = make_coef<f2>(c->P);
    c->cp.sr = c->cf.sr;
    c->cf.seed_off = (long long)(c->slab_y0 - c->G.jb) * c->G.pitch;
    c->cd.poro = (c->poro && c->rsz == 8) ? (const double*)c->poro : nullptr;
    c->cf.poro = (c->poro && c->rsz == 4) ? (const float*)c->poro : nullptr;
    if (c->graph) {   // constants are baked into the captured launches
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    c->t = h.t;
    c->cur = slot;
    c->snap_valid = false;
    return LBM_OK;
}

lbm_status lbm_get_params(const lbm_ctx* c, lbm_params* out) {
    if (!c || !out) {
        set_global_error("lbm_get_params: NULL argument");
        return LBM_ERR_INVALID;
    }
    *out = c->P;
    return LBM_OK;
}

size_t lbm_device_bytes(const lbm_ctx* c) { return c ? c->bytes : 0; }

void lbm_destroy(lbm_ctx* c) {
    if (!c) return;
    DeviceGuard dg(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->dfree(c->buf[0], c->state_bytes());
    c->dfree(c->buf[1], c->state_bytes());
    c->dfree(c->hist, c->hist_bytes());
    c->dfree(c->d_out, 64 * sizeof(double));
    c->dfree(c->d_fields, 5 * c->fields_cap * sizeof(double));
    c->dfree(c->d_snap, 4 * c->nodes() * c->rsz);
    c->dfree(c->d_partial, (size_t)RES_SLOTS * 9 * sizeof(double));
    c->dfree(c->d_stage, 2 * c->nodes() * sizeof(double));
    c->dfree(c->poro, 2 * c->G.plane * c->rsz);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->aux) cudaStreamDestroy(c->aux);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char* lbm_last_error(const lbm_ctx* c) {
    if (c) return c->err.c_str();
    return g_last_error.c_str();
}

}  // extern "C"
