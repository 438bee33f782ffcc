// Device-side building blocks of the fused three-lattice step.
//
// Storage holds deviations from the rest equilibria (u = 0, rho = rho0,
// T = T0, C = C0) of Eqs. 20 and 28:
//   f'_i = f_i - w_i rho0,  g'_i = g_i - g_i^eq(T0, 0),  h'_i = h_i - h_i^eq(C0, 0).
// Every equilibrium moment that is linear in rho, T or C (Eqs. 14, 24, 25)
// has its rest part cancelled exactly by the shift, so the collision below
// is the paper's collision rewritten in these variables (no approximation);
// it keeps small numbers small, which is what FP32 / FP16 / BF16 storage needs.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

namespace lbm {

// D2Q9 velocities (Eq. 8), same ordering as the paper; D2Q5 uses q = 0..4.
//   q : 0  1  2  3  4  5  6  7  8
//   ex: 0  1  0 -1  0  1 -1 -1  1
//   ey: 0  0  1  0 -1  1  1 -1 -1
__host__ __device__ constexpr int ex_of(int q) {
    return q == 1 || q == 5 || q == 8 ? 1 : (q == 3 || q == 6 || q == 7 ? -1 : 0);
}
__host__ __device__ constexpr int ey_of(int q) {
    return q == 2 || q == 5 || q == 6 ? 1 : (q == 4 || q == 7 || q == 8 ? -1 : 0);
}
__host__ __device__ constexpr int opp_of(int q) {
    return q == 0 ? 0 : (q <= 4 ? ((q + 1) & 3) + 1 : ((q - 3) & 3) + 5);
}
static_assert(opp_of(1) == 3 && opp_of(3) == 1 && opp_of(2) == 4 && opp_of(4) == 2, "opp");
static_assert(opp_of(5) == 7 && opp_of(7) == 5 && opp_of(6) == 8 && opp_of(8) == 6, "opp");

// D2Q9 weights (Eq. 20).
__host__ __device__ constexpr double w9_of(int q) {
    return q == 0 ? 4.0 / 9.0 : (q <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
}

// Plane index of each lattice inside the 19-plane state: f 0..8, g 9..13, h 14..18.
constexpr int QF = 0, QG = 9, QH = 14, NQ = 19;

// ---- storage conversions -------------------------------------------------------
// 32-bit mixing function (the MurmurHash3 finaliser): random bits for stochastic rounding.
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x85EBCA6Bu;
    x ^= x >> 13;
    x *= 0xC2B2AE35u;
    x ^= x >> 16;
    return x;
}

template <typename R> __device__ __forceinline__ R sqrt_(R x);
template <> __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
template <> __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
// |x|, max(a, b) and finiteness in the precision of the argument (FP32 stays on the
// FP32 pipes; GB300's FP64 pipe is narrow).
template <typename R> __device__ __forceinline__ R abs_(R x);
template <> __device__ __forceinline__ float abs_(float x) { return fabsf(x); }
template <> __device__ __forceinline__ double abs_(double x) { return fabs(x); }
template <typename R> __device__ __forceinline__ R max_(R a, R b);
template <> __device__ __forceinline__ float max_(float a, float b) { return fmaxf(a, b); }
template <> __device__ __forceinline__ double max_(double a, double b) { return fmax(a, b); }
template <typename R> __device__ __forceinline__ bool finite_(R x);
template <> __device__ __forceinline__ bool finite_(float x) { return fabsf(x) <= 3.402823466e38f; }
template <> __device__ __forceinline__ bool finite_(double x) { return fabs(x) <= 1.7976931348623157e308; }

// st() rounds to nearest even; st_sr() rounds stochastically (up with probability
// equal to the distance to the lower neighbour in ulps), so that the expected stored
// value equals the computed one.  With 8-11 significand bits, rounding to nearest
// makes per-step changes smaller than half an ulp vanish (the state stagnates);
// stochastic rounding keeps them on average.
// ld_nc() reads through the non-coherent read-only path (__ldg).  gather_local() uses
// it: the in-place even step loads and stores the same array, and with coherent loads
// it was compiled to 98 registers (25 % occupancy) against 64 with ld_nc (GB300,
// 4096^2 FP32 in-place step 516 -> 483 us).  Valid there because each thread writes
// only the locations it has itself read before, and reads nothing another thread of
// the launch writes.  (For the pulls of the odd step the same change cost registers.)
template <typename S> struct Store;
template <> struct Store<double> {
    static constexpr bool kLow = false;
    __device__ static double ld(const double* p) { return *p; }
    __device__ static double ld_nc(const double* p) { return __ldg(p); }
    __device__ static void st(double* p, double v) { *p = v; }
    __device__ static void st_sr(double* p, double v, uint32_t) { *p = v; }
};
template <> struct Store<float> {
    static constexpr bool kLow = false;
    __device__ static float ld(const float* p) { return *p; }
    __device__ static float ld_nc(const float* p) { return __ldg(p); }
    __device__ static void st(float* p, float v) { *p = v; }
    __device__ static void st_sr(float* p, float v, uint32_t) { *p = v; }
};
template <> struct Store<__nv_bfloat16> {
    static constexpr bool kLow = true;
    __device__ static float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
    __device__ static float ld_nc(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
    __device__ static void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
    __device__ static void st_sr(__nv_bfloat16* p, float v, uint32_t r) {
        // bfloat16 is the top half of the float: add 16 random bits (r < 2^16) below it,
        // truncate (on the sign-magnitude encoding this rounds |v| away from zero with
        // the right odds).  v must be finite (put() routes non-finite nodes to st()).
        const uint32_t b = __float_as_uint(v) + r;
        *p = __ushort_as_bfloat16((unsigned short)(b >> 16));
    }
};
// FP16 holds the deviations scaled by 2^12 (exact in both directions), so that
// deviations down to ~1.5e-8 sit in FP16's normal range (11 significant bits)
// instead of its subnormals; |deviation| must stay below 16 (65504 / 2^12).
template <> struct Store<__half> {
    static constexpr bool kLow = true;
    static constexpr float kScale = 4096.0f, kInvScale = 1.0f / 4096.0f;
    __device__ static float ld(const __half* p) { return __half2float(*p) * kInvScale; }
    __device__ static float ld_nc(const __half* p) { return __half2float(__ldg(p)) * kInvScale; }
    __device__ static void st(__half* p, float v) { *p = __float2half_rn(v * kScale); }
    __device__ static void st_sr(__half* p, float v, uint32_t r) {
        // In FP16's normal range the 13 float mantissa bits below the 10 kept ones are
        // the fraction of an FP16 ulp: add 13 random bits there, then truncate.  v must
        // be finite (put() routes non-finite nodes to st()).
        const uint32_t b = __float_as_uint(v * kScale) + (r & 0x1FFFu);
        *p = __float2half_rz(__uint_as_float(b));
    }
};

// Store one of a node's populations: stochastic rounding for 16-bit storage when
// sr is set (see sr_node).  The random bits come from a per-node linear
// congruential stream (the 32-bit constants of Numerical Recipes) seeded by node_seed(); only its high
// 16 bits are used, which is enough for rounding decisions and costs one
// multiply-add per value.
template <typename S, typename R>
__device__ __forceinline__ void put(S* p, R v, int sr, uint32_t& state, int) {
    if (Store<S>::kLow && sr) {
        state = state * 1664525u + 1013904223u;
        Store<S>::st_sr(p, v, state >> 16);
    } else {
        Store<S>::st(p, v);
    }
}

// Whether a node's post-collision values are stored with stochastic rounding: 16-bit
// storage with rounding enabled and all 19 values finite (one check on their sum
// instead of one per value; a node holding a NaN or an infinity is rounded to
// nearest, which keeps it non-finite for the residual's divergence check).
template <typename S, typename R>
__device__ __forceinline__ int sr_node(int sr, const R f[9], const R g[5], const R h[5]) {
    if (!Store<S>::kLow || !sr) return 0;
    R s = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7]));
    s += ((f[8] + g[0]) + (g[1] + g[2])) + ((g[3] + g[4]) + (h[0] + h[1]));
    s += (h[2] + h[3]) + h[4];
    return finite_(s) ? 1 : 0;
}

// Per-node seed of the random stream: a hash of the node's index and of the bits of
// two of its pre-collision populations.  The populations change from step to step,
// so the stream does too, with no step counter (graph replay stays valid) and the
// same result whenever the same state is stepped (runs are reproducible).
template <typename R>
__device__ __forceinline__ uint32_t node_seed(size_t node, R a, R b) {
    const uint32_t ia = __float_as_uint((float)a), ib = __float_as_uint((float)b);
    return mix32(ia ^ mix32(ib ^ mix32((uint32_t)node ^ (uint32_t)(node >> 32) * 0x27D4EB2Fu)));
}

// ---- two nodes per thread ----------------------------------------------------------
// f2: the FP32 values of one quantity at two x-adjacent nodes, computed with the packed
// FP32x2 instructions of sm_100 and later (one add, multiply or fused multiply-add for
// both nodes).  Products are kept unevaluated (f2m) until they meet an addition or a
// subtraction, which then becomes one fused multiply-add, as a compiler contracts
// a * b + c in scalar code.  Division and square root act per component.  The scalar
// collision and macroscopic code (collide, macro) is instantiated with R = f2.
struct f2 {
    float2 v;
    f2() = default;
    __host__ __device__ f2(float2 a) : v(a) {}
    template <typename T, typename std::enable_if<std::is_arithmetic<T>::value, int>::type = 0>
    __host__ __device__ explicit f2(T s) : v(make_float2((float)s, (float)s)) {}
};
#ifdef __CUDACC__
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
struct f2m {
    float2 a, b;
    __device__ __forceinline__ operator f2() const { return f2(__fmul2_rn(a, b)); }
};
__device__ __forceinline__ f2m operator*(f2 a, f2 b) { return f2m{a.v, b.v}; }
__device__ __forceinline__ f2m operator*(f2m a, f2 b) { return f2m{f2(a).v, b.v}; }
__device__ __forceinline__ f2m operator*(f2 a, f2m b) { return f2m{a.v, f2(b).v}; }
__device__ __forceinline__ f2m operator*(f2m a, f2m b) { return f2m{f2(a).v, f2(b).v}; }
__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return f2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ f2 operator-(f2 a, f2 b) {
    return f2(__ffma2_rn(b.v, make_float2(-1.0f, -1.0f), a.v));   // round(a - b) exactly
}
__device__ __forceinline__ f2 operator+(f2m p, f2 c) { return f2(__ffma2_rn(p.a, p.b, c.v)); }
__device__ __forceinline__ f2 operator+(f2 c, f2m p) { return f2(__ffma2_rn(p.a, p.b, c.v)); }
__device__ __forceinline__ f2 operator-(f2 c, f2m p) { return f2(__ffma2_rn(neg2(p.a), p.b, c.v)); }
__device__ __forceinline__ f2 operator-(f2m p, f2 c) { return f2(__ffma2_rn(p.a, p.b, neg2(c.v))); }
__device__ __forceinline__ f2 operator+(f2m p, f2m q) { return f2(__ffma2_rn(p.a, p.b, f2(q).v)); }
__device__ __forceinline__ f2 operator-(f2m p, f2m q) {
    return f2(__ffma2_rn(neg2(q.a), q.b, f2(p).v));
}
__device__ __forceinline__ f2 operator-(f2 a) { return f2(neg2(a.v)); }
__device__ __forceinline__ f2 operator-(f2m p) { return f2m{neg2(p.a), p.b}; }
__device__ __forceinline__ f2& operator+=(f2& a, f2 b) { return a = a + b; }
__device__ __forceinline__ f2& operator-=(f2& a, f2 b) { return a = a - b; }
__device__ __forceinline__ f2& operator+=(f2& a, f2m b) { return a = a + b; }
__device__ __forceinline__ f2& operator-=(f2& a, f2m b) { return a = a - b; }
__device__ __forceinline__ f2 operator/(f2 a, f2 b) { return f2(make_float2(a.v.x / b.v.x, a.v.y / b.v.y)); }
template <> __device__ __forceinline__ f2 sqrt_(f2 x) {
    return f2(make_float2(sqrtf(x.v.x), sqrtf(x.v.y)));
}
#endif

// Compute type for a storage type: FP64 stays FP64, everything else is FP32.
template <typename S> struct Real { using type = float; };
template <> struct Real<double> { using type = double; };

// ---- per-instance constants (prepared on the host, passed by value) ------------
template <typename R>
struct Coef {
    R T0, C0;
    R inv_sigma, inv_eps;      // Eq. 26
    R eps, half_eps;           // eps of Eqs. 5, 14, 15, 19
    R inv_eps_f;               // 1/eps for the flow equilibria (Eqs. 14, 15)
    R gbT, gbC, Gx;            // Eq. 6 (+ optional constant Gx)
    R l0, l0sq, l1;            // Eq. 19
    R drag_lin, drag_quad;     // eps nu / K and eps F_eps / sqrt(K) (Eq. 5)
    R s1, s2, s3, s4, s5, s6, s7, s8;   // Lambda (s_rho plays no role: m_0 is conserved)
    R h1, h2, h3, h4, h5, h6, h7, h8;   // 1 - s_k / 2, the factors of the forcing (Eq. 10)
    R za1, za2, za3, za4;      // Theta (zeta_0 plays no role)
    R ed1, ed2, ed3, ed4;      // Q
    R hz1, hz2, he1, he2;      // 1 - zeta_k / 2, 1 - eta_k / 2 (source terms of Eqs. 21-22)
    R c3T, c3C;                // 5 varpi - 4 sigma, 5 varpi - 4 eps (Eqs. 24, 25)
    // Per wall side (0 left, 1 right, 2 bottom, 3 top): 2 w~ (Phi_w - Phi0) with
    // w~ = varpi / 4, the anti-bounce-back constant in deviations.
    R wallT[4], wallC[4];
    int dirichlet_mask;        // bit s set: side s is Dirichlet for g and h, else adiabatic
    int sr;                    // 1: stochastic rounding when storing 16-bit populations
    // Moving walls: wmom[s] = 2 rho0 u_w / c_s^2 of side s; moving = 1 if any is nonzero.
    R wmom[4][2];
    int moving;
    // Spatially varying porous medium: NULL, or planes [2][ny][pitch] of (eps, K); then
    // the porous constants above are recomputed per node (porous_at).
    const R* poro;
    R nu, varpi5;              // fluid viscosity of Eq. 5, 5 varpi of Eq. 25
    // Walls with nodes on them (Sec. 3.3, nee = 1): wall values Phi_w - Phi0 by side,
    // Bi / L of convective sides (Eq. 39; 0 otherwise), wall velocities, and the D2Q5
    // equilibria as g_eq,0 = a0 Phi, g_eq,i = a1 Phi + (e_i . u) Phi / 2 (i = 1..4) with
    // a0 = (cap - c3) / 5, a1 = cap / 5 + c3 / 20 (N^-1 n_eq of Eqs. 24-25 / 30-31).
    int nee;
    // Added to a node's storage index to key its stochastic-rounding stream: 0 for a
    // cavity; for a slab of a cavity split along y, the offset that makes the key the
    // node's index in the undivided cavity (so a split run rounds as the whole one does).
    long long seed_off;
    R TwP[4], CwP[4];
    R bT[4], bC[4];
    R uwall[4][2];
    R aT0, aT1, aC0, aC1;
};



// The constants of node `self` of a cavity with a porosity / permeability field:
// eps and K from the field, F_eps from Eq. 7, l0 and l1 from Eq. 19, the drag
// coefficients of Eq. 5 and the n_eq,3 factor of Eq. 25.
template <typename R>
__device__ __forceinline__ void porous_at(Coef<R>& c, size_t self, size_t plane) {
    const R e = c.poro[self], K = c.poro[plane + self];
    const R Fe = R(1.75) / sqrt_(R(150) * e * e * e);
    c.eps = e;
    c.half_eps = R(0.5) * e;
    c.inv_eps = R(1) / e;
    c.inv_eps_f = c.inv_eps;
    c.drag_lin = e * c.nu / K;
    c.drag_quad = e * Fe / sqrt_(K);
    c.l0 = R(0.5) * (R(1) + R(0.5) * c.drag_lin);
    c.l0sq = c.l0 * c.l0;
    c.l1 = R(0.5) * c.drag_quad;
    c.c3C = c.varpi5 - R(4) * e;
    c.aC0 = (e - c.c3C) * R(0.2);
    c.aC1 = e * R(0.2) + c.c3C * R(0.05);
}

// Macroscopic quantities of one node from pre-collision deviations.
template <typename R>
struct Macro {
    R rho, ux, uy, Tp, Cp, Fx, Fy;   // rho' (deviation), u, T - T0, C - C0, F
};

template <typename R>
__device__ __forceinline__ Macro<R> macro(const Coef<R>& c, const R f[9], const R g[5],
                                          const R h[5]) {
    Macro<R> o;
    R rho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];  // Eq. 16
    R jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
    R jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
    R Tp = (((g[0] + g[1]) + (g[2] + g[3])) + g[4]) * c.inv_sigma;   // Eq. 26
    R Cp = (((h[0] + h[1]) + (h[2] + h[3])) + h[4]) * c.inv_eps;
    R Gy = c.gbT * Tp + c.gbC * Cp;                                  // Eq. 6
    R vx = jx + c.half_eps * c.Gx;                                   // Eq. 19, rho0 = 1
    R vy = jy + c.half_eps * Gy;
    R vm = sqrt_(vx * vx + vy * vy);
    R den = c.l0 + sqrt_(c.l0sq + c.l1 * vm);                       // Eq. 18
    const R inv_den = R(1) / den;
    R ux = vx * inv_den, uy = vy * inv_den;
    R um = sqrt_(ux * ux + uy * uy);
    R drag = c.drag_lin + c.drag_quad * um;                          // Eq. 5
    o.rho = rho;
    o.ux = ux;
    o.uy = uy;
    o.Tp = Tp;
    o.Cp = Cp;
    o.Fx = c.eps * c.Gx - drag * ux;
    o.Fy = c.eps * Gy - drag * uy;
    return o;
}

// D2Q5 collision (Eq. 21 / 22 with Eq. 24 / 25 and the moment-space source
// (0, X_x, X_y, 0, 0) of Eq. 27), written as d* = d - N^-1 [Theta (n - n_eq)
// - (I - Theta/2) S] so that only the change is rounded; the zeroth moment
// (cap * Phi) is conserved exactly, its change is set to zero.  N^-1 uses the
// orthogonality of N: N^-1 = N^T D^-1, D = diag(5, 2, 2, 20, 4).
// Pp = Phi - Phi0, P = Phi (Phi = T or C), c3 = 5 varpi - 4 cap.
template <typename R>
__device__ __forceinline__ void collide_d2q5(R d[5], R Pp, R P, R ux, R uy, R Xx, R Xy,
                                             R r1, R r2, R r3, R r4, R c3, R q1, R q2) {
    const R n1 = d[1] - d[3];
    const R n2 = d[2] - d[4];
    const R n3 = ((d[1] + d[2]) + (d[3] + d[4])) - R(4) * d[0];
    const R n4 = (d[1] - d[2]) + (d[3] - d[4]);
    const R k1 = r1 * (n1 - ux * P) - q1 * Xx;   // q_k = 1 - r_k / 2
    const R k2 = r2 * (n2 - uy * P) - q2 * Xy;
    const R k3 = r3 * (n3 - c3 * Pp);
    const R k4 = r4 * n4;
    const R b1 = k1 * R(0.5), b2 = k2 * R(0.5), b3 = k3 * R(0.05), b4 = k4 * R(0.25);
    d[0] += R(4) * b3;
    d[1] -= b1 + b3 + b4;
    d[2] -= b2 + b3 - b4;
    d[3] -= -b1 + b3 + b4;
    d[4] -= -b2 + b3 - b4;
}

// The collision of one node, in place on the deviations f, g, h: collide_flow (the D2Q9
// part), then collide_scalars; collide() does both.  hist = (T u_x, T u_y, C u_x, C u_y)
// at the previous step; updated.  The D2Q9 part is Eq. 10 written as
// f* = f - M^-1 [Lambda (m - m_eq) - (I - Lambda/2) S] (only the change is rounded; the
// density moment is conserved exactly).
template <typename R>
__device__ __forceinline__ void collide_flow(const Coef<R>& c, const Macro<R>& M, R f[9]) {
    const R ux = M.ux, uy = M.uy, Fx = M.Fx, Fy = M.Fy, rho = M.rho;
    const R ie = c.inv_eps_f;
    // m = M f (Eq. 13), deviation part; m_0 = rho' is not needed
    const R fa = (f[1] + f[2]) + (f[3] + f[4]);
    const R fd = (f[5] + f[6]) + (f[7] + f[8]);
    const R m1 = R(2) * fd - fa - R(4) * f[0];
    const R m2 = R(4) * f[0] - R(2) * fa + fd;
    const R m3 = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
    const R m4 = R(2) * (f[3] - f[1]) + (f[5] - f[6]) + (f[8] - f[7]);
    const R m5 = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
    const R m6 = R(2) * (f[4] - f[2]) + (f[5] + f[6]) - (f[7] + f[8]);
    const R m7 = (f[1] - f[2]) + (f[3] - f[4]);
    const R m8 = (f[5] - f[6]) + (f[7] - f[8]);
    // m_eq (Eq. 14, alpha1 = 1, alpha2 = -3, rho0 = 1) minus its rest part, and S (Eq. 15)
    const R u2e = (ux * ux + uy * uy) * ie;
    const R uF = (ux * Fx + uy * Fy) * ie;
    const R e1 = R(-2) * rho + R(3) * u2e;
    const R e2 = rho - R(3) * u2e;
    const R e7 = (ux * ux - uy * uy) * ie;
    const R e8 = ux * uy * ie;
    const R S1 = R(6) * uF;
    const R S7 = R(2) * (ux * Fx - uy * Fy) * ie;
    const R S8 = (ux * Fy + uy * Fx) * ie;
    // Lambda (m - m_eq) - (I - Lambda/2) S, component by component (S_2 = -S_1, S_4 = -F_x, ...)
    const R d1 = c.s1 * (m1 - e1) - c.h1 * S1;
    const R d2 = c.s2 * (m2 - e2) + c.h2 * S1;
    const R d3 = c.s3 * (m3 - ux) - c.h3 * Fx;
    const R d4 = c.s4 * (m4 + ux) + c.h4 * Fx;
    const R d5 = c.s5 * (m5 - uy) - c.h5 * Fy;
    const R d6 = c.s6 * (m6 + uy) + c.h6 * Fy;
    const R d7 = c.s7 * (m7 - e7) - c.h7 * S7;
    const R d8 = c.s8 * (m8 - e8) - c.h8 * S8;
    // M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4)
    const R a1 = d1 * R(1.0 / 36.0), a2 = d2 * R(1.0 / 36.0);
    const R a3 = d3 * R(1.0 / 6.0), a4 = d4 * R(1.0 / 12.0);
    const R a5 = d5 * R(1.0 / 6.0), a6 = d6 * R(1.0 / 12.0);
    const R a7 = d7 * R(0.25), a8 = d8 * R(0.25);
    const R axis = -a1 - R(2) * a2;
    const R diag = R(2) * a1 + a2;
    const R px = a3 - R(2) * a4, py = a5 - R(2) * a6;
    const R qx = a3 + a4, qy = a5 + a6;
    f[0] -= R(4) * (a2 - a1);
    f[1] -= axis + px + a7;
    f[2] -= axis + py - a7;
    f[3] -= axis - px + a7;
    f[4] -= axis - py - a7;
    f[5] -= diag + qx + qy + a8;
    f[6] -= diag - qx + qy - a8;
    f[7] -= diag - qx - qy + a8;
    f[8] -= diag + qx - qy - a8;
}

// The two D2Q5 collisions of a node (Eqs. 21-22) with the source of Eq. 27; hist is
// read and updated.
template <typename R>
__device__ __forceinline__ void collide_scalars(const Coef<R>& c, const Macro<R>& M, R g[5], R h[5],
                                                R hist[4]) {
    const R ux = M.ux, uy = M.uy;
    // Eq. 27 with d(Phi u)/dt = (Phi u)|t - (Phi u)|t-1 (Sec. 3.2)
    const R T = c.T0 + M.Tp, C = c.C0 + M.Cp;
    const R Tux = T * ux, Tuy = T * uy, Cux = C * ux, Cuy = C * uy;
    const R XTx = Tux - hist[0], XTy = Tuy - hist[1], XCx = Cux - hist[2], XCy = Cuy - hist[3];
    hist[0] = Tux;
    hist[1] = Tuy;
    hist[2] = Cux;
    hist[3] = Cuy;
    collide_d2q5(g, M.Tp, T, ux, uy, XTx, XTy, c.za1, c.za2, c.za3, c.za4, c.c3T, c.hz1, c.hz2);
    collide_d2q5(h, M.Cp, C, ux, uy, XCx, XCy, c.ed1, c.ed2, c.ed3, c.ed4, c.c3C, c.he1, c.he2);
}

template <typename R>
__device__ __forceinline__ void collide(const Coef<R>& c, R f[9], R g[5], R h[5], R hist[4]) {
    const Macro<R> M = macro(c, f, g, h);
    collide_flow(c, M, f);
    collide_scalars(c, M, g, h, hist);
}

// ---- SplitMix64 (Steele, Lea & Flood 2014): k-th output of a generator seeded with s
__host__ __device__ inline uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__host__ __device__ inline double uniform01(uint64_t seed, uint64_t k) {
    return (double)(splitmix64_at(seed, k) >> 11) * (1.0 / 9007199254740992.0);
}

}  // namespace lbm
