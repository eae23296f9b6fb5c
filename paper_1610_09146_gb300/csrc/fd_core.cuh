// fd_core.cuh -- device building blocks shared by the algorithm families:
// grid/physics constants, periodic neighbour offsets, the fourth-order
// central stencils (Section 2), the precision modes and the assembly of the
// residual of Eqs. 1-5 from its derivative terms.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fd_df64.cuh"

namespace fd {

// Grid of the periodic cube [0, 2*pi]^3 (Section 3); h_a = 2*pi / n_a.
// Division is avoided on the device: 1/(12 h) and 1/(12 h^2) are precomputed
// on the host (Section 2 evaluates such rationals once at start-up).
// Largest grid: ten fields of one instance must be addressable with 32-bit
// offsets (10 * n <= 2^31 - 1).
constexpr long long kMaxPoints = 214748364;

struct Grid {
    int nx, ny, nz;
    int n;               // nx * ny * nz, <= kMaxPoints
    double inv12h[3];    // 1 / (12 h_a)
    double inv12h2[3];   // 1 / (12 h_a^2)
    float inv12hf[3];
    float inv12h2f[3];
    df64 inv12h_w[3];    // as double-words (df64 mode)
    df64 inv12h2_w[3];
};

// Flow constants of Eqs. 4-7, with negative powers precomputed.
struct Phys {
    double gamma, gm1;   // gamma, gamma - 1
    double gM2;          // gamma * Mach^2
    double nu;           // 1 / Re
    double kappa;        // 1 / ((gamma - 1) Mach^2 Pr Re)
    double p0;           // 1 / (gamma Mach^2): mean pressure of the TGV state
    double rhoE0;        // p0 / (gamma - 1): mean total energy at rest
    df64 gm1_w, gM2_w, rhoE0_w;  // the same constants as double-words (df64 mode)
    df64 nu_w, kappa_w, cE_w;     // nu, kappa and rhoE0 + p0 as double-words
};

// Two-register low-storage RK3 (Section 2 / Fig. 1, read as
//   Q <- Qs + a_s dt R(Q),  Qs <- Qs + b_s dt R(Q),  Qs = Q at save-state)
// with a = (2/3, 5/12, 3/5), b = (1/4, 3/20, -).
struct RKStage {
    double adt;   // a_s * dt
    double bdt;   // b_s * dt
    int stage;    // 0, 1, 2 (stage 0 reads Q as Qs; stage 2 leaves Qs alone)
    df64 adt_w, bdt_w;  // a_s dt, b_s dt as double-words (df64 mode)
};

// Five per-variable constants (the shift of the df64 state at the API boundary).
struct Shift5 {
    double s[5];
};

// Precision modes.  T is the arithmetic of the stencils and the residual; the
// conserved state (and the RK accumulation) is kept in state_t<T>:
//   double  binary64 everywhere;
//   float   binary32 stencils on shifted fields; double-word (compensated
//           binary32, ~48 bits) state and RK accumulation;
//   df64    double-word stencils on shifted fields and a double-word state.
// A double-word state is itself shifted (rho - 1, rho u_i, rho E - rhoE0) so
// that its bits resolve the perturbations; in both of these modes no binary64
// instruction is issued in a step.
template <class T>
struct Prec;
// Whether the store-some gradient arrays carry the three pair sums of their
// diagonal (binary64 only; see the store-some kernels).
template <class T>
constexpr bool kStoresPairSums = false;
template <>
constexpr bool kStoresPairSums<double> = true;
// Whether the fused residual weights each tap value separately (binary64,
// bound by FP64 instruction issue: one FMA per tap instead of a difference,
// a scale and an accumulate per pair) or forms the unscaled differences of the
// stencil first (binary32 and double-word: the error analysis of the binary32
// mode and the exact power-of-two scalings of the double-word helpers).
template <class T>
constexpr bool kTapWeighted = false;
template <>
constexpr bool kTapWeighted<double> = true;
// Gradient arrays of the store-some / recompute-some families per precision.
template <class T>
constexpr int kGradArrays = kStoresPairSums<T> ? 12 : 9;
// Gradient arrays of the mixed binary64 / double-word store-some form: G_ii only.
constexpr int kHybGradArrays = 3;
template <>
struct Prec<double> {
    using S = double;
    static constexpr bool shifted = false;
};
template <>
struct Prec<float> {
    using S = df64;
    static constexpr bool shifted = true;
};
template <>
struct Prec<df64> {
    using S = df64;
    static constexpr bool shifted = true;
};
template <class T>
using state_t = typename Prec<T>::S;

// Linear index of a grid point and the offsets to its periodic neighbours
// at -2, -1, +1, +2 along each axis.  Offsets along different axes add, so
// the corner taps of a mixed derivative are c + o[i][a] + o[k][b].
struct Nbr {
    int c;
    int o[3][4];
};

__device__ __forceinline__ void axis_offsets(int i, int n, int stride, int* o) {
    o[0] = (i >= 2 ? -2 : n - 2) * stride;
    o[1] = (i >= 1 ? -1 : n - 1) * stride;
    o[2] = (i + 1 < n ? 1 : 1 - n) * stride;
    o[3] = (i + 2 < n ? 2 : 2 - n) * stride;
}

__device__ __forceinline__ Nbr make_nbr(const Grid& g, int idx) {
    int x = idx % g.nx;
    int t = idx / g.nx;
    int y = t % g.ny;
    int z = t / g.ny;
    Nbr s;
    s.c = idx;
    axis_offsets(x, g.nx, 1, s.o[0]);
    axis_offsets(y, g.ny, g.nx, s.o[1]);
    axis_offsets(z, g.nz, g.nx * g.ny, s.o[2]);
    return s;
}

// Fused multiply-add in the working precision.
__device__ __forceinline__ double fmx(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fmx(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// Unscaled first difference 8 (f_{+1} - f_{-1}) - (f_{+2} - f_{-2}); the
// derivative is this times 1/(12 h).  `f` maps a linear index to a value.
template <class T, class F>
__device__ __forceinline__ T delta1(F f, int c, const int* o) {
    T m2 = f(c + o[0]), m1 = f(c + o[1]), p1 = f(c + o[2]), p2 = f(c + o[3]);
    return fmx(T(8), p1 - m1, m2 - p2);
}

// Unscaled second difference 16 (f_{+1} + f_{-1}) - (f_{+2} + f_{-2}) - 30 f_0;
// the derivative is this times 1/(12 h^2).
template <class T, class F>
__device__ __forceinline__ T delta2(F f, int c, const int* o, T f0) {
    T m2 = f(c + o[0]), m1 = f(c + o[1]), p1 = f(c + o[2]), p2 = f(c + o[3]);
    return fmx(T(-30), f0, fmx(T(16), p1 + m1, -(p2 + m2)));
}

// Unscaled difference of a product formed at the taps,
//   8 (a_{+1} b_{+1} - a_{-1} b_{-1}) - (a_{+2} b_{+2} - a_{-2} b_{-2}),
// for tap values a[4], b[4] ordered -2, -1, +1, +2 (two products, three FMAs).
template <class T>
__device__ __forceinline__ T delta1_prod(const T a[4], const T b[4]) {
    T x = fmx(-a[1], b[1], a[2] * b[2]);
    T y = fmx(-a[0], b[0], a[3] * b[3]);
    return fmx(T(8), x, -y);
}

// Unscaled first difference from tap values ordered -2, -1, +1, +2.
template <class T>
__device__ __forceinline__ T delta1_taps(const T t[4]) {
    return fmx(T(8), t[2] - t[1], t[0] - t[3]);
}

// Unscaled second difference from tap values and the centre value.
template <class T>
__device__ __forceinline__ T delta2_taps(const T t[4], T f0) {
    return fmx(T(-30), f0, fmx(T(16), t[2] + t[1], -(t[3] + t[0])));
}

// Double-word forms of the three stencil helpers: the weights 8 and 16 scale
// exactly (powers of two), 30 through an exact binary32 product.  They use the unnormalised
// products and sums of fd_df64.cuh (mul_nn, add_nn): the result carries an
// absolute error of ~2^-47 of the taps' magnitude (times the weights), which is
// what a stencil difference of double-word taps resolves in any case.
__device__ __forceinline__ df64 delta1_prod(const df64 a[4], const df64 b[4]) {
    const df64 x = sub_nn(mul_nn(a[2], b[2]), mul_nn(a[1], b[1]));
    const df64 y = sub_nn(mul_nn(a[3], b[3]), mul_nn(a[0], b[0]));
    return sub_nn(scale2(x, 8.0f), y);
}
__device__ __forceinline__ df64 delta1_taps(const df64 t[4]) {
    return add_nn(scale2(sub_nn(t[2], t[1]), 8.0f), sub_nn(t[0], t[3]));
}
__device__ __forceinline__ df64 delta2_taps(const df64 t[4], df64 f0) {
    const df64 s = sub_nn(scale2(add_nn(t[2], t[1]), 16.0f), add_nn(t[3], t[0]));
    return sub_nn(s, mul_nn(f0, 30.0f));
}

// Multiply-accumulate a b + c of the fused residual's long sums: fmx in
// binary64 and binary32, the unnormalised double-word forms in df64.
__device__ __forceinline__ double acc(double a, double b, double c) { return fmx(a, b, c); }
__device__ __forceinline__ float acc(float a, float b, float c) { return fmx(a, b, c); }
__device__ __forceinline__ df64 acc(df64 a, df64 b, df64 c) { return add_nn(mul_nn(a, b), c); }
// The same for a product a b and a sum a + b, and the final renormalisation of
// a residual.
__device__ __forceinline__ double prod(double a, double b) { return a * b; }
__device__ __forceinline__ float prod(float a, float b) { return a * b; }
__device__ __forceinline__ df64 prod(df64 a, df64 b) { return mul_nn(a, b); }
__device__ __forceinline__ double sum(double a, double b) { return a + b; }
__device__ __forceinline__ float sum(float a, float b) { return a + b; }
__device__ __forceinline__ df64 sum(df64 a, df64 b) { return add_nn(a, b); }
__device__ __forceinline__ double settle(double a) { return a; }
__device__ __forceinline__ float settle(float a) { return a; }
__device__ __forceinline__ df64 settle(df64 a) { return renorm(a); }

// Per-tap weights of the binary64 fused residual (kTapWeighted), where every
// tap value enters the residual through one fused multiply-add:
//   c8[j]      = 8 c1[j]                  convective taps -1, +1 (c1[j]: taps -2, +2)
//   v16[i][j]  = 16 vs2[i][j]             Laplacian taps -1, +1 (vs2: taps -2, +2)
//   vc[i]      = -30 sum_j vs2[i][j]      Laplacian centre
//   k16[j], kc = 16 ks2[j], -30 sum_j ks2[j]   heat flux
// Empty in the other precisions, so their coefficient records keep their size
// (the batched TMA kernel holds one per block in shared memory beside its ring).
template <class T>
struct TapWeights {};
template <>
struct TapWeights<double> {
    double c8[3];
    double v16[3][3];
    double vc[3];
    double k16[3];
    double kc;
};

// Coefficients of the fused residual (RA and SS), precomputed on the host so
// that every derivative enters the residual through one multiply-add:
//   c1[j]      = -1/2 / (12 h_j)      skew convective sums (Eq. skewscalar)
//   cp[j]      = -1 / (12 h_j)        pressure gradient and pressure work
//   vs2[i][j]  = nu / (12 h_j^2), times 4/3 for j == i: the viscous Laplacian
//                plus the D_ii u_i part of the 1/3 grad(div u) term (Eq. 4)
//   vmix[i][k] = nu/3 / (12 h_i 12 h_k)   RA: D_i(D_k u_k), k != i, from u taps
//   vmix1[i]   = nu/3 / (12 h_i)          SS: D_i of the stored gradients G_kk
//   ks2[j]     = kappa / (12 h_j^2)       heat flux (Eq. 5)
//   c_rho, c_E = -1, -(rhoE0 + p0) in the binary32 perturbation form, 0 otherwise
// and, through TapWeights, the per-tap weights of the binary64 form (kTapWeighted).
template <class T>
struct Coef : TapWeights<T> {
    T s1[3];
    T c1[3];
    T cp[3];
    T vs2[3][3];
    T vmix[3][3];
    T vmix1[3];
    T ks2[3];
    T nu;
    T c_rho, c_E;
};

// Derivative terms that enter the residual at one point (physical units).
template <class T>
struct Terms {
    T G[3][3];    // D_j u_i
    T conv[5];    // sum_j [ D_j(Q_f u_j) + u_j D_j Q_f ]  for Q_f = rho, rho u_i, rho E
    T dp[3];      // D_i p
    T dpu;        // sum_j D_j(p u_j)
    T lap[3];     // sum_j D2_j u_i
    T gd[3];      // D2_i u_i + sum_{k != i} D_i(D_k u_k)   (= sum_k D_ik u_k)
    T lapT;       // sum_j D2_j T
};

// Residual of Eqs. 1-5 with the skew-symmetric convective form (Eq.
// skewscalar, phi = 1, u_i, E) and the viscous terms expanded to second
// derivatives:
//   R_f    = -1/2 [ conv_f + Q_f div ]                      (f = rho, rho u_i, rho E)
//   R_rhoui += -D_i p + nu (lap_i + gd_i / 3)
//   R_rhoE  += -sum_j D_j(p u_j) + kappa lapT
//              + nu sum_ij (G_ij + G_ji - 2/3 delta_ij div) G_ij + u_i nu (lap_i + gd_i / 3)
//
// In the perturbation form of the binary32 mode the fields are rho' = rho-1,
// rho u_i, E' = rho E - rhoE0, p' = p - p0, T' = T - 1.  By linearity of D,
// conv_rho and conv_rhoE then lack the terms div and rhoE0 div, and
// sum_j D_j(p u_j) lacks p0 div; `c_rho` and `c_E` add them back:
//   R_rho  -= c_rho div   (c_rho = 1)
//   R_rhoE -= c_E div     (c_E = rhoE0 + p0)
// (both 0 in the binary64 mode, where the fields are not shifted).
template <class T>
__device__ __forceinline__ void assemble(const Terms<T>& t, const T q[5], const T u[3], T nu, T kappa,
                                         T c_rho, T c_E, T R[5]) {
    T div = t.G[0][0] + t.G[1][1] + t.G[2][2];
#pragma unroll
    for (int f = 0; f < 5; ++f) R[f] = T(-0.5) * fmx(q[f], div, t.conv[f]);
    R[0] = fmx(-c_rho, div, R[0]);
    R[4] = fmx(-c_E, div, R[4]);
    T work = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        T vi = nu * fmx(t.gd[i], T(1.0 / 3.0), t.lap[i]);
        R[1 + i] += vi - t.dp[i];
        work = fmx(u[i], vi, work);
    }
    T diss = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            T s = t.G[i][j] + t.G[j][i];
            if (i == j) s = fmx(T(-2.0 / 3.0), div, s);
            diss = fmx(s, t.G[i][j], diss);
        }
    R[4] += fmx(nu, diss, fmx(kappa, t.lapT, work)) - t.dpu;
}

}  // namespace fd
