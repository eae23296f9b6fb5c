// fd_kernels.cu -- kernels of one Runge-Kutta stage for the five algorithm
// families of Section 2 (BL store-all, SS store-some, RA recompute-all, RS
// recompute-some, SN store-none), the Taylor-Green initial condition and the
// kinetic-energy / enstrophy reduction (Section 3), and the batched forms.
//
// Layout: every field is a grid-sized array [z][y][x] (x fastest).  The
// conserved state Q (rho, rho u, rho v, rho w, rho E) and the saved RK
// register Qs are binary64, or shifted double-words (rho - 1, rho u_i,
// rho E - rhoE0) in the binary32 and df64 modes.  The stencils read ten
// "working" fields:  Qf = five conserved-like fields, Wf = five
// primitive-like fields.
//   binary64 mode (T = double): Qf = Q itself, Wf = (u, v, w, p, T).
//   binary32 / df64 (T = float / df64):
//                       Qf = (rho-1, rho u, rho v, rho w, rho E - rhoE0),
//                       Wf = (u, v, w, p - p0, T - 1),
// the shifted (perturbation) fields avoid the loss of digits that the large
// mean pressure and energy (p0 = 1/(gamma M^2)) would cause in the
// differences.  One thread evaluates one grid point (RS: one thread per point
// and equation), except the z-marching recompute-all kernels (binary32 and
// df64), where a block stages planes of a tile in shared memory; periodic
// boundaries (Section 3) are the wrapped neighbour offsets of fd::Nbr, modulo
// halo indices (thread-staged tiles), or a ghost-padded field layout for the
// TMA-staged binary32 recompute-all kernel.
//
// Sections: initial condition; primitives and the RK update; the fused
// residual (RA, SS) and its accessors; RA (global memory, shared-memory
// tiled, TMA-staged); SS; BL; SN and RS; the batched kernels; diagnostics;
// launchers.
//
// On GB300 binary64 issues at 1/64 of the binary32 rate, so the binary64
// kernels are bound by FP64 instructions per point, not by memory traffic;
// stencil taps are read through the read-only data cache, and the binary64
// fused residual weights every tap through one FMA (kTapWeighted).
#include <cuda.h>

#include <cstdlib>
#include <type_traits>

#include "fd_core.cuh"
#include "fd_internal.h"

namespace fd {

namespace {

template <class T>
__device__ __forceinline__ T ld(const T* __restrict__ p, int i) {
    return __ldg(p + i);
}
__device__ __forceinline__ df64 ld(const df64* __restrict__ p, int i) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p + i));
    return df64(v.x, v.y);
}

__device__ __forceinline__ int grid_index() { return blockIdx.x * blockDim.x + threadIdx.x; }

template <class T>
__device__ __forceinline__ T s1(const Grid& g, int a);
template <>
__device__ __forceinline__ double s1<double>(const Grid& g, int a) {
    return g.inv12h[a];
}
template <>
__device__ __forceinline__ float s1<float>(const Grid& g, int a) {
    return g.inv12hf[a];
}
template <>
__device__ __forceinline__ df64 s1<df64>(const Grid& g, int a) {
    return g.inv12h_w[a];
}
template <class T>
__device__ __forceinline__ T s2(const Grid& g, int a);
template <>
__device__ __forceinline__ double s2<double>(const Grid& g, int a) {
    return g.inv12h2[a];
}
template <>
__device__ __forceinline__ float s2<float>(const Grid& g, int a) {
    return g.inv12h2f[a];
}
template <>
__device__ __forceinline__ df64 s2<df64>(const Grid& g, int a) {
    return g.inv12h2_w[a];
}

// Constants that restore the mean-field terms removed by the shift (see
// fd::assemble): zero in binary64 mode.
template <class T>
struct Shift {
    T c_rho, c_E;
};
template <class T>
__device__ __forceinline__ Shift<T> shift_of(const Phys& ph);
template <>
__device__ __forceinline__ Shift<double> shift_of<double>(const Phys&) {
    return {0.0, 0.0};
}
template <>
__device__ __forceinline__ Shift<float> shift_of<float>(const Phys& ph) {
    return {1.0f, (float)(ph.rhoE0 + ph.p0)};
}
template <>
__device__ __forceinline__ Shift<df64> shift_of<df64>(const Phys& ph) {
    return {df64(1.0f, 0.0f), ph.cE_w};
}

// nu and kappa in the working precision.
__device__ __forceinline__ void visc_consts(const Phys& ph, double& nu, double& ka) {
    nu = ph.nu;
    ka = ph.kappa;
}
__device__ __forceinline__ void visc_consts(const Phys& ph, float& nu, float& ka) {
    nu = (float)ph.nu;
    ka = (float)ph.kappa;
}
__device__ __forceinline__ void visc_consts(const Phys& ph, df64& nu, df64& ka) {
    nu = ph.nu_w;
    ka = ph.kappa_w;
}

// The stage's residual in the state precision, and the RK constants in it.
__device__ __forceinline__ double to_state(double r) { return r; }
__device__ __forceinline__ df64 to_state(float r) { return df64(r, 0.0f); }
__device__ __forceinline__ df64 to_state(df64 r) { return r; }
// a R + q for the update: a binary32 residual multiplies a double-word
// constant with the cheaper double-word x binary32 product.
__device__ __forceinline__ double upd(double a, double r, double q) { return fmx(a, r, q); }
__device__ __forceinline__ df64 upd(df64 a, df64 r, df64 q) { return fmx(a, r, q); }
__device__ __forceinline__ df64 upd(df64 a, float r, df64 q) { return times_fp(a, r) + q; }
__device__ __forceinline__ double rk_a(const RKStage& rk, double) { return rk.adt; }
__device__ __forceinline__ df64 rk_a(const RKStage& rk, df64) { return rk.adt_w; }
__device__ __forceinline__ double rk_b(const RKStage& rk, double) { return rk.bdt; }
__device__ __forceinline__ df64 rk_b(const RKStage& rk, df64) { return rk.bdt_w; }

}  // namespace

// ---------------------------------------------------------------- Section 3
// Taylor-Green vortex (DeBonis 2013, cited in Section 3).
// Plane k of the array is plane (k + z0) mod nzp of the periodic grid (z0 = 0,
// nzp = nz for a whole grid; a slab of the z-slab decomposition passes its offset).
__global__ void k_tgv_ic(Grid g, Phys ph, double hx, double hy, double hz, int z0, int nzp,
                         double* __restrict__ Q) {
    int idx = grid_index();
    if (idx >= g.n) return;
    int i = idx % g.nx, t = idx / g.nx, j = t % g.ny, k = ((t / g.ny + z0) % nzp + nzp) % nzp;
    double sx, cx, sy, cy, sz, cz, s2x, c2x, s2y, c2y, s2z, c2z;
    sincos(i * hx, &sx, &cx);
    sincos(j * hy, &sy, &cy);
    sincos(k * hz, &sz, &cz);
    sincos(2.0 * (i * hx), &s2x, &c2x);
    sincos(2.0 * (j * hy), &s2y, &c2y);
    sincos(2.0 * (k * hz), &s2z, &c2z);
    double u = sx * cy * cz;
    double v = -cx * sy * cz;
    double p = ph.p0 + (c2x + c2y) * (c2z + 2.0) * (1.0 / 16.0);
    double rho = ph.gM2 * p;
    int n = g.n;
    Q[idx] = rho;
    Q[n + idx] = rho * u;
    Q[2 * n + idx] = rho * v;
    Q[3 * n + idx] = 0.0;
    Q[4 * n + idx] = p / ph.gm1 + 0.5 * rho * (u * u + v * v);
}

// ------------------------------------------------------- Section 2, Eqs. 6-7
// binary64: u_i = rho u_i / rho, p = (gamma-1)(rho E - rho u_i u_i / 2),
// T = gamma M^2 p / rho, written to W = (u, v, w, p, T) at point c.
__device__ __forceinline__ void prims_point(const Phys& ph, const double q[5], double* __restrict__ W, int n,
                                            int c) {
    double inv = 1.0 / q[0];
    double u = q[1] * inv, v = q[2] * inv, w = q[3] * inv;
    double p = ph.gm1 * fmx(-0.5, fmx(q[1], u, fmx(q[2], v, q[3] * w)), q[4]);
    W[c] = u;
    W[n + c] = v;
    W[2 * n + c] = w;
    W[3 * n + c] = p;
    W[4 * n + c] = ph.gM2 * p * inv;
}

// binary32 perturbation fields F = (rho-1, rho u, rho v, rho w, rhoE-rhoE0,
// u, v, w, p-p0, T-1) from the shifted double-word state (q0 = rho - 1,
// q4 = rho E - rhoE0).  With p0 = (gamma-1) rhoE0 and gamma M^2 p0 = 1, Eqs.
// 6-7 become
//   p - p0 = (gamma-1)(E' - rho u_i u_i / 2),  T - 1 = (gamma M^2 (p-p0) - rho') / rho.
__device__ __forceinline__ float to_f32(df64 x) { return __fadd_rn(x.hi, x.lo); }
__device__ __forceinline__ void prims_values(const Phys& ph, const df64 q[5], float v[10]) {
    float rp = to_f32(q[0]);
    float Ep = to_f32(q[4]);
    float m0 = to_f32(q[1]), m1 = to_f32(q[2]), m2 = to_f32(q[3]);
    float inv = 1.0f / to_f32(q[0] + df64(1.0f, 0.0f));
    float u = m0 * inv, v_ = m1 * inv, w = m2 * inv;
    float pp = ph.gm1_w.hi * fmx(-0.5f, fmx(m0, u, fmx(m1, v_, m2 * w)), Ep);
    float Tp = fmx(ph.gM2_w.hi, pp, -rp) * inv;
    v[0] = rp;
    v[1] = m0;
    v[2] = m1;
    v[3] = m2;
    v[4] = Ep;
    v[5] = u;
    v[6] = v_;
    v[7] = w;
    v[8] = pp;
    v[9] = Tp;
}
__device__ __forceinline__ void prims_point(const Phys& ph, const df64 q[5], float* __restrict__ F, int n, int c) {
    float v[10];
    prims_values(ph, q, v);
#pragma unroll
    for (int f = 0; f < 10; ++f) F[(size_t)f * n + c] = v[f];
}

// Ghost-padded layout of the binary32 working fields of the TMA-staged
// recompute-all kernel: each field is an (nx + 4) x (ny + 4) x nz array that
// holds x = -2 .. nx+1 and y = -2 .. ny+1, and the cells x = -2, -1, nx, nx+1
// and y = -2, -1, ny, ny+1 hold the periodic images, written by whoever writes
// the point they copy.  The box of the tile at x0 then starts at padded column
// x0 (a multiple of 32 floats, so on a 16-byte boundary) and covers
// x0 - 2 .. x0 + 33; rows are nx + 4 floats, a multiple of 16 bytes when
// nx % 4 = 0; no tile needs a special case at the periodic boundary.
struct PadLayout {
    int nx, ny, px, py;
    long long np;  // points per padded field
    __device__ __forceinline__ long long at(int x, int y, int z) const {
        return ((long long)z * py + (y + 2)) * px + (x + 2);
    }
};
__host__ __device__ __forceinline__ PadLayout pad_layout(const Grid& g) {
    PadLayout L;
    L.nx = g.nx;
    L.ny = g.ny;
    L.px = g.nx + 4;
    L.py = g.ny + 4;
    L.np = (long long)L.px * L.py * g.nz;
    return L;
}
// Write the ten values of point (x, y, z) and its periodic images.
__device__ __forceinline__ void put_padded(const PadLayout& L, float* __restrict__ F, int x, int y, int z,
                                           const float v[10]) {
    const int x2 = x < 2 ? x + L.nx : (x >= L.nx - 2 ? x - L.nx : x);
    const int y2 = y < 2 ? y + L.ny : (y >= L.ny - 2 ? y - L.ny : y);
    const int xs[2] = {x, x2}, ys[2] = {y, y2};
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        if (b == 1 && y2 == y) break;
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            if (a == 1 && x2 == x) break;
            const long long i = L.at(xs[a], ys[b], z);
#pragma unroll
            for (int f = 0; f < 10; ++f) F[f * L.np + i] = v[f];
        }
    }
}

// Double-word perturbation fields from the double-word state, which is itself
// stored shifted (q0 = rho - 1, q4 = rho E - rhoE0): the binary32 formulas
// above in double-word arithmetic (1/rho by one Newton step).
__device__ __forceinline__ void prims_point(const Phys& ph, const df64 q[5], df64* __restrict__ F, int n, int c) {
    const df64 rp = q[0];
    const df64 Ep = q[4];
    const df64 inv = recip(q[0] + df64(1.0f, 0.0f));
    const df64 u = q[1] * inv, v = q[2] * inv, w = q[3] * inv;
    const df64 pp = ph.gm1_w * fmx(df64(-0.5f, 0.0f), fmx(q[1], u, fmx(q[2], v, q[3] * w)), Ep);
    const df64 Tp = fmx(ph.gM2_w, pp, -rp) * inv;
    F[c] = rp;
    F[n + c] = q[1];
    F[2 * n + c] = q[2];
    F[3 * n + c] = q[3];
    F[4 * n + c] = Ep;
    F[5 * n + c] = u;
    F[6 * n + c] = v;
    F[7 * n + c] = w;
    F[8 * n + c] = pp;
    F[9 * n + c] = Tp;
}

// Primitives of the whole state (at creation, after fd_set_state, or when
// no stage has produced them yet).
template <class T>
__global__ void __launch_bounds__(256) k_prims(Grid g, Phys ph, const state_t<T>* __restrict__ Q,
                                               T* __restrict__ W) {
    int idx = grid_index();
    if (idx >= g.n) return;
    const int n = g.n;
    state_t<T> q[5];
#pragma unroll
    for (int f = 0; f < 5; ++f) q[f] = Q[f * n + idx];
    prims_point(ph, q, W, n, idx);
}

// The same, into the ghost-padded layout (TMA-staged binary32 recompute-all).
__global__ void __launch_bounds__(256) k_prims_padded(Grid g, Phys ph, const df64* __restrict__ Q,
                                                      float* __restrict__ F) {
    int idx = grid_index();
    if (idx >= g.n) return;
    const int n = g.n;
    df64 q[5];
#pragma unroll
    for (int f = 0; f < 5; ++f) q[f] = Q[f * n + idx];
    float v[10];
    prims_values(ph, q, v);
    put_padded(pad_layout(g), F, idx % g.nx, (idx / g.nx) % g.ny, idx / (g.nx * g.ny), v);
}

// RK update from a preloaded saved register qs (Q_in at stage 0, else Qs):
// the same arithmetic as the update branch of stage_write below.
template <class T, class S = state_t<T>>
__device__ __forceinline__ void stage_update(const RKStage& rk, const Phys& ph, int n, int c, const S qs[5],
                                             const T R[5], S* __restrict__ out, S* __restrict__ Qs,
                                             T* __restrict__ Wnext) {
    S qn[5];
#pragma unroll
    for (int f = 0; f < 5; ++f) {
        qn[f] = upd(rk_a(rk, S()), R[f], qs[f]);
        out[f * n + c] = qn[f];
        if (rk.stage < 2) Qs[f * n + c] = upd(rk_b(rk, S()), R[f], qs[f]);
    }
    prims_point(ph, qn, Wnext, n, c);
}

// Final write of a stage: the residual itself (fd_residual), or the
// two-register RK update (Fig. 1, advance-solution-in-time) in the state
// precision (binary64, or double-word in the binary32 and df64 modes),
//   Q_out = Qs + a dt R,  Qs <- Qs + b dt R,  with Qs = Q_in at stage 0 (save-state),
// followed by the primitives of Q_out for the next stage (evaluate-u_i,p,T of
// Fig. 1 moved to the end of the previous stage: it is pointwise, so the point
// that produces Q_out can produce them without another pass over memory).
template <class T, bool RESID, class S = state_t<T>>
__device__ __forceinline__ void stage_write(const RKStage& rk, const Phys& ph, int n, int c,
                                            const S* __restrict__ Q64, const T R[5], S* __restrict__ out,
                                            S* __restrict__ Qs, T* __restrict__ Wnext) {
    S qn[5];
#pragma unroll
    for (int f = 0; f < 5; ++f) {
        if (RESID) {
            out[f * n + c] = to_state(R[f]);
        } else {
            const S qs = rk.stage == 0 ? Q64[f * n + c] : Qs[f * n + c];
            qn[f] = upd(rk_a(rk, S()), R[f], qs);
            out[f * n + c] = qn[f];
            if (rk.stage < 2) Qs[f * n + c] = upd(rk_b(rk, S()), R[f], qs);
        }
    }
    if (!RESID) prims_point(ph, qn, Wnext, n, c);
}

// Load the four taps (-2, -1, +1, +2) of field f around c along one axis.
template <class T>
__device__ __forceinline__ void taps(const T* __restrict__ f, int c, const int* o, T t[4]) {
#pragma unroll
    for (int a = 0; a < 4; ++a) t[a] = ld(f, c + o[a]);
}

// Where the fused residual reads its fields.  Field index f: 0..4 the
// conserved-like working fields Qf, 5..9 the primitive-like fields Wf (u, v,
// w, p, T).  Taps are ordered -2, -1, +1, +2 along an axis (0 = x, 1 = y,
// 2 = z).  The global accessor reads through the read-only cache with the
// periodic neighbour offsets; the shared-memory accessor (tiled kernel) reads a
// staged ring of planes.  Both feed the same arithmetic below.
template <class T>
struct GlobalAcc {
    static constexpr bool kZQueue = false;
    const Nbr& s;
    int n;
    const T* __restrict__ Qf;
    const T* __restrict__ Wf;
    const T* __restrict__ Gw;
    __device__ __forceinline__ const T* field(int f) const { return f < 5 ? Qf + f * n : Wf + (f - 5) * n; }
    __device__ __forceinline__ T center(int f) const { return ld(field(f), s.c); }
    __device__ __forceinline__ void taps(int f, int j, T t[4]) const {
        const T* p = field(f);
#pragma unroll
        for (int a = 0; a < 4; ++a) t[a] = ld(p, s.c + s.o[j][a]);
    }
    // taps along j around the point shifted by tap a along axis i
    __device__ __forceinline__ void taps_shifted(int f, int j, int i, int a, T t[4]) const {
        const T* p = field(f);
        const int c = s.c + s.o[i][a];
#pragma unroll
        for (int b = 0; b < 4; ++b) t[b] = ld(p, c + s.o[j][b]);
    }
    __device__ __forceinline__ T grad(int i, int j) const { return ld(Gw + (3 * i + j) * n, s.c); }
    // taps along i of the stored gradient G_ab
    __device__ __forceinline__ void grad_taps(int ga, int gb, int i, T t[4]) const {
        const T* p = Gw + (3 * ga + gb) * n;
#pragma unroll
        for (int a = 0; a < 4; ++a) t[a] = ld(p, s.c + s.o[i][a]);
    }
    // taps along i of G_aa + G_bb, summed at each tap
    __device__ __forceinline__ void grad_pair_taps(int ga, int gb, int i, T t[4]) const {
        const T* pa = Gw + (3 * ga + ga) * n;
        const T* pb = Gw + (3 * gb + gb) * n;
#pragma unroll
        for (int a = 0; a < 4; ++a) t[a] = ld(pa, s.c + s.o[i][a]) + ld(pb, s.c + s.o[i][a]);
    }
    // taps along i of the stored pair sum P_i = G_jj + G_kk (j, k the other axes)
    __device__ __forceinline__ void pair_taps(int i, T t[4]) const {
        const T* p = Gw + 9 * (size_t)n + (size_t)i * n;
#pragma unroll
        for (int a = 0; a < 4; ++a) t[a] = ld(p, s.c + s.o[i][a]);
    }
};

// Residual at one point for the fused families, evaluated into registers
// (the "thread-local variables" of Section 2, paragraphs SN / SS):
//   R_f = -1/2 sum_j [ D_j(Q_f u_j) + u_j D_j Q_f ] - 1/2 Q_f div u         (Eq. skewscalar)
//   R_rho u_i += -D_i p + v_i,   v_i = nu [ sum_j D2_j u_i + 1/3 sum_k D_ik u_k ]   (Eqs. 2, 4)
//   R_rho E   += -sum_j D_j(p u_j) + kappa sum_j D2_j T + sum_i u_i v_i
//                + nu [ 2 sum_i G_ii^2 + sum_{i<j} (G_ij + G_ji)^2 - 2/3 div^2 ]  (Eqs. 3-5)
// with G_ij = D_j u_i.  The convective pair of each direction is one
// difference of the product Q_f (u_j + u_j(centre)) formed at the taps, equal
// to D_j(Q_f u_j) + u_j D_j Q_f by linearity of the stencil.  In binary64
// (kTapWeighted) the stencil weight of each tap is folded into that product's
// velocity factor and every tap value enters through one FMA (the same sums,
// associated per tap instead of per difference), and the viscous terms come
// first so that each momentum residual starts as Q_f (-div/2) + v_i in one
// FMA.  STORED_G: SS reads G from the nine gradient arrays and, for the mixed
// derivatives, differences P_i = G_jj + G_kk (stored by the gradient pass in
// binary64, summed at the taps otherwise); without it (RA) G and D_i(D_k u_k)
// come from u taps.
//
// PGRAD = false leaves the pressure gradient -D_i p out of the momentum
// residuals (the mixed binary64 / double-word kernel adds it in binary64).
// PART (not in the binary64 tap-weighted form): 0 the whole residual; 1 the
// convective part (Q_f (-div/2), the convective sums, the pressure gradient,
// the mean-state terms); 2 the rest (pressure work, heat flux, viscous stress
// divergence and its work, dissipation), so that two kernels can each
// evaluate one part.
template <class T, bool STORED_G, class Acc, bool PGRAD = true, int PART = 0>
__device__ __forceinline__ void fused_residual(const Acc& A, const Coef<T>& k, T R[5]) {
    static_assert(PART == 0 || !kTapWeighted<T>, "the binary64 tap-weighted residual is not split");
    constexpr int U = 5, P = 8, TT = 9;  // field indices of u_0, p, T
    T uc[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) uc[i] = A.center(U + i);

    T G[3][3];
    if constexpr (STORED_G) {
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) G[i][j] = A.grad(i, j);
    } else {
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                T t[4];
                A.taps(U + i, j, t);
                G[i][j] = k.s1[j] * delta1_taps(t);
            }
    }
    const T div = sum(sum(G[0][0], G[1][1]), G[2][2]);
    const T hd = prod(T(-0.5), div);
    // viscous stress divergence v_i = nu [ sum_j D2_j u_i + 1/3 sum_k D_ik u_k ]
    auto viscous = [&](int i) {
        T vi = 0;
        if constexpr (kTapWeighted<T>) {
            vi = k.vc[i] * uc[i];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                T t[4];
                A.taps(U + i, j, t);
                vi = fmx(k.v16[i][j], t[1], vi);
                vi = fmx(k.v16[i][j], t[2], vi);
                vi = fmx(-k.vs2[i][j], t[0], vi);
                vi = fmx(-k.vs2[i][j], t[3], vi);
            }
        } else {
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                T t[4];
                A.taps(U + i, j, t);
                vi = acc(k.vs2[i][j], delta2_taps(t, uc[i]), vi);
            }
        }
        const int j1 = i == 0 ? 1 : 0, j2 = i == 2 ? 1 : 2;  // the two axes other than i
        if constexpr (STORED_G) {
            T t[4];
            if constexpr (kStoresPairSums<T>)
                A.pair_taps(i, t);
            else
                A.grad_pair_taps(j1, j2, i, t);
            vi = acc(k.vmix1[i], delta1_taps(t), vi);
        } else {
            bool queued = false;
            if constexpr (Acc::kZQueue) {
                if (i == 2) {  // D_z(D_x u_x + D_y u_y) from the queued planes
                    const T t[4] = {A.zq[0], A.zq[1], A.zq[3], A.zq[4]};
                    vi = acc(k.vmix1[2], delta1_taps(t), vi);
                    queued = true;
                }
            }
#pragma unroll
            for (int q = 0; q < (queued ? 0 : 2); ++q) {
                const int kk = q == 0 ? j1 : j2;
                T t[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    T u4[4];
                    A.taps_shifted(U + kk, kk, i, a, u4);
                    t[a] = delta1_taps(u4);
                }
                vi = acc(k.vmix[i][kk], delta1_taps(t), vi);
            }
        }
        return vi;
    };
    // binary64: the viscous terms first, so that each momentum residual starts
    // as Q_f hd + v_i in one FMA
    [[maybe_unused]] T vis[3];
    if constexpr (kTapWeighted<T>) {
#pragma unroll
        for (int i = 0; i < 3; ++i) vis[i] = viscous(i);
        R[0] = A.center(0) * hd;
#pragma unroll
        for (int i = 0; i < 3; ++i) R[1 + i] = fmx(A.center(1 + i), hd, vis[i]);
        R[4] = A.center(4) * hd;
    } else if constexpr (PART == 2) {
#pragma unroll
        for (int f = 0; f < 5; ++f) R[f] = T(0);
    } else {
#pragma unroll
        for (int f = 0; f < 5; ++f) R[f] = prod(A.center(f), hd);
    }

    // convective sums, pressure gradient and pressure work, direction by direction
    if constexpr (kTapWeighted<T>) {
        // w_a (u_j(tap a) + u_j(centre)) with the stencil weight w_a of tap a
        // folded in once per direction; each of the five fields then adds
        // Q_f(tap a) times it, one FMA per tap.  The pressure work sums
        // p(tap a) w_a u_j(tap a) (c1 = cp / 2, doubled at the end).
        T pw = 0;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            T ut[4], pt[4], wu[4], ws[4];
            A.taps(U + j, j, ut);
            A.taps(P, j, pt);
            const T w[4] = {k.c1[j], -k.c8[j], k.c8[j], -k.c1[j]};
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                wu[a] = w[a] * ut[a];
                ws[a] = fmx(w[a], uc[j], wu[a]);
            }
#pragma unroll
            for (int f = 0; f < 5; ++f) {
                T qt[4];
                A.taps(f, j, qt);
#pragma unroll
                for (int a = 0; a < 4; ++a) R[f] = fmx(qt[a], ws[a], R[f]);
            }
            if constexpr (PGRAD) R[1 + j] = fmx(k.cp[j], delta1_taps(pt), R[1 + j]);
#pragma unroll
            for (int a = 0; a < 4; ++a) pw = fmx(pt[a], wu[a], pw);
        }
        R[4] = fmx(T(2), pw, R[4]);
    } else if constexpr (PART != 2) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            T ut[4], st[4], pt[4];
            A.taps(U + j, j, ut);
            A.taps(P, j, pt);
#pragma unroll
            for (int a = 0; a < 4; ++a) st[a] = sum(ut[a], uc[j]);
#pragma unroll
            for (int f = 0; f < 5; ++f) {
                T qt[4];
                A.taps(f, j, qt);
                R[f] = acc(k.c1[j], delta1_prod(qt, st), R[f]);
            }
            if constexpr (PGRAD) R[1 + j] = acc(k.cp[j], delta1_taps(pt), R[1 + j]);
            if constexpr (PART == 0) R[4] = acc(k.cp[j], delta1_prod(pt, ut), R[4]);
        }
    }
    // split residual: the pressure work goes with the rest, whose pressure
    // gradient and viscous terms load the same p and u_j taps
    if constexpr (PART == 2) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            T ut[4], pt[4];
            A.taps(U + j, j, ut);
            A.taps(P, j, pt);
            R[4] = acc(k.cp[j], delta1_prod(pt, ut), R[4]);
        }
    }

    // heat flux
    if constexpr (PART != 1) {
        const T T0 = A.center(TT);
        if constexpr (kTapWeighted<T>) {
            T h = fmx(k.kc, T0, R[4]);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                T t[4];
                A.taps(TT, j, t);
                h = fmx(k.k16[j], t[1], h);
                h = fmx(k.k16[j], t[2], h);
                h = fmx(-k.ks2[j], t[0], h);
                h = fmx(-k.ks2[j], t[3], h);
            }
            R[4] = h;
        } else {
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                T t[4];
                A.taps(TT, j, t);
                R[4] = acc(k.ks2[j], delta2_taps(t, T0), R[4]);
            }
        }
    }

    // viscous stress divergence and its work
    if constexpr (kTapWeighted<T>) {
#pragma unroll
        for (int i = 0; i < 3; ++i) R[4] = fmx(uc[i], vis[i], R[4]);
    } else if constexpr (PART != 1) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const T vi = viscous(i);
            R[1 + i] = sum(R[1 + i], vi);
            R[4] = acc(uc[i], vi, R[4]);
        }
    }

    // viscous dissipation tau_ij D_j u_i
    if constexpr (PART != 1) {
        T d = prod(G[0][0], G[0][0]);
        d = acc(G[1][1], G[1][1], d);
        d = acc(G[2][2], G[2][2], d);
        T s01 = sum(G[0][1], G[1][0]), s02 = sum(G[0][2], G[2][0]), s12 = sum(G[1][2], G[2][1]);
        T o = prod(s01, s01);
        o = acc(s02, s02, o);
        o = acc(s12, s12, o);
        T diss = acc(T(2), d, o);
        diss = acc(prod(T(-2.0 / 3.0), div), div, diss);
        R[4] = acc(k.nu, diss, R[4]);
    }
    // the perturbation form's mean-state terms (binary64 fields are not shifted)
    if constexpr (!std::is_same<T, double>::value && PART != 2) {
        if (k.c_rho != T(0)) {
            R[0] = acc(k.c_rho, div, R[0]);
            R[4] = acc(k.c_E, div, R[4]);
        }
    }
#pragma unroll
    for (int f = 0; f < 5; ++f) R[f] = settle(R[f]);
}

// ------------------------------------------------------------------ RA
// Recompute-all (Section 2, paragraph RA): every derivative, including the
// products inside a derivative and the 4x4-tap mixed derivatives, is
// evaluated from its finite-difference formula at the point of use.
template <class T, bool RESID>
__global__ void __launch_bounds__(128) k_ra(Grid g, Coef<T> k, Phys ph, RKStage rk, const T* __restrict__ Qf,
                                            const T* __restrict__ Wf, const state_t<T>* __restrict__ Q64,
                                            state_t<T>* __restrict__ out, state_t<T>* __restrict__ Qs,
                                            T* __restrict__ Wnext) {
    int idx = grid_index();
    if (idx >= g.n) return;
    const Nbr s = make_nbr(g, idx);
    T R[5];
    fused_residual<T, false>(GlobalAcc<T>{s, g.n, Qf, Wf, nullptr}, k, R);
    stage_write<T, RESID>(rk, ph, g.n, s.c, Q64, R, out, Qs, Wnext);
}

// Recompute-all with the primitives recomputed at every tap (binary64): the
// paragraph RA of Section 2 read literally, with nothing but the state in
// memory -- no primitive arrays (which every other family stores, as the
// paragraph after Fig. 1 has it).  Each tap's u_i, p or T comes from that
// tap's five conserved values with the binary64 path's formulas (Eqs. 6-7),
// so the arithmetic per value is that of the stored primitives; a point
// evaluates them at every tap of every stencil that needs them.
struct InlineAcc {
    static constexpr bool kZQueue = false;
    const Nbr& s;
    int n;
    const double* __restrict__ Q;
    double gm1, gM2;
    __device__ __forceinline__ double q(int f, int i) const { return ld(Q + f * n, i); }
    // field f at linear index i: 0..4 the state, 5..7 u_i, 8 p, 9 T
    __device__ __forceinline__ double at(int f, int i) const {
        if (f < 5) return q(f, i);
        const double inv = 1.0 / q(0, i);
        if (f < 8) return q(f - 4, i) * inv;
        const double m0 = q(1, i), m1 = q(2, i), m2 = q(3, i);
        const double p = gm1 * fmx(-0.5, fmx(m0, m0 * inv, fmx(m1, m1 * inv, m2 * (m2 * inv))), q(4, i));
        return f == 8 ? p : gM2 * p * inv;
    }
    __device__ __forceinline__ double center(int f) const { return at(f, s.c); }
    __device__ __forceinline__ void taps(int f, int j, double t[4]) const {
#pragma unroll
        for (int a = 0; a < 4; ++a) t[a] = at(f, s.c + s.o[j][a]);
    }
    __device__ __forceinline__ void taps_shifted(int f, int j, int i, int a, double t[4]) const {
        const int c = s.c + s.o[i][a];
#pragma unroll
        for (int b = 0; b < 4; ++b) t[b] = at(f, c + s.o[j][b]);
    }
};

template <bool RESID>
__global__ void __launch_bounds__(128) k_ra_inline(Grid g, Coef<double> k, Phys ph, RKStage rk,
                                                   const double* __restrict__ Q64, double* __restrict__ out,
                                                   double* __restrict__ Qs) {
    const int idx = grid_index();
    if (idx >= g.n) return;
    const int n = g.n;
    const Nbr s = make_nbr(g, idx);
    double R[5];
    fused_residual<double, false>(InlineAcc{s, n, Q64, ph.gm1, ph.gM2}, k, R);
#pragma unroll
    for (int f = 0; f < 5; ++f) {
        if constexpr (RESID) {
            out[f * n + s.c] = R[f];
        } else {
            const double qs = rk.stage == 0 ? Q64[f * n + s.c] : Qs[f * n + s.c];
            out[f * n + s.c] = fmx(rk.adt, R[f], qs);
            if (rk.stage < 2) Qs[f * n + s.c] = fmx(rk.bdt, R[f], qs);
        }
    }
}

// Recompute-all with shared-memory staging (binary32 and df64 modes).  A block of
// kTX x kTY threads owns that x-y tile and marches a chunk of z-planes; the
// ten working fields of planes z-2 .. z+2, each with a two-point x-y halo
// (periodic, by modulo index), sit in a ring of five shared-memory planes.
// Each step of the march stages one new plane (one coalesced read of every
// field per point plus the halo) and evaluates the points of plane z from
// shared memory with the same arithmetic as k_ra.  The saved register the
// update needs is loaded before the stencil work so its latency overlaps it.
constexpr int kTX = 32, kTY = 8, kSX = kTX + 4, kSY = kTY + 4, kPlane = kSX * kSY, kRing = 5, kNF = 10;
constexpr int kZChunk = 64;

// Shared-memory accessor over a ring of staged planes: plane slot s, field f,
// row ty + OY + dy, column tx + OX + dx of an SX x SY array per field.
template <class T, int SX, int SY, int OX, int OY, bool ZQ = false>
struct SmemAccT {
    // ZQ: the z-marching kernels keep A = D_x u_x + D_y u_y of planes z-2 .. z+2
    // of the thread's column in registers (zq), so D_z(D_x u_x + D_y u_y) is one
    // difference of five queued values instead of 32 shared-memory taps.
    static constexpr bool kZQueue = ZQ;
    const T* sm;
    int slot[5];  // ring slots of planes z-2 .. z+2
    int tx, ty;
    const T* zq = nullptr;
    __device__ __forceinline__ T at(int f, int dz, int dy, int dx) const {
        return sm[((slot[dz + 2] * kNF + f) * SY + (ty + OY + dy)) * SX + (tx + OX + dx)];
    }
    __device__ __forceinline__ static int d(int a) { return a < 2 ? a - 2 : a - 1; }
    __device__ __forceinline__ T center(int f) const { return at(f, 0, 0, 0); }
    __device__ __forceinline__ void taps(int f, int j, T t[4]) const {
#pragma unroll
        for (int a = 0; a < 4; ++a)
            t[a] = j == 0 ? at(f, 0, 0, d(a)) : (j == 1 ? at(f, 0, d(a), 0) : at(f, d(a), 0, 0));
    }
    __device__ __forceinline__ void taps_shifted(int f, int j, int i, int a, T t[4]) const {
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            int o[3] = {0, 0, 0};
            o[i] += d(a);
            o[j] += d(b);
            t[b] = at(f, o[2], o[1], o[0]);
        }
    }
    // D_x u_x + D_y u_y at the thread's column, plane z + dz (fields 5, 6: u, v)
    __device__ __forceinline__ T gxx_gyy(int dz, const Coef<T>& k) const {
        T tu[4], tv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            tu[a] = at(5, dz, 0, d(a));
            tv[a] = at(6, dz, d(a), 0);
        }
        return fmx(k.s1[0], delta1_taps(tu), k.s1[1] * delta1_taps(tv));
    }
};
template <class T>
using SmemAcc = SmemAccT<T, kSX, kSY, 2, 2, true>;

// One tile (x0, y0) and z-chunk starting at zbeg, by one block of kTX x kTY
// threads, with `sm` the block's ring of staged planes.
template <class T, bool RESID>
__device__ __forceinline__ void ra_tiled_block(T* sm, const Grid& g, const Coef<T>& k, const Phys& ph,
                                               const RKStage& rk, const T* __restrict__ Qf,
                                               const T* __restrict__ Wf, const state_t<T>* __restrict__ Q64,
                                               state_t<T>* __restrict__ out, state_t<T>* __restrict__ Qs,
                                               T* __restrict__ Wnext, int x0, int y0, int zbeg) {
    const int tid = threadIdx.x;
    const int tx = tid % kTX, ty = tid / kTX;
    const int nx = g.nx, ny = g.ny, nz = g.nz, n = g.n;
    const int zend = min(nz, zbeg + kZChunk);
    // in-plane offsets of the (at most two) staged cells of this thread
    int off[2];
    bool has[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int e = tid + r * kTX * kTY;
        has[r] = e < kPlane;
        const int hx = e % kSX, hy = e / kSX;
        const int gx = ((x0 + hx - 2) % nx + nx) % nx;
        const int gy = ((y0 + hy - 2) % ny + ny) % ny;
        off[r] = gy * nx + gx;
    }
    auto stage_plane = [&](int z, int slot) {
        const int zz = ((z % nz) + nz) % nz;
        const size_t base = (size_t)zz * nx * ny;
        T* dst = sm + slot * kNF * kPlane;
#pragma unroll
        for (int f = 0; f < kNF; ++f) {
            const T* src = f < 5 ? Qf + (size_t)f * n : Wf + (size_t)(f - 5) * n;
#pragma unroll
            for (int r = 0; r < 2; ++r)
                if (has[r]) dst[f * kPlane + tid + r * kTX * kTY] = ld(src + base, off[r]);
        }
    };
    for (int dz = -2; dz <= 1; ++dz) stage_plane(zbeg + dz, dz + 2);
    const int x = x0 + tx, y = y0 + ty;
    const bool inside = x < nx && y < ny;
    T aq[5];  // D_x u_x + D_y u_y of planes z-2 .. z+2 at (x, y)
    for (int z = zbeg; z < zend; ++z) {
        const int r0 = z - zbeg;  // ring slot of plane z + dz is (r0 + dz + 2) % 5
        const int c = (z * ny + y) * nx + x;
        state_t<T> qs[5];
        if (!RESID && inside) {
            const state_t<T>* src = rk.stage == 0 ? Q64 : Qs;
#pragma unroll
            for (int f = 0; f < 5; ++f) qs[f] = src[(size_t)f * n + c];
        }
        stage_plane(z + 2, (r0 + 4) % kRing);
        __syncthreads();
        if (inside) {
            SmemAcc<T> A{sm, {r0 % kRing, (r0 + 1) % kRing, (r0 + 2) % kRing, (r0 + 3) % kRing, (r0 + 4) % kRing},
                         tx, ty};
            if (z == zbeg) {
#pragma unroll
                for (int dz = -2; dz <= 1; ++dz) aq[dz + 2] = A.gxx_gyy(dz, k);
            }
            aq[4] = A.gxx_gyy(2, k);
            A.zq = aq;
            T R[5];
            fused_residual<T, false>(A, k, R);
#pragma unroll
            for (int q = 0; q < 4; ++q) aq[q] = aq[q + 1];
            if (RESID) {
#pragma unroll
                for (int f = 0; f < 5; ++f) out[(size_t)f * n + c] = to_state(R[f]);
            } else {
                stage_update(rk, ph, n, c, qs, R, out, Qs, Wnext);
            }
        }
        __syncthreads();
    }
}

template <class T, bool RESID>
__global__ void __launch_bounds__(kTX* kTY, sizeof(T) == 4 ? 2 : 1)
    k_ra_tiled(Grid g, Coef<T> k, Phys ph, RKStage rk, const T* __restrict__ Qf, const T* __restrict__ Wf,
               const state_t<T>* __restrict__ Q64, state_t<T>* __restrict__ out, state_t<T>* __restrict__ Qs,
               T* __restrict__ Wnext) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ra_tiled_block<T, RESID>(reinterpret_cast<T*>(smem_raw), g, k, ph, rk, Qf, Wf, Q64, out, Qs, Wnext,
                             blockIdx.x * kTX, blockIdx.y * kTY, blockIdx.z * kZChunk);
}

// Recompute-all, binary32, with the planes staged by the Tensor Memory
// Accelerator.  The ten working fields are one ghost-padded array (PadLayout)
// [10][nz][ny+4][nx+4]; one four-dimensional TMA copy moves a 36 x 12 box of
// all ten fields of one plane (the 32 x 8 tile and its two-point halos) into a
// ring of six plane slots, each with its own mbarrier.  While plane z is
// evaluated, plane z+3 is already in flight, so no thread issues a staging
// load and the copy latency is hidden behind the stencil arithmetic.  The
// padding holds the periodic images, so boxes at the domain edge need nothing
// special.  Every wait is bounded (0.5 s of wall time): a wait that runs out
// sets *err, drains the copies in flight (again bounded) and ends the block.
constexpr int kMX = 32, kMY = 8, kMThreads = kMX * kMY;
constexpr int kBX = kMX + 4, kBY = kMY + 4, kBPlane = kBX * kBY;
constexpr int kMSlots = 6, kMZChunk = 64;
constexpr int kMLook = kMSlots - 5;  // planes in flight beyond the five a plane's stencils read
constexpr int kMBlocks = kMY == 8 ? 2 : 1;  // resident blocks per SM the ring allows
constexpr unsigned kMSlotBytes = kNF * kBPlane * 4;  // 17280, a multiple of 128
// All of a block's shared memory is dynamic: the ring (6 x 17280 bytes, first,
// so that it starts on the 128-byte boundary the TMA destination needs), the
// six mbarriers, and in the batched kernel the instance record: two blocks per
// SM, 2 x (103680 + 48 + record + 1024 reserved) <= 228 KB.
constexpr unsigned long long kMWaitNs = 500000000ull;  // a wait gives up after 0.5 s
using TmaAcc = SmemAccT<float, kBX, kBY, 2, 2, true>;
// Dynamic shared memory of a TMA block: ring, then mbarriers (then, batched,
// the instance record on a 16-byte boundary).
constexpr unsigned kMBarOff = kMSlots * kMSlotBytes;
constexpr unsigned kMSmem = (kMBarOff + 8 * kMSlots + 15) / 16 * 16;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the completion of the phase of parity `parity` of an mbarrier,
// polling for at most kMWaitNs of wall time.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
    const unsigned long long t0 = global_ns();
    for (;;) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (global_ns() - t0 > kMWaitNs) return false;
    }
}

__device__ __forceinline__ void mbar_init_ring(unsigned bar0) {
    for (int s = 0; s < kMSlots; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8 * s));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One (tile, z-chunk) work item of the TMA-staged kernel: tile origin (x0, y0),
// planes zbeg .. min(nz, zbeg + zlen) - 1.  `phase` holds the parity of the
// next completion of each ring slot (bit s) and carries over between the work
// items of a persistent block; every plane issued is waited for exactly once,
// so it stays the same in every thread.  Returns false when a wait ran out;
// the block has then drained its copies and must end.
template <bool RESID>
__device__ __forceinline__ bool ra_tma_item(float* sm, unsigned bar0, unsigned& phase, const CUtensorMap* map,
                                            const Grid& g, const Coef<float>& k, const Phys& ph, const RKStage& rk,
                                            const df64* __restrict__ Q64, df64* __restrict__ out,
                                            df64* __restrict__ Qs, float* __restrict__ Wnext,
                                            int* __restrict__ err, int x0, int y0, int zbeg, int zlen,
                                            int skip_plane = -1000000) {
    const int tid = threadIdx.x, tx = tid % kMX, ty = tid / kMX;
    const int nx = g.nx, ny = g.ny, nz = g.nz, n = g.n;
    const int zend = min(nz, zbeg + zlen);
    const int zlast = zend + 1;  // last plane the item reads
    const unsigned sm0 = smem_u32(sm);
    const PadLayout L = pad_layout(g);
    auto slot_of = [&](int p) { return (p - zbeg + 2) % kMSlots; };
    auto issue = [&](int p) {  // one thread; padded coordinates of (x0 - 2, y0 - 2) are (x0, y0)
        if (p == skip_plane) return;  // failure-detection test: this plane never arrives
        const int s = slot_of(p);
        const unsigned bar = bar0 + 8 * s, dst = sm0 + s * kMSlotBytes;
        const int zz = ((p % nz) + nz) % nz;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kMSlotBytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
            "%4, %5}], [%6];" ::"r"(dst),
            "l"(reinterpret_cast<unsigned long long>(map)), "r"(x0), "r"(y0), "r"(zz), "r"(0), "r"(bar)
            : "memory");
    };
    int consumed = zbeg - 3;  // planes up to here have been waited for (in order, with success)
    auto wait = [&](int p) {
        const int s = slot_of(p);
        if (!mbar_wait(bar0 + 8 * s, (phase >> s) & 1u)) return false;
        phase ^= 1u << s;
        consumed = p;
        return true;
    };
    // After a wait ran out: record it, wait (bounded) for every copy still in flight, end.
    auto fail = [&](int issued) {
        if (tid == 0) {
            atomicExch(err, 1);
            for (int p = consumed + 1; p <= issued; ++p) {
                const int s = slot_of(p);
                mbar_wait(bar0 + 8 * s, (phase >> s) & 1u);
                phase ^= 1u << s;
            }
        }
        __syncthreads();
        return false;
    };

    int issued = zbeg + 1 + kMLook;
    if (tid == 0)
        for (int p = zbeg - 2; p <= issued; ++p) issue(p);
    {
        bool ok = true;
        for (int p = zbeg - 2; p <= zbeg + 1 && ok; ++p) ok = wait(p);
        if (__syncthreads_or(!ok)) return fail(issued);
    }
    const int x = x0 + tx, y = y0 + ty;
    const bool inside = x < nx && y < ny;
    float aq[5];  // D_x u_x + D_y u_y of planes z-2 .. z+2 at (x, y)
    for (int z = zbeg; z < zend; ++z) {
        const int c = (z * ny + y) * nx + x;
        if (z + 2 + kMLook <= zlast) {
            if (tid == 0) issue(z + 2 + kMLook);
            issued = z + 2 + kMLook;
        }
        df64 qs[5];
        if (!RESID && inside) {
            const df64* src = rk.stage == 0 ? Q64 : Qs;
#pragma unroll
            for (int f = 0; f < 5; ++f) qs[f] = ld(src + (size_t)f * n, c);
        }
        if (__syncthreads_or(!wait(z + 2))) return fail(issued);
        if (inside) {
            TmaAcc A{sm, {slot_of(z - 2), slot_of(z - 1), slot_of(z), slot_of(z + 1), slot_of(z + 2)}, tx, ty};
            if (z == zbeg) {
#pragma unroll
                for (int dz = -2; dz <= 1; ++dz) aq[dz + 2] = A.gxx_gyy(dz, k);
            }
            aq[4] = A.gxx_gyy(2, k);
            A.zq = aq;
            float R[5];
            fused_residual<float, false>(A, k, R);
#pragma unroll
            for (int q = 0; q < 4; ++q) aq[q] = aq[q + 1];
            if (RESID) {
#pragma unroll
                for (int f = 0; f < 5; ++f) out[(size_t)f * n + c] = to_state(R[f]);
            } else {  // stage_update, with the next-stage fields into the padded layout
                df64 qn[5];
#pragma unroll
                for (int f = 0; f < 5; ++f) {
                    qn[f] = upd(rk_a(rk, df64()), R[f], qs[f]);
                    out[(size_t)f * n + c] = qn[f];
                    if (rk.stage < 2) Qs[(size_t)f * n + c] = upd(rk_b(rk, df64()), R[f], qs[f]);
                }
                float v[10];
                prims_values(ph, qn, v);
                put_padded(L, Wnext, x, y, z, v);
            }
        }
        __syncthreads();
    }
    return true;
}

// The ring must start on a 128-byte boundary (the TMA destination rule); the
// dynamic shared window is declared so aligned, and a block that finds it
// otherwise reports it (*err = 2) and issues no copy.
__device__ __forceinline__ bool tma_ring_aligned(const unsigned char* raw, int* err) {
    if ((smem_u32(raw) & 127) == 0) return true;
    if (threadIdx.x == 0) atomicExch(err, 2);
    return false;
}

template <bool RESID>
__global__ void __launch_bounds__(kMThreads, kMBlocks)
    k_ra_tma(const __grid_constant__ CUtensorMap map, Grid g, Coef<float> k, Phys ph, RKStage rk,
             const df64* __restrict__ Q64, df64* __restrict__ out, df64* __restrict__ Qs,
             float* __restrict__ Wnext, int* __restrict__ err, int zlen, int skip_plane) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    if (!tma_ring_aligned(smem_raw, err)) return;
    const unsigned bar0 = smem_u32(smem_raw + kMBarOff);
    if (threadIdx.x == 0) mbar_init_ring(bar0);
    __syncthreads();
    unsigned phase = 0;
    ra_tma_item<RESID>(reinterpret_cast<float*>(smem_raw), bar0, phase, &map, g, k, ph, rk, Q64, out, Qs, Wnext,
                       err, blockIdx.x * kMX, blockIdx.y * kMY, blockIdx.z * zlen, zlen, skip_plane);
}

// Batched form: a persistent grid walks the (tile, z-chunk) items of the
// binary32 recompute-all instances, numbered as tma_work_items counts them;
// each instance record carries the tensor maps of its two working-field
// buffers, which the copies read from global memory.  Only what an item needs
// of the record is staged in shared memory (two blocks per SM leave 512 bytes
// beside the two rings, for the barriers and this record).
struct TmaItem {
    Grid g;
    Coef<float> k;
    Phys ph;
    RKStage rk;
    const df64* Q64;
    df64* out;
    df64* Qs;
    float* Wnext;
};
// Two blocks per SM need 2 x (ring + barriers + item) + 2 x 1 KB reserved of the
// SM's 228 KB.
static_assert(kMBlocks == 1 || 2 * (kMSmem + sizeof(TmaItem) + 1024) <= 228 * 1024,
              "TmaItem too large for two batched TMA blocks per SM");
static_assert(kMSmem % 16 == 0, "the instance record follows the mbarriers on a 16-byte boundary");

template <bool RESID>
__global__ void __launch_bounds__(kMThreads, kMBlocks)
    k_batch_ra_tma(const BatchInst<float>* __restrict__ insts, const BatchTile* __restrict__ tiles, int ntiles,
                   int stage, int parity, int* __restrict__ err, int zlen) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TmaItem& it = *reinterpret_cast<TmaItem*>(smem_raw + kMSmem);
    if (!tma_ring_aligned(smem_raw, err)) return;
    const unsigned bar0 = smem_u32(smem_raw + kMBarOff);
    if (threadIdx.x == 0) mbar_init_ring(bar0);
    unsigned phase = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const BatchTile tl = tiles[t];
        __syncthreads();
        if (threadIdx.x == 0) {
            const BatchInst<float>& I = insts[tl.inst];
            it.g = I.g;
            it.k = I.k;
            it.ph = I.ph;
            it.rk = I.rk[stage];
            it.Q64 = I.Q[parity];
            it.out = I.Q[1 - parity];
            it.Qs = I.Qs;
            it.Wnext = I.W[1 - parity];
        }
        __syncthreads();
        const int ntx = (it.g.nx + kMX - 1) / kMX, nty = (it.g.ny + kMY - 1) / kMY;
        const int zc = tl.start / (ntx * nty), r = tl.start % (ntx * nty);
        if (!ra_tma_item<RESID>(reinterpret_cast<float*>(smem_raw), bar0, phase, &insts[tl.inst].fmap[parity],
                                it.g, it.k, it.ph, it.rk, it.Q64, it.out, it.Qs, it.Wnext, err,
                                (r % ntx) * kMX, (r / ntx) * kMY, zc * zlen, zlen))
            return;
    }
}

// ------------------------------------------------------------------ SS
// Store-some (Section 2, paragraph SS): the nine velocity gradients
// du_i/dx_j go to global work arrays; every other derivative is evaluated
// into thread-local registers in the fused kernel.  The mixed derivatives
// D_i(D_k u_k) difference the stored gradients.  In binary64, where FP64
// instructions are the limit, the gradient pass also stores the three pair
// sums P_i = G_jj + G_kk (j, k the axes other than i), the sum the fused
// kernel otherwise forms at each of the four taps (same operands, same order,
// same result; 9 fewer FP64 instructions per point).  The binary32 and df64
// kernels are bound by memory and latency, where the three extra arrays cost
// more than they save, so they keep forming the sums.
template <class T>
__device__ __forceinline__ void store_pair_sums(const T G[3][3], T* __restrict__ P, int n, int c) {
    if constexpr (kStoresPairSums<T>) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int j1 = i == 0 ? 1 : 0, j2 = i == 2 ? 1 : 2;
            P[i * n + c] = G[j1][j1] + G[j2][j2];
        }
    }
}
template <class T>
__global__ void __launch_bounds__(256) k_ss_grad(Grid g, Coef<T> k, const T* __restrict__ Wf, T* __restrict__ Gw) {
    int idx = grid_index();
    if (idx >= g.n) return;
    const int n = g.n;
    const Nbr s = make_nbr(g, idx);
    T G[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            T t[4];
            taps(Wf + i * n, s.c, s.o[j], t);
            G[i][j] = k.s1[j] * delta1_taps(t);
            Gw[(3 * i + j) * n + s.c] = G[i][j];
        }
    store_pair_sums(G, Gw + 9 * (size_t)n, n, s.c);
}

template <class T, bool RESID>
__device__ __forceinline__ void ss_point(const Grid& g, const Coef<T>& k, const Phys& ph, const RKStage& rk,
                                         const T* __restrict__ Qf, const T* __restrict__ Wf,
                                         const T* __restrict__ Gw, const state_t<T>* __restrict__ Q64,
                                         state_t<T>* __restrict__ out, state_t<T>* __restrict__ Qs,
                                         T* __restrict__ Wnext) {
    int idx = grid_index();
    if (idx >= g.n) return;
    const Nbr s = make_nbr(g, idx);
    T R[5];
    fused_residual<T, true>(GlobalAcc<T>{s, g.n, Qf, Wf, Gw}, k, R);
    stage_write<T, RESID>(rk, ph, g.n, s.c, Q64, R, out, Qs, Wnext);
}

// binary64 and df64: registers capped for four blocks (16 warps) per SM; the
// binary32 form keeps the compiler's own register choice (fewer, no cap).
template <class T, bool RESID>
__global__ void __launch_bounds__(128, 4) k_ss(Grid g, Coef<T> k, Phys ph, RKStage rk, const T* __restrict__ Qf,
                                            const T* __restrict__ Wf, const T* __restrict__ Gw,
                                            const state_t<T>* __restrict__ Q64, state_t<T>* __restrict__ out,
                                            state_t<T>* __restrict__ Qs, T* __restrict__ Wnext) {
    ss_point<T, RESID>(g, k, ph, rk, Qf, Wf, Gw, Q64, out, Qs, Wnext);
}

template <bool RESID>
__global__ void __launch_bounds__(128) k_ss_f32(Grid g, Coef<float> k, Phys ph, RKStage rk,
                                                const float* __restrict__ Qf, const float* __restrict__ Wf,
                                                const float* __restrict__ Gw, const df64* __restrict__ Q64,
                                                df64* __restrict__ out, df64* __restrict__ Qs,
                                                float* __restrict__ Wnext) {
    ss_point<float, RESID>(g, k, ph, rk, Qf, Wf, Gw, Q64, out, Qs, Wnext);
}

// ------------------------------------- SS, binary64 with double-word stencils
// Store-some in mixed arithmetic (FD_F64_DW).  On GB300 a binary64 instruction
// occupies its pipe as long as 64 binary32 ones do, and the binary64 fused
// kernel is bound by that pipe.  This form keeps in binary64 what decides the
// binary64 result, and evaluates the rest in double-word arithmetic:
//   binary64:
//   - the state Q, the saved register Qs and the RK update (Fig. 1), two FMAs
//     per variable and register, so the state rounds as in the binary64 path;
//   - the primitives u_i and p of Eq. 6, formed as in the binary64 path and
//     stored.  The mean of p, 1/(gamma M^2), is ~70 times its variation at
//     M = 0.1, and its binary64 rounding (one unit is 1.4e-14) is what the
//     smallest variable, rho w, resolves through -D_z p; the pressure
//     gradient differences p - p0, exact in binary64 and held exactly by the
//     double-word working field at M = 0.1 (ss_hyb_point), so the differences
//     of the binary64 pressures are exact;
//   - div u = sum_i D_i u_i from the binary64 velocities (formed with the
//     gradients by the first fused kernel), for the two terms that carry a mean: -div
//     in the mass residual and -(rhoE0 + p0) div in the energy residual (the
//     mean energy and the mean pressure work; ~250 div at M = 0.1, which would
//     magnify a double-word div 250-fold);
//   double-word, on shifted fields (rho-1, rho u_i, rho E - rhoE0, u_i,
//   p - p0, T - 1) on the binary32 pipe, as in the df64 mode: convection,
//   pressure work, the viscous stress divergence and its work, the
//   dissipation, the heat flux and the nine velocity gradients.  Each is a
//   stencil sum of operands no larger than the residual's own scale times the
//   stencil weights, so its rounding (~2^-48 of the operands) stays near 1e-14
//   of the residual.
// Values move between the formats by integer operations on the IEEE fields
// (dw_of_f64, f64_of_dw): a conversion instruction would cost a DFMA.
//
// Binary64 instructions per point and stage in the fused pass: 2 FMAs adding
// the div terms, 5 sums hi + lo of the residual, 10 RK FMAs (5 in stage 2), and
// ~17 for the next stage's primitives (1 / rho, u_i, p, and rho - 1,
// rho E - rhoE0, p - p0); 12 in the gradient pass (div u).  (div u moved from
// the fused kernel to the gradient pass: fused 3.67 -> 3.23 ms, gradients
// 0.35 -> 0.61 ms per 256^3 stage.)

// Working fields of a binary64 state: the ten shifted double-word fields F and
// the binary64 velocities W64 = (u, v, w).  u_i and p are the binary64 path's
// own formulas; rho - 1, rho E - rhoE0 and p - p0 are exact in
// binary64 (operands within a factor 2) and then split, and
// T - 1 = (gamma M^2 (p - p0) - (rho - 1)) / rho is double-word arithmetic
// (gamma M^2 p0 = 1).
__device__ __forceinline__ void hyb_prims_point(const Phys& ph, const double q[5], df64* __restrict__ F,
                                                double* __restrict__ W64, int n, int c) {
    const double inv = 1.0 / q[0];
    const double u = q[1] * inv, v = q[2] * inv, w = q[3] * inv;
    const double p = ph.gm1 * fmx(-0.5, fmx(q[1], u, fmx(q[2], v, q[3] * w)), q[4]);
    const df64 rp = dw_of_f64(q[0] - 1.0);
    const df64 pp = dw_of_f64(p - ph.p0);
    F[c] = rp;
    F[n + c] = dw_of_f64(q[1]);
    F[2 * n + c] = dw_of_f64(q[2]);
    F[3 * n + c] = dw_of_f64(q[3]);
    F[4 * n + c] = dw_of_f64(q[4] - ph.rhoE0);
    F[5 * n + c] = dw_of_f64(u);
    F[6 * n + c] = dw_of_f64(v);
    F[7 * n + c] = dw_of_f64(w);
    F[8 * n + c] = pp;
    F[9 * n + c] = fmx(ph.gM2_w, pp, -rp) * dw_of_f64(inv);
    W64[c] = u;
    W64[n + c] = v;
    W64[2 * n + c] = w;
}

__global__ void __launch_bounds__(256) k_prims_hyb(Grid g, Phys ph, const double* __restrict__ Q,
                                                   df64* __restrict__ F, double* __restrict__ W64) {
    const int idx = grid_index();
    if (idx >= g.n) return;
    const int n = g.n;
    double q[5];
#pragma unroll
    for (int f = 0; f < 5; ++f) q[f] = Q[f * n + idx];
    hyb_prims_point(ph, q, F, W64, n, idx);
}

// One double-word velocity gradient G_ij = D_j u_i at a point, from the taps
// of u_i along j (both fused kernels form it this way, so the bits agree).
__device__ __forceinline__ df64 hyb_grad(const Coef<df64>& k, int j, const df64 t[4]) {
    return mul_nn(k.s1[j], delta1_taps(t));  // unnormalised, as the stencil sums
}
// Gradients of the mixed kernels at one point: the three double-word
// gradients G_ii (stored as Gw[i], returned in G) and div u = sum_i D_i u_i in
// binary64 from the binary64 velocities W64 (as the binary64 gradient pass
// forms D_i u_i), which the second fused kernel reads for the two mean-state
// terms.  The second kernel differences G_jj + G_kk at its neighbours for the
// mixed derivatives; the six G_ij, i != j, it needs only at the point itself
// (the dissipation), and forms them there from the u_i taps its viscous terms
// load anyway (hyb_grad, the same bits).
__device__ __forceinline__ void ss_grad_hyb_point(const Grid& g, const Coef<df64>& k, const df64* __restrict__ Wf,
                                                  const double* __restrict__ W64, df64* __restrict__ Gw,
                                                  double* __restrict__ Dv, int idx, df64 G[3][3]) {
    const int n = g.n;
    const Nbr s = make_nbr(g, idx);
    // div u = sum_j s_j delta_j u_j with the scales folded into the sum (12 FP64
    // instructions: 6 DADD + 3 DFMA for the differences, DMUL + 2 DFMA for the sum)
    double d[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        double t[4];
        taps(W64 + j * (size_t)n, s.c, s.o[j], t);
        d[j] = delta1_taps(t);
    }
    Dv[s.c] = fmx(g.inv12h[0], d[0], fmx(g.inv12h[1], d[1], g.inv12h[2] * d[2]));
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int j = 0; j < 3; ++j) G[i][j] = df64(0.0f, 0.0f);  // (only G_ii is formed here)
        df64 t[4];
        taps(Wf + i * n, s.c, s.o[i], t);
        G[i][i] = hyb_grad(k, i, t);
        Gw[(size_t)i * n + s.c] = G[i][i];
    }
}

// Fused residual + RK update + next-stage working fields.  F / W64: the
// working fields of the stage's state, Gw: its nine velocity gradients
// (double-word, from k_ss_grad<df64>), Q64 the binary64 state the stage starts
// from (read as Qs in stage 0), out the next state (or R when RESID), Fnext /
// W64next the next stage's working fields.  k is the df64 mode's coefficient
// record with its two mean-state terms (c_rho, c_E) set to zero: those enter
// here in binary64, with c_E = -(rhoE0 + p0).
// The convective part of the residual (PART 1), into Rc for ss_hyb_point.  The
// residual is split over two kernels so that each runs at a higher occupancy
// than the whole residual could (128 registers and 84 bytes of spill at 16 warps
// per SM): this one at five blocks of 128 threads per SM (96 registers), the
// second at six (80 registers and 88 bytes of spill, 1 % faster than five
// without; the batched form runs at four: 26.5 solves/s on the 64-solve
// ensemble against 26.0 at five and 24.8 at six), for 40 bytes per point written
// and read again.  The kernels are latency-bound on their tap loads, so the
// warps pay: 256^3 step 11.53 ms (one kernel) -> 11.01 (two, four blocks
// each) -> 9.63-9.89 (five and six blocks).  The pressure work later moved to
// the second kernel, which loads its taps anyway (9.10 -> 9.00 ms), and so
// did the six off-diagonal gradients (8.74 -> 8.54 ms); forming the
// dissipation there before the stencil sums was slower (9.63 ms).
// The gradient pass rides in this kernel: the point's G_ii and binary64 div u
// (ss_grad_hyb_point) are stored for the second kernel, whose stencils read the
// G_ii at neighbouring points, and the convective part takes G_ii from
// registers.  Its binary64 div u fills the FP64 pipe, idle in the double-word
// convective sums.
template <class Acc>
struct RegGradAcc : Acc {
    const df64 (*Gr)[3];
    __device__ __forceinline__ df64 grad(int i, int j) const { return Gr[i][j]; }
};
// The second kernel's view of the gradients: G_ii from the three stored
// arrays, G_ij (i != j) formed from the u_i taps along j (hyb_grad).
struct HybRestAcc : GlobalAcc<df64> {
    const Coef<df64>& k;
    __device__ __forceinline__ df64 grad(int i, int j) const {
        if (i == j) return ld(Gw + (size_t)i * n, s.c);
        df64 t[4];
        taps(5 + i, j, t);
        return hyb_grad(k, j, t);
    }
    __device__ __forceinline__ void grad_pair_taps(int ga, int gb, int i, df64 t[4]) const {
        const df64* pa = Gw + (size_t)ga * n;
        const df64* pb = Gw + (size_t)gb * n;
#pragma unroll
        for (int a = 0; a < 4; ++a) t[a] = ld(pa, s.c + s.o[i][a]) + ld(pb, s.c + s.o[i][a]);
    }
};
__device__ __forceinline__ void ss_hyb_conv_point(const Grid& g, const Coef<df64>& k, const df64* __restrict__ F,
                                                  const double* __restrict__ W64, df64* __restrict__ Gw,
                                                  double* __restrict__ Dv, df64* __restrict__ Rc, int idx) {
    const int n = g.n;
    df64 G[3][3];
    ss_grad_hyb_point(g, k, F + 5 * (size_t)n, W64, Gw, Dv, idx, G);
    const Nbr s = make_nbr(g, idx);
    df64 R[5];
    using A = RegGradAcc<GlobalAcc<df64>>;
    fused_residual<df64, true, A, false, 1>(A{{s, n, F, F + 5 * (size_t)n, Gw}, G}, k, R);
#pragma unroll
    for (int f = 0; f < 5; ++f) Rc[(size_t)f * n + idx] = R[f];
}
__global__ void __launch_bounds__(128, 5) k_ss_hyb_conv(Grid g, Coef<df64> k, const df64* __restrict__ F,
                                                       const double* __restrict__ W64, df64* __restrict__ Gw,
                                                       double* __restrict__ Dv, df64* __restrict__ Rc) {
    const int idx = grid_index();
    if (idx >= g.n) return;
    ss_hyb_conv_point(g, k, F, W64, Gw, Dv, Rc, idx);
}

template <bool RESID>
__device__ __forceinline__ void ss_hyb_point(const Grid& g, const Coef<df64>& k, const Phys& ph, const RKStage& rk,
                                             double c_E, const df64* __restrict__ F, const df64* __restrict__ Gw,
                                             const df64* __restrict__ Rc, const double* __restrict__ Dv,
                                             const double* __restrict__ Q64, double* __restrict__ out,
                                             double* __restrict__ Qs, df64* __restrict__ Fnext,
                                             double* __restrict__ W64next, int idx) {
    const int n = g.n;
    df64 Rw[5];
    {
        const Nbr s = make_nbr(g, idx);
        fused_residual<df64, true, HybRestAcc, false, 2>(HybRestAcc{{s, n, F, F + 5 * (size_t)n, Gw}, k}, k, Rw);
    }
#pragma unroll
    for (int f = 0; f < 5; ++f) Rw[f] = renorm(add_nn(Rw[f], ld(Rc + (size_t)f * n, idx)));
    // the neighbour offsets again (cheaper than keeping them live through the residual)
    const Nbr s = make_nbr(g, idx);
    // -D_j p: 8 (p_{+1} - p_{-1}) + (p_{-2} - p_{+2}) from the double-word p - p0
    // of the working fields (hyb_prims_point: the binary64 pressure minus p0,
    // exact in binary64).  At Mach 0.1 (p0 = 71.4, whose binade holds every
    // pressure of the flow) p - p0 is a multiple of 2^-46 below 0.5: at most 45
    // significant bits, so the pair holds it exactly, and each difference of two
    // taps is exact too (TwoSum of the leading words; the trailing words and the
    // TwoSum error, multiples of 2^-46 below 2^-24, add exactly).  At higher Mach
    // p0 is smaller and the pair may round p - p0, to 2^-48 |p - p0|: less than
    // one unit in the last place of p0 while |p - p0| < p0 / 16.
    const df64* Pw = F + 8 * (size_t)n;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        df64 t[4];
        taps(Pw, s.c, s.o[j], t);
        const df64 d = scale2(sub_nn(t[2], t[1]), 8.0f) + sub_nn(t[0], t[3]);
        Rw[1 + j] = fmx(k.cp[j], d, Rw[1 + j]);
    }
    const double div = ld(Dv, s.c);  // binary64 div u of the gradient pass
    double R[5];
    R[0] = fmx(-1.0, div, f64_of_f32(Rw[0].hi)) + f64_of_f32(Rw[0].lo);
#pragma unroll
    for (int f = 1; f < 4; ++f) R[f] = f64_of_dw(Rw[f]);
    R[4] = fmx(c_E, div, f64_of_f32(Rw[4].hi)) + f64_of_f32(Rw[4].lo);
    if constexpr (RESID) {
#pragma unroll
        for (int f = 0; f < 5; ++f) out[f * n + s.c] = R[f];
    } else {
        double qn[5];
#pragma unroll
        for (int f = 0; f < 5; ++f) {
            const double qs = rk.stage == 0 ? Q64[f * n + s.c] : Qs[f * n + s.c];
            qn[f] = fmx(rk.adt, R[f], qs);
            out[f * n + s.c] = qn[f];
            if (rk.stage < 2) Qs[f * n + s.c] = fmx(rk.bdt, R[f], qs);
        }
        hyb_prims_point(ph, qn, Fnext, W64next, n, s.c);
    }
}
template <bool RESID>
__global__ void __launch_bounds__(128, 6) k_ss_hyb(Grid g, Coef<df64> k, Phys ph, RKStage rk, double c_E,
                                                   const df64* __restrict__ F, const df64* __restrict__ Gw,
                                                   const df64* __restrict__ Rc, const double* __restrict__ Dv,
                                                   const double* __restrict__ Q64,
                                                   double* __restrict__ out, double* __restrict__ Qs,
                                                   df64* __restrict__ Fnext, double* __restrict__ W64next) {
    const int idx = grid_index();
    if (idx >= g.n) return;
    ss_hyb_point<RESID>(g, k, ph, rk, c_E, F, Gw, Rc, Dv, Q64, out, Qs, Fnext, W64next, idx);
}

// ------------------------------------------------------------------ BL
// Store-all (Section 2, paragraph BL): every product inside a derivative is
// first written to a product work array, every derivative to its own
// derivative work array; the residual is then a pointwise loop.
// Work-array indices (each a grid-sized array):
//   P : Qf_f u_j at 3f+j (f = 0..4, j = 0..2), p u_j at 15+j
//   D1: D_j Qf_f at 3f+j, D_j u_i at 15+3i+j, D_i p at 24+i,
//       D_j(Qf_f u_j) at 27+3f+j, D_j(p u_j) at 42+j
//   D2: D2_j u_i at 3i+j, D2_j T at 9+j, D_i(D_k u_k) (k != i) at 12+2i+(k>i ? k-1 : k)
template <class T>
__global__ void __launch_bounds__(256) k_bl_prod(Grid g, const T* __restrict__ Qf, const T* __restrict__ Wf,
                                                 T* __restrict__ P) {
    int idx = grid_index();
    if (idx >= g.n) return;
    const long long n = g.n;  // work arrays index up to 45 n
    T u[3] = {Wf[idx], Wf[n + idx], Wf[2 * n + idx]};
    T p = Wf[3 * n + idx];
#pragma unroll
    for (int f = 0; f < 5; ++f) {
        T qf = Qf[f * n + idx];
#pragma unroll
        for (int j = 0; j < 3; ++j) P[(3 * f + j) * n + idx] = qf * u[j];
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) P[(15 + j) * n + idx] = p * u[j];
}

template <class T>
__global__ void __launch_bounds__(256) k_bl_d1(Grid g, const T* __restrict__ Qf, const T* __restrict__ Wf,
                                               const T* __restrict__ P, T* __restrict__ D1) {
    int idx = grid_index();
    if (idx >= g.n) return;
    const long long n = g.n;  // work arrays index up to 45 n
    const Nbr s = make_nbr(g, idx);
    const int c = s.c;
#pragma unroll
    for (int f = 0; f < 5; ++f)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            D1[(3 * f + j) * n + c] = s1<T>(g, j) * delta1<T>([&](int k) { return ld(Qf + f * n, k); }, c, s.o[j]);
            D1[(27 + 3 * f + j) * n + c] =
                s1<T>(g, j) * delta1<T>([&](int k) { return ld(P + (3 * f + j) * n, k); }, c, s.o[j]);
        }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            D1[(15 + 3 * i + j) * n + c] = s1<T>(g, j) * delta1<T>([&](int k) { return ld(Wf + i * n, k); }, c, s.o[j]);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        D1[(24 + j) * n + c] = s1<T>(g, j) * delta1<T>([&](int k) { return ld(Wf + 3 * n, k); }, c, s.o[j]);
        D1[(42 + j) * n + c] = s1<T>(g, j) * delta1<T>([&](int k) { return ld(P + (15 + j) * n, k); }, c, s.o[j]);
    }
}

template <class T>
__global__ void __launch_bounds__(256) k_bl_d2(Grid g, const T* __restrict__ Wf, const T* __restrict__ D1,
                                               T* __restrict__ D2) {
    int idx = grid_index();
    if (idx >= g.n) return;
    const long long n = g.n;  // work arrays index up to 45 n
    const Nbr s = make_nbr(g, idx);
    const int c = s.c;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        T u0 = ld(Wf + i * n, c);
#pragma unroll
        for (int j = 0; j < 3; ++j)
            D2[(3 * i + j) * n + c] = s2<T>(g, j) * delta2<T>([&](int k) { return ld(Wf + i * n, k); }, c, s.o[j], u0);
    }
    T T0 = ld(Wf + 4 * n, c);
#pragma unroll
    for (int j = 0; j < 3; ++j)
        D2[(9 + j) * n + c] = s2<T>(g, j) * delta2<T>([&](int k) { return ld(Wf + 4 * n, k); }, c, s.o[j], T0);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (k == i) continue;
            const T* __restrict__ gkk = D1 + (15 + 3 * k + k) * n;
            D2[(12 + 2 * i + (k > i ? k - 1 : k)) * n + c] =
                s1<T>(g, i) * delta1<T>([&](int r) { return ld(gkk, r); }, c, s.o[i]);
        }
}

template <class T, bool RESID>
__global__ void __launch_bounds__(256) k_bl_res(Grid g, Phys ph, RKStage rk, const T* __restrict__ Qf,
                                                const T* __restrict__ Wf, const T* __restrict__ D1,
                                                const T* __restrict__ D2, const state_t<T>* __restrict__ Q64,
                                                state_t<T>* __restrict__ out, state_t<T>* __restrict__ Qs,
                                                T* __restrict__ Wnext) {
    int idx = grid_index();
    if (idx >= g.n) return;
    const long long n = g.n;  // work arrays index up to 45 n
    const int c = idx;
    Terms<T> t;
    T uc[3], q[5];
#pragma unroll
    for (int i = 0; i < 3; ++i) uc[i] = Wf[i * n + c];
#pragma unroll
    for (int f = 0; f < 5; ++f) q[f] = Qf[f * n + c];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) t.G[i][j] = D1[(15 + 3 * i + j) * n + c];
#pragma unroll
    for (int f = 0; f < 5; ++f) {
        T acc = 0;
#pragma unroll
        for (int j = 0; j < 3; ++j) acc += fmx(uc[j], D1[(3 * f + j) * n + c], D1[(27 + 3 * f + j) * n + c]);
        t.conv[f] = acc;
    }
    T dpu = 0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        t.dp[j] = D1[(24 + j) * n + c];
        dpu += D1[(42 + j) * n + c];
    }
    t.dpu = dpu;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        t.lap[i] = D2[(3 * i) * n + c] + D2[(3 * i + 1) * n + c] + D2[(3 * i + 2) * n + c];
        T gd = D2[(3 * i + i) * n + c];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (k == i) continue;
            gd += D2[(12 + 2 * i + (k > i ? k - 1 : k)) * n + c];
        }
        t.gd[i] = gd;
    }
    t.lapT = D2[9 * n + c] + D2[10 * n + c] + D2[11 * n + c];
    const Shift<T> sh = shift_of<T>(ph);
    T nu, ka;
    visc_consts(ph, nu, ka);
    T R[5];
    assemble<T>(t, q, uc, nu, ka, sh.c_rho, sh.c_E, R);
    stage_write<T, RESID>(rk, ph, n, c, Q64, R, out, Qs, Wnext);
}

// ------------------------------------------------------- SN and RS families
// The two remaining families of Section 2 evaluate the paper's derivative set
// as written: every derivative of a product is the difference of the product
// formed at the taps, D_j(Q_f u_j) and u_j D_j Q_f are separate derivatives,
// the mixed derivatives are D_i of D_k u_k, and the residual is assembled by
// the same pointwise code as BL (fd::assemble).  Each derivative is the same
// arithmetic as BL's work-array entry, so BL, SN and RS differ only in where a
// derivative lives and how often it is evaluated.  (RA and SS instead merge
// the derivatives that the residual adds along one direction into one
// stencil; see fused_residual.)
//
// One derivative from the taps of field f along axis j, scaled as BL scales it.
template <class T, class Acc>
__device__ __forceinline__ T d1_of(const Acc& A, const Grid& g, int f, int j) {
    T t[4];
    A.taps(f, j, t);
    return s1<T>(g, j) * delta1_taps(t);
}

// D_j of the product of fields f and w formed at the taps along j.
template <class T, class Acc>
__device__ __forceinline__ T d1_prod_of(const Acc& A, const Grid& g, int f, int w, int j) {
    T a[4], b[4], pr[4];
    A.taps(f, j, a);
    A.taps(w, j, b);
#pragma unroll
    for (int q = 0; q < 4; ++q) pr[q] = a[q] * b[q];
    return s1<T>(g, j) * delta1_taps(pr);
}

template <class T, class Acc>
__device__ __forceinline__ T d2_of(const Acc& A, const Grid& g, int f, int j, T f0) {
    T t[4];
    A.taps(f, j, t);
    return s2<T>(g, j) * delta2_taps(t, f0);
}

// conv_f = sum_j [ D_j(Q_f u_j) + u_j D_j Q_f ], in BL's order of operations.
template <class T, class Acc>
__device__ __forceinline__ T conv_of(const Acc& A, const Grid& g, int f, const T uc[3]) {
    constexpr int U = 5;
    T acc = 0;
#pragma unroll
    for (int j = 0; j < 3; ++j) acc += fmx(uc[j], d1_of<T>(A, g, f, j), d1_prod_of<T>(A, g, f, U + j, j));
    return acc;
}

// sum_j D2_j u_i and D2_i u_i + sum_{k != i} D_i(D_k u_k); the inner D_k u_k
// comes from u_k taps at the shifted points (SN) or the stored gradient G_kk
// (RS), both the arithmetic of BL's two passes.
template <class T, bool STORED_G, class Acc>
__device__ __forceinline__ void viscous_of(const Acc& A, const Grid& g, int i, T uci, T& lap, T& gd) {
    constexpr int U = 5;
    T d2[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) d2[j] = d2_of<T>(A, g, U + i, j, uci);
    lap = d2[0] + d2[1] + d2[2];
    gd = d2[i];
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) {
        if (kk == i) continue;
        T t[4];
        if constexpr (STORED_G) {
            A.grad_taps(kk, kk, i, t);
        } else {
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                T u4[4];
                A.taps_shifted(U + kk, kk, i, a, u4);
                t[a] = s1<T>(g, kk) * delta1_taps(u4);
            }
        }
        gd += s1<T>(g, i) * delta1_taps(t);
    }
}

// Store-none (Section 2, paragraph SN, and its pseudo-code figure): no work
// arrays; every derivative is evaluated once into a thread-local variable
// (the Terms record) and the residual of each equation is assembled from
// those locals, so a derivative that several equations use (div u, G_ij, the
// viscous terms) is evaluated once.
template <class T, bool RESID>
__global__ void __launch_bounds__(128) k_sn(Grid g, Phys ph, RKStage rk, const T* __restrict__ Qf,
                                            const T* __restrict__ Wf, const state_t<T>* __restrict__ Q64,
                                            state_t<T>* __restrict__ out, state_t<T>* __restrict__ Qs,
                                            T* __restrict__ Wnext) {
    constexpr int U = 5, P = 8, TT = 9;
    int idx = grid_index();
    if (idx >= g.n) return;
    const Nbr s = make_nbr(g, idx);
    const GlobalAcc<T> A{s, g.n, Qf, Wf, nullptr};
    Terms<T> t;
    T uc[3], q[5];
#pragma unroll
    for (int i = 0; i < 3; ++i) uc[i] = A.center(U + i);
#pragma unroll
    for (int f = 0; f < 5; ++f) q[f] = A.center(f);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) t.G[i][j] = d1_of<T>(A, g, U + i, j);
#pragma unroll
    for (int f = 0; f < 5; ++f) t.conv[f] = conv_of<T>(A, g, f, uc);
    T dpu = 0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        t.dp[j] = d1_of<T>(A, g, P, j);
        dpu += d1_prod_of<T>(A, g, P, U + j, j);
    }
    t.dpu = dpu;
#pragma unroll
    for (int i = 0; i < 3; ++i) viscous_of<T, false>(A, g, i, uc[i], t.lap[i], t.gd[i]);
    {
        const T T0 = A.center(TT);
        T d2[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) d2[j] = d2_of<T>(A, g, TT, j, T0);
        t.lapT = d2[0] + d2[1] + d2[2];
    }
    const Shift<T> sh = shift_of<T>(ph);
    T nu, ka;
    visc_consts(ph, nu, ka);
    T R[5];
    assemble<T>(t, q, uc, nu, ka, sh.c_rho, sh.c_E, R);
    stage_write<T, RESID>(rk, ph, g.n, s.c, Q64, R, out, Qs, Wnext);
}

// Recompute-some (Section 2, paragraph RS): the nine velocity gradients come
// from the work arrays of the gradient pass (k_ss_grad); every other
// derivative is written out as its formula inside the equation that uses it.
// Equation E evaluates exactly the terms fd::assemble gives it, with the same
// operations, so a derivative that several equations use is evaluated again
// in each: the energy equation re-evaluates the three viscous terms of the
// momentum equations, and every equation re-reads div u and the velocities.
template <class T, int E, class Acc>
__device__ __forceinline__ T rs_equation(const Acc& A, const Grid& g, const Phys& ph) {
    constexpr int U = 5, P = 8, TT = 9;
    T uc[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) uc[i] = A.center(U + i);
    const T div = A.grad(0, 0) + A.grad(1, 1) + A.grad(2, 2);
    const Shift<T> sh = shift_of<T>(ph);
    T nu, ka;
    visc_consts(ph, nu, ka);
    T r = T(-0.5) * fmx(A.center(E), div, conv_of<T>(A, g, E, uc));
    if constexpr (E == 0) {
        r = fmx(-sh.c_rho, div, r);
    } else if constexpr (E < 4) {
        constexpr int i = E - 1;
        T lap, gd;
        viscous_of<T, true>(A, g, i, uc[i], lap, gd);
        const T vi = nu * fmx(gd, T(1.0 / 3.0), lap);
        r += vi - d1_of<T>(A, g, P, i);
    } else {
        r = fmx(-sh.c_E, div, r);
        T work = 0;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            T lap, gd;
            viscous_of<T, true>(A, g, i, uc[i], lap, gd);
            work = fmx(uc[i], nu * fmx(gd, T(1.0 / 3.0), lap), work);
        }
        T diss = 0;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                T sij = A.grad(i, j) + A.grad(j, i);
                if (i == j) sij = fmx(T(-2.0 / 3.0), div, sij);
                diss = fmx(sij, A.grad(i, j), diss);
            }
        T dpu = 0;
#pragma unroll
        for (int j = 0; j < 3; ++j) dpu += d1_prod_of<T>(A, g, P, U + j, j);
        T lapT;
        {
            const T T0 = A.center(TT);
            T d2[3];
#pragma unroll
            for (int j = 0; j < 3; ++j) d2[j] = d2_of<T>(A, g, TT, j, T0);
            lapT = d2[0] + d2[1] + d2[2];
        }
        r += fmx(nu, diss, fmx(ka, lapT, work)) - dpu;
    }
    return r;
}

// One thread per (point, equation): threadIdx.y is the equation, so a warp
// (32 consecutive points of one equation) never diverges, and no derivative
// is shared between the equations of a point, since each is evaluated by its
// own thread.  Each thread updates its own conserved variable; the five new
// values of a point meet in shared memory for the next-stage primitives.
constexpr int kRsPoints = 64;

template <class T, bool RESID>
__global__ void __launch_bounds__(kRsPoints * 5) k_rs(Grid g, Phys ph, RKStage rk, const T* __restrict__ Qf,
                                                      const T* __restrict__ Wf, const T* __restrict__ Gw,
                                                      const state_t<T>* __restrict__ Q64,
                                                      state_t<T>* __restrict__ out, state_t<T>* __restrict__ Qs,
                                                      T* __restrict__ Wnext) {
    using S = state_t<T>;
    __shared__ S qn_sh[5][kRsPoints];
    const int tx = threadIdx.x, e = threadIdx.y;
    const int idx = blockIdx.x * kRsPoints + tx;
    const int n = g.n;
    const bool valid = idx < n;
    if (valid) {
        const Nbr s = make_nbr(g, idx);
        const GlobalAcc<T> A{s, n, Qf, Wf, Gw};
        T r;
        switch (e) {
            case 0: r = rs_equation<T, 0>(A, g, ph); break;
            case 1: r = rs_equation<T, 1>(A, g, ph); break;
            case 2: r = rs_equation<T, 2>(A, g, ph); break;
            case 3: r = rs_equation<T, 3>(A, g, ph); break;
            default: r = rs_equation<T, 4>(A, g, ph); break;
        }
        // the per-variable branch of stage_write
        if (RESID) {
            out[e * n + idx] = to_state(r);
        } else {
            const S qs = rk.stage == 0 ? Q64[e * n + idx] : Qs[e * n + idx];
            const S qn = upd(rk_a(rk, S()), r, qs);
            out[e * n + idx] = qn;
            if (rk.stage < 2) Qs[e * n + idx] = upd(rk_b(rk, S()), r, qs);
            qn_sh[e][tx] = qn;
        }
    }
    if (RESID) return;
    __syncthreads();
    if (valid && e == 0) {
        S q[5];
#pragma unroll
        for (int f = 0; f < 5; ++f) q[f] = qn_sh[f][tx];
        prims_point(ph, q, Wnext, n, idx);
    }
}

// ------------------------------------------------------------- batched path
// Many instances of different grids in one launch per kernel: a persistent
// grid walks a work list of tiles (instance, first point, count) with a grid
// stride; each block stages its tile's instance record in shared memory and
// runs the same per-point code as the single-instance kernels, so a batched
// instance evolves bitwise as it would alone.  `parity` selects Q[parity] /
// W[parity] as the stage's input (all instances of a batch flip together).
// Launch shape of the batched global-memory fused kernel: binary64 store-some
// 128 threads with registers capped for three blocks (12 warps per SM; the
// FP64 pipe needs the warps: 8 warps of 256-thread blocks gave 7.1 solves/s
// on the 64-instance ensemble, 16 warps with 100 bytes of spills 11.9, 12
// warps 12.0), binary64 recompute-all 128 threads without a cap (its residual
// needs ~170 registers), binary32 256 threads, two blocks per SM.
template <class T>
constexpr int kBatchFusedThreads = sizeof(T) == sizeof(double) ? 128 : 256;
template <class T, bool STORED_G>
constexpr int kBatchFusedMinBlocks = sizeof(T) == sizeof(double) ? (STORED_G ? 3 : 1) : 2;

// The instance record of a work item, copied to shared memory by the whole
// block in 16-byte pieces, and only when the item belongs to another instance
// than the block's previous one (a block's items are mostly of one instance).
template <class Rec>
__device__ __forceinline__ void stage_inst(Rec& I, const Rec* __restrict__ insts, int inst, int& cur) {
    static_assert(sizeof(Rec) % 16 == 0, "the record is copied in 16-byte pieces");
    if (inst == cur) return;
    __syncthreads();  // every thread is done with the previous record
    const int4* src = reinterpret_cast<const int4*>(insts + inst);
    int4* dst = reinterpret_cast<int4*>(&I);
    for (int i = threadIdx.x; i < (int)(sizeof(Rec) / 16); i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    cur = inst;
}

template <class T, bool STORED_G>
__global__ void __launch_bounds__(kBatchFusedThreads<T>, kBatchFusedMinBlocks<T, STORED_G>)
    k_batch_fused(const BatchInst<T>* __restrict__ insts, const BatchTile* __restrict__ tiles, int ntiles, int stage,
                  int parity) {
    __shared__ BatchInst<T> I;
    int cur = -1;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const BatchTile tl = tiles[t];
        stage_inst(I, insts, tl.inst, cur);
        const int n = I.g.n;
        const state_t<T>* Qin = I.Q[parity];
        state_t<T>* Qout = I.Q[1 - parity];
        const T* Wc = I.W[parity];
        const T* Qf = sizeof(T) == sizeof(double) ? reinterpret_cast<const T*>(Qin) : Wc;
        const T* Wf = sizeof(T) == sizeof(double) ? Wc : Wc + 5 * (size_t)n;
        const RKStage rk = I.rk[stage];
        for (int p = threadIdx.x; p < tl.count; p += blockDim.x) {
            const Nbr s = make_nbr(I.g, tl.start + p);
            T R[5];
            fused_residual<T, STORED_G>(GlobalAcc<T>{s, n, Qf, Wf, I.G}, I.k, R);
            stage_write<T, false>(rk, I.ph, n, s.c, Qin, R, Qout, I.Qs, I.W[1 - parity]);
        }
    }
}

// Batched recompute-all with shared-memory staging: work item t of an
// instance is the x-y tile t % (ntx nty) of z-chunk t / (ntx nty) (tiles of
// kTX x kTY points, chunks of kZChunk planes), carried in BatchTile::start.
template <class T>
__global__ void __launch_bounds__(kTX* kTY, sizeof(T) == 4 ? 2 : 1)
    k_batch_ra_tiled(const BatchInst<T>* __restrict__ insts, const BatchTile* __restrict__ tiles, int ntiles,
                     int stage, int parity) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ BatchInst<T> I;
    int cur = -1;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const BatchTile tl = tiles[t];
        stage_inst(I, insts, tl.inst, cur);
        const int ntx = (I.g.nx + kTX - 1) / kTX, nty = (I.g.ny + kTY - 1) / kTY;
        const int zt = tl.start / (ntx * nty), r = tl.start % (ntx * nty);
        const int n = I.g.n;
        const state_t<T>* Qin = I.Q[parity];
        const T* Wc = I.W[parity];
        const T* Qf = sizeof(T) == sizeof(double) ? reinterpret_cast<const T*>(Qin) : Wc;
        const T* Wf = sizeof(T) == sizeof(double) ? Wc : Wc + 5 * (size_t)n;
        const RKStage rk = I.rk[stage];
        ra_tiled_block<T, false>(reinterpret_cast<T*>(smem_raw), I.g, I.k, I.ph, rk, Qf, Wf, Qin, I.Q[1 - parity],
                                 I.Qs, I.W[1 - parity], (r % ntx) * kTX, (r / ntx) * kTY, zt * kZChunk);
    }
}

template <class T>
__global__ void __launch_bounds__(256) k_batch_grad(const BatchInst<T>* __restrict__ insts,
                                                    const BatchTile* __restrict__ tiles, int ntiles, int parity) {
    __shared__ BatchInst<T> I;
    int cur = -1;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const BatchTile tl = tiles[t];
        stage_inst(I, insts, tl.inst, cur);
        const int n = I.g.n;
        const T* Wc = I.W[parity];
        const T* Wf = sizeof(T) == sizeof(double) ? Wc : Wc + 5 * (size_t)n;
        for (int p = threadIdx.x; p < tl.count; p += blockDim.x) {
            const Nbr s = make_nbr(I.g, tl.start + p);
            T G[3][3];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    T tp[4];
                    taps(Wf + i * n, s.c, s.o[j], tp);
                    G[i][j] = I.k.s1[j] * delta1_taps(tp);
                    I.G[(3 * i + j) * n + s.c] = G[i][j];
                }
            store_pair_sums(G, I.G + 9 * (size_t)n, n, s.c);
        }
    }
}

template <class T>
__global__ void __launch_bounds__(256) k_batch_prims(const BatchInst<T>* __restrict__ insts,
                                                     const BatchTile* __restrict__ tiles, int ntiles, int parity) {
    __shared__ BatchInst<T> I;
    int cur = -1;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const BatchTile tl = tiles[t];
        stage_inst(I, insts, tl.inst, cur);
        const int n = I.g.n;
        for (int p = threadIdx.x; p < tl.count; p += blockDim.x) {
            const int c = tl.start + p;
            state_t<T> q[5];
#pragma unroll
            for (int f = 0; f < 5; ++f) q[f] = I.Q[parity][f * n + c];
            if constexpr (sizeof(T) == sizeof(float)) {
                if (I.padded) {  // TMA-staged recompute-all instance: ghost-padded fields
                    float v[10];
                    prims_values(I.ph, q, v);
                    put_padded(pad_layout(I.g), I.W[parity], c % I.g.nx, (c / I.g.nx) % I.g.ny,
                               c / (I.g.nx * I.g.ny), v);
                    continue;
                }
            }
            prims_point(I.ph, q, I.W[parity], n, c);
        }
    }
}

// Batched mixed store-some: the single-instance per-point code (hyb_prims_point,
// ss_hyb_conv_point, ss_hyb_point) over the tile work lists, so a batched
// instance evolves bitwise as it would alone.
__global__ void __launch_bounds__(256) k_batch_prims_hyb(const BatchHyb* __restrict__ insts,
                                                         const BatchTile* __restrict__ tiles, int ntiles,
                                                         int parity) {
    __shared__ BatchHyb I;
    int cur = -1;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const BatchTile tl = tiles[t];
        stage_inst(I, insts, tl.inst, cur);
        const int n = I.g.n;
        for (int p = threadIdx.x; p < tl.count; p += blockDim.x) {
            const int c = tl.start + p;
            double q[5];
#pragma unroll
            for (int f = 0; f < 5; ++f) q[f] = I.Q[parity][f * n + c];
            hyb_prims_point(I.ph, q, I.F[parity], I.W64[parity], n, c);
        }
    }
}

__global__ void __launch_bounds__(128, 4) k_batch_ss_hyb(const BatchHyb* __restrict__ insts,
                                                         const BatchTile* __restrict__ tiles, int ntiles, int stage,
                                                         int parity) {
    __shared__ BatchHyb I;
    int cur = -1;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const BatchTile tl = tiles[t];
        stage_inst(I, insts, tl.inst, cur);
        for (int p = threadIdx.x; p < tl.count; p += blockDim.x)
            ss_hyb_point<false>(I.g, I.k, I.ph, I.rk[stage], I.c_E, I.F[parity], I.G, I.Rc, I.Dv, I.Q[parity],
                                I.Q[1 - parity], I.Qs, I.F[1 - parity], I.W64[1 - parity], tl.start + p);
    }
}

__global__ void __launch_bounds__(128, 5) k_batch_ss_hyb_conv(const BatchHyb* __restrict__ insts,
                                                              const BatchTile* __restrict__ tiles, int ntiles,
                                                              int parity) {
    __shared__ BatchHyb I;
    int cur = -1;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const BatchTile tl = tiles[t];
        stage_inst(I, insts, tl.inst, cur);
        for (int p = threadIdx.x; p < tl.count; p += blockDim.x)
            ss_hyb_conv_point(I.g, I.k, I.F[parity], I.W64[parity], I.G, I.Dv, I.Rc, tl.start + p);
    }
}

int batch_hyb_blocks_per_sm(int kernel) {
    int b = 0;
    cudaError_t e = kernel == 0   ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch_prims_hyb, 256, 0)
                    : kernel == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch_ss_hyb, 128, 0)
                                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch_ss_hyb_conv, 128, 0);
    return e == cudaSuccess && b > 0 ? b : 1;
}

cudaError_t launch_batch_prims_hyb(const BatchHyb* insts, const BatchTile* tiles, int ntiles, int parity, int grid,
                                   cudaStream_t st) {
    if (ntiles <= 0) return cudaSuccess;
    k_batch_prims_hyb<<<grid, 256, 0, st>>>(insts, tiles, ntiles, parity);
    return cudaGetLastError();
}


cudaError_t launch_batch_ss_hyb(const BatchHyb* insts, const BatchTile* tiles, int ntiles, int stage, int parity,
                                int grid_conv, int grid, cudaStream_t st) {
    if (ntiles <= 0) return cudaSuccess;
    k_batch_ss_hyb_conv<<<grid_conv, 128, 0, st>>>(insts, tiles, ntiles, parity);
    k_batch_ss_hyb<<<grid, 128, 0, st>>>(insts, tiles, ntiles, stage, parity);
    return cudaGetLastError();
}

int tiled_work_items(int nx, int ny, int nz) {
    return ((nx + kTX - 1) / kTX) * ((ny + kTY - 1) / kTY) * ((nz + kZChunk - 1) / kZChunk);
}

template <class T>
size_t tiled_smem_bytes() {
    return (size_t)kRing * kNF * kPlane * sizeof(T);
}

template <class T>
int batch_tiled_blocks_per_sm() {
    int b = 0;
    const size_t smem = tiled_smem_bytes<T>();
    if (cudaFuncSetAttribute(k_batch_ra_tiled<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 1;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch_ra_tiled<T>, kTX * kTY, smem);
    return e == cudaSuccess && b > 0 ? b : 1;
}

template <class T>
cudaError_t launch_batch_ra_tiled(const BatchInst<T>* insts, const BatchTile* tiles, int ntiles, int stage,
                                  int parity, int grid, cudaStream_t st) {
    if (ntiles <= 0) return cudaSuccess;
    // The shared-memory size attribute was set by batch_tiled_blocks_per_sm (a
    // host call, kept out of this launch so that the launch can be captured).
    k_batch_ra_tiled<T><<<grid, kTX * kTY, tiled_smem_bytes<T>(), st>>>(insts, tiles, ntiles, stage, parity);
    return cudaGetLastError();
}

template <class T>
int batch_blocks_per_sm(bool fused, bool stored_g) {
    int b = 0;
    cudaError_t e;
    if (!fused)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch_grad<T>, 256, 0);
    else if (stored_g)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch_fused<T, true>, kBatchFusedThreads<T>, 0);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch_fused<T, false>, kBatchFusedThreads<T>, 0);
    return e == cudaSuccess && b > 0 ? b : 1;
}

template <class T>
cudaError_t launch_batch_prims(const BatchInst<T>* insts, const BatchTile* tiles, int ntiles, int parity, int grid,
                               cudaStream_t st) {
    if (ntiles <= 0) return cudaSuccess;
    k_batch_prims<T><<<grid, 256, 0, st>>>(insts, tiles, ntiles, parity);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_batch_grad(const BatchInst<T>* insts, const BatchTile* tiles, int ntiles, int parity, int grid,
                              cudaStream_t st) {
    if (ntiles <= 0) return cudaSuccess;
    k_batch_grad<T><<<grid, 256, 0, st>>>(insts, tiles, ntiles, parity);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_batch_fused(const BatchInst<T>* insts, const BatchTile* tiles, int ntiles, bool stored_g,
                               int stage, int parity, int grid, cudaStream_t st) {
    if (ntiles <= 0) return cudaSuccess;
    if (stored_g)
        k_batch_fused<T, true><<<grid, kBatchFusedThreads<T>, 0, st>>>(insts, tiles, ntiles, stage, parity);
    else
        k_batch_fused<T, false><<<grid, kBatchFusedThreads<T>, 0, st>>>(insts, tiles, ntiles, stage, parity);
    return cudaGetLastError();
}

#define FD_INSTANTIATE_BATCH(T)                                                                                  \
    template int batch_blocks_per_sm<T>(bool, bool);                                                            \
    template int batch_tiled_blocks_per_sm<T>();                                                                \
    template cudaError_t launch_batch_ra_tiled<T>(const BatchInst<T>*, const BatchTile*, int, int, int, int,    \
                                                  cudaStream_t);                                                \
    template cudaError_t launch_batch_prims<T>(const BatchInst<T>*, const BatchTile*, int, int, int,            \
                                               cudaStream_t);                                                   \
    template cudaError_t launch_batch_grad<T>(const BatchInst<T>*, const BatchTile*, int, int, int, cudaStream_t); \
    template cudaError_t launch_batch_fused<T>(const BatchInst<T>*, const BatchTile*, int, bool, int, int, int,  \
                                               cudaStream_t);
FD_INSTANTIATE_BATCH(double)
FD_INSTANTIATE_BATCH(float)
#undef FD_INSTANTIATE_BATCH

// ---------------------------------------------------------------- Section 3
// Kinetic energy and enstrophy, always in binary64.  Pass 1 writes
// u = rho u / rho into Wv; pass 2 forms rho|u|^2/2 and rho|omega|^2/2 per
// point, sums them over a fixed grid-stride assignment and a fixed shuffle
// tree into one partial per block; pass 3 sums the partials in index order.
// The rounding therefore depends only on the grid size, never on scheduling.
__global__ void __launch_bounds__(256) k_velocity_f64(Grid g, const double* __restrict__ Q, double* __restrict__ Wv) {
    int idx = grid_index();
    if (idx >= g.n) return;
    const int n = g.n;
    double inv = 1.0 / Q[idx];
    Wv[idx] = Q[n + idx] * inv;
    Wv[n + idx] = Q[2 * n + idx] * inv;
    Wv[2 * n + idx] = Q[3 * n + idx] * inv;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    return v;
}

__global__ void __launch_bounds__(kDiagThreads) k_diag_partial_f64(Grid g, const double* __restrict__ Q,
                                                                    const double* __restrict__ Wv,
                                                                    double* __restrict__ partial) {
    const int n = g.n;
    double ke = 0.0, en = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const Nbr s = make_nbr(g, (int)i);
        const int c = s.c;
        double G[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                G[i][j] = g.inv12h[j] * delta1<double>([&](int k) { return ld(Wv + i * n, k); }, c, s.o[j]);
        double rho = Q[c];
        double u = Wv[c], v = Wv[n + c], w = Wv[2 * n + c];
        double ox = G[2][1] - G[1][2];
        double oy = G[0][2] - G[2][0];
        double oz = G[1][0] - G[0][1];
        ke = fmx(0.5 * rho, fmx(u, u, fmx(v, v, w * w)), ke);
        en = fmx(0.5 * rho, fmx(ox, ox, fmx(oy, oy, oz * oz)), en);
    }
    __shared__ double sk[kDiagThreads / 32], se[kDiagThreads / 32];
    ke = warp_sum(ke);
    en = warp_sum(en);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sk[wid] = ke;
        se[wid] = en;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < kDiagThreads / 32; ++i) {
            a += sk[i];
            b += se[i];
        }
        partial[2 * blockIdx.x] = a;
        partial[2 * blockIdx.x + 1] = b;
    }
}

__global__ void k_diag_final_f64(const double* __restrict__ partial, int nblocks, double inv_n,
                                 double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < nblocks; ++i) {
            a += partial[2 * i];
            b += partial[2 * i + 1];
        }
        out[0] = a * inv_n;
        out[1] = b * inv_n;
    }
}

// Non-finite scan of m values; sets *flag to 1 if any is NaN or infinite.
__global__ void k_check_finite(const double* __restrict__ x, long long m, int* __restrict__ flag) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x)
        if (!isfinite(x[i])) {
            *flag = 1;
            return;
        }
}

// ---------------------------------------------------------------- launchers

static inline int blocks_for(int n, int threads) { return (n + threads - 1) / threads; }

cudaError_t launch_tgv_ic(const Grid& g, const Phys& ph, double hx, double hy, double hz, double* Q,
                          cudaStream_t st, int z0, int nz_period) {
    k_tgv_ic<<<blocks_for(g.n, 256), 256, 0, st>>>(g, ph, hx, hy, hz, z0, nz_period > 0 ? nz_period : g.nz, Q);
    return cudaGetLastError();
}

cudaError_t launch_prims_f64(const Grid& g, const Phys& ph, const double* Q, double* W, cudaStream_t st) {
    k_prims<double><<<blocks_for(g.n, 256), 256, 0, st>>>(g, ph, Q, W);
    return cudaGetLastError();
}

cudaError_t launch_prims_f32(const Grid& g, const Phys& ph, const df64* Q, float* F, cudaStream_t st) {
    k_prims<float><<<blocks_for(g.n, 256), 256, 0, st>>>(g, ph, Q, F);
    return cudaGetLastError();
}

cudaError_t launch_prims_df64(const Grid& g, const Phys& ph, const df64* Q, df64* F, cudaStream_t st) {
    k_prims<df64><<<blocks_for(g.n, 256), 256, 0, st>>>(g, ph, Q, F);
    return cudaGetLastError();
}

// binary64 <-> double-word conversion of 5 arrays of n values (API boundary of
// the df64 mode).  The double-word state is kept shifted, Q - shift with
// shift = (1, 0, 0, 0, rhoE0) for the state, so its 48 bits resolve the
// perturbations rather than the means; the shift is applied in binary64.
__global__ void k_to_df64(const double* __restrict__ src, df64* __restrict__ dst, long long n, Shift5 sh) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 5 * n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = df64(src[i] - sh.s[i / n]);
}
__global__ void k_from_df64(const df64* __restrict__ src, double* __restrict__ dst, long long n, Shift5 sh) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 5 * n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = src[i].to_double() + sh.s[i / n];
}
cudaError_t launch_to_df64(const double* src, df64* dst, long long n, const Shift5& sh, cudaStream_t st) {
    k_to_df64<<<kDiagBlocks, 256, 0, st>>>(src, dst, n, sh);
    return cudaGetLastError();
}
cudaError_t launch_from_df64(const df64* src, double* dst, long long n, const Shift5& sh, cudaStream_t st) {
    k_from_df64<<<kDiagBlocks, 256, 0, st>>>(src, dst, n, sh);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_ra(const Grid& g, const Coef<T>& k, const Phys& ph, const RKStage& rk, bool resid, const T* Qf,
                      const T* Wf, const state_t<T>* Q64, state_t<T>* out, state_t<T>* Qs, T* Wnext, cudaStream_t st) {
    if (resid)
        k_ra<T, true><<<blocks_for(g.n, 128), 128, 0, st>>>(g, k, ph, rk, Qf, Wf, Q64, out, Qs, Wnext);
    else
        k_ra<T, false><<<blocks_for(g.n, 128), 128, 0, st>>>(g, k, ph, rk, Qf, Wf, Q64, out, Qs, Wnext);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_ra_tiled(const Grid& g, const Coef<T>& k, const Phys& ph, const RKStage& rk, bool resid,
                            const T* Qf, const T* Wf, const state_t<T>* Q64, state_t<T>* out, state_t<T>* Qs, T* Wnext,
                            cudaStream_t st) {
    const size_t smem = tiled_smem_bytes<T>();
    dim3 grid((g.nx + kTX - 1) / kTX, (g.ny + kTY - 1) / kTY, (g.nz + kZChunk - 1) / kZChunk);
    cudaError_t e;
    if (resid) {
        if ((e = cudaFuncSetAttribute(k_ra_tiled<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
            return e;
        k_ra_tiled<T, true><<<grid, kTX * kTY, smem, st>>>(g, k, ph, rk, Qf, Wf, Q64, out, Qs, Wnext);
    } else {
        if ((e = cudaFuncSetAttribute(k_ra_tiled<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem)) != cudaSuccess)
            return e;
        k_ra_tiled<T, false><<<grid, kTX * kTY, smem, st>>>(g, k, ph, rk, Qf, Wf, Q64, out, Qs, Wnext);
    }
    return cudaGetLastError();
}

bool tma_staging_ok(const Grid& g) { return g.nx % 4 == 0 && g.nx >= 8 && g.ny >= 4; }

size_t padded_field_points(const Grid& g) { return (size_t)pad_layout(g).np; }

// Planes per block of the single-instance TMA kernel: the longest chunk (of
// 64, 32, 16) that still gives at least twelve waves of two blocks per SM,
// else 8.  Shorter chunks re-read more halo planes (four per chunk) but even
// out the last wave; measured on GB300 (binary32 step, ms): 128^3 chunk 8 /
// 16 / 64: 0.326 / 0.351 / 0.437; 256^3 16 / 32 / 64: 2.15 / 2.20 / 2.27;
// 384^3 16 / 32 / 64: 7.13 / 7.12 / 7.16.  FDGB300_TMA_ZCHUNK overrides it
// (a tuning knob; any value from 4 to 256).
int tma_zchunk(const Grid& g) {
    static const int forced = [] {
        const char* v = std::getenv("FDGB300_TMA_ZCHUNK");
        const int z = v ? std::atoi(v) : 0;
        return z >= 4 && z <= 256 ? z : 0;
    }();
    if (forced) return forced;
    int sms = 152;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long tiles = (long long)((g.nx + kMX - 1) / kMX) * ((g.ny + kMY - 1) / kMY);
    for (int z : {64, 32, 16})
        if (tiles * ((g.nz + z - 1) / z) >= 12LL * kMBlocks * sms) return z;
    return 8;
}

cudaError_t launch_prims_padded(const Grid& g, const Phys& ph, const df64* Q, float* F, cudaStream_t st) {
    k_prims_padded<<<blocks_for(g.n, 256), 256, 0, st>>>(g, ph, Q, F);
    return cudaGetLastError();
}

size_t tma_smem_bytes() { return kMSmem; }
size_t batch_tma_smem_bytes() { return tma_smem_bytes() + sizeof(TmaItem); }

cudaError_t launch_ra_tma(const CUtensorMap& map, const Grid& g, const Coef<float>& k, const Phys& ph,
                          const RKStage& rk, bool resid, const df64* Q64, df64* out, df64* Qs, float* Wnext,
                          int* err, cudaStream_t st, int skip_plane) {
    const int zlen = tma_zchunk(g);
    const dim3 grid((g.nx + kMX - 1) / kMX, (g.ny + kMY - 1) / kMY, (g.nz + zlen - 1) / zlen);
    const size_t smem = tma_smem_bytes();
    if (resid) {
        k_ra_tma<true><<<grid, kMThreads, smem, st>>>(map, g, k, ph, rk, Q64, out, Qs, Wnext, err, zlen, skip_plane);
    } else {
        k_ra_tma<false><<<grid, kMThreads, smem, st>>>(map, g, k, ph, rk, Q64, out, Qs, Wnext, err, zlen, skip_plane);
    }
    return cudaGetLastError();
}

// Tensor map of the ten ghost-padded binary32 working fields (PadLayout) with
// the box the kernel copies; the encoder is the driver's, looked up once.
cudaError_t encode_field_map(CUtensorMap* map, const float* F, const Grid& g) {
    using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static Encode encode = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<Encode>(p);
    }();
    if (!encode) return cudaErrorNotSupported;
    if (!tma_staging_ok(g) || (reinterpret_cast<uintptr_t>(F) & 15)) return cudaErrorInvalidValue;
    const PadLayout L = pad_layout(g);
    const cuuint64_t dims[4] = {(cuuint64_t)L.px, (cuuint64_t)L.py, (cuuint64_t)g.nz, (cuuint64_t)kNF};
    const cuuint64_t strides[3] = {(cuuint64_t)L.px * 4, (cuuint64_t)L.px * L.py * 4, (cuuint64_t)L.np * 4};
    const cuuint32_t box[4] = {kBX, kBY, 1, kNF};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(F), dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t prepare_ra_tma() {
    const int smem = (int)tma_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(k_ra_tma<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_ra_tma<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_batch_ra_tma<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)batch_tma_smem_bytes());
    return e;
}

int batch_tma_blocks_per_sm() {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch_ra_tma<false>, kMThreads, batch_tma_smem_bytes()) !=
            cudaSuccess ||
        b < 1)
        b = 1;
    return b;
}

int tma_work_items(int nx, int ny, int nz, int zlen) {
    return ((nx + kMX - 1) / kMX) * ((ny + kMY - 1) / kMY) * ((nz + zlen - 1) / zlen);
}

int tma_batch_zchunk(const int* dims, int count, int blocks) {
    for (int z : {64, 32, 16}) {
        long long items = 0;
        for (int i = 0; i < count; ++i) items += tma_work_items(dims[3 * i], dims[3 * i + 1], dims[3 * i + 2], z);
        if (items >= 12LL * blocks) return z;
    }
    return 8;
}

cudaError_t launch_batch_ra_tma(const BatchInst<float>* insts, const BatchTile* tiles, int ntiles, int stage,
                                int parity, int grid, int zlen, int* err, cudaStream_t st) {
    if (ntiles == 0) return cudaSuccess;
    k_batch_ra_tma<false><<<grid, kMThreads, batch_tma_smem_bytes(), st>>>(insts, tiles, ntiles, stage, parity, err,
                                                                          zlen);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_ss_grad(const Grid& g, const Coef<T>& k, const T* Wf, T* Gw, cudaStream_t st) {
    k_ss_grad<T><<<blocks_for(g.n, 256), 256, 0, st>>>(g, k, Wf, Gw);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_ss(const Grid& g, const Coef<T>& k, const Phys& ph, const RKStage& rk, bool resid, const T* Qf,
                      const T* Wf, const T* Gw, const state_t<T>* Q64, state_t<T>* out, state_t<T>* Qs, T* Wnext,
                      cudaStream_t st) {
    if constexpr (std::is_same<T, float>::value) {
        if (resid)
            k_ss_f32<true><<<blocks_for(g.n, 128), 128, 0, st>>>(g, k, ph, rk, Qf, Wf, Gw, Q64, out, Qs, Wnext);
        else
            k_ss_f32<false><<<blocks_for(g.n, 128), 128, 0, st>>>(g, k, ph, rk, Qf, Wf, Gw, Q64, out, Qs, Wnext);
    } else {
        if (resid)
            k_ss<T, true><<<blocks_for(g.n, 128), 128, 0, st>>>(g, k, ph, rk, Qf, Wf, Gw, Q64, out, Qs, Wnext);
        else
            k_ss<T, false><<<blocks_for(g.n, 128), 128, 0, st>>>(g, k, ph, rk, Qf, Wf, Gw, Q64, out, Qs, Wnext);
    }
    return cudaGetLastError();
}

cudaError_t launch_ra_inline(const Grid& g, const Coef<double>& k, const Phys& ph, const RKStage& rk, bool resid,
                             const double* Q64, double* out, double* Qs, cudaStream_t st) {
    if (resid)
        k_ra_inline<true><<<blocks_for(g.n, 128), 128, 0, st>>>(g, k, ph, rk, Q64, out, Qs);
    else
        k_ra_inline<false><<<blocks_for(g.n, 128), 128, 0, st>>>(g, k, ph, rk, Q64, out, Qs);
    return cudaGetLastError();
}

cudaError_t launch_prims_hyb(const Grid& g, const Phys& ph, const double* Q, df64* F, double* W64,
                             cudaStream_t st) {
    k_prims_hyb<<<blocks_for(g.n, 256), 256, 0, st>>>(g, ph, Q, F, W64);
    return cudaGetLastError();
}


cudaError_t launch_ss_hyb(const Grid& g, const Coef<df64>& k, const Phys& ph, const RKStage& rk, bool resid,
                          const df64* F, const double* W64, df64* Gw, df64* Rc, double* Dv, const double* Q64,
                          double* out, double* Qs, df64* Fnext, double* W64next, cudaStream_t st) {
    Coef<df64> kh = k;  // the mean-state terms enter in binary64 (see k_ss_hyb)
    kh.c_rho = df64(0.0f, 0.0f);
    kh.c_E = df64(0.0f, 0.0f);
    const double c_E = -(ph.rhoE0 + ph.p0);
    k_ss_hyb_conv<<<blocks_for(g.n, 128), 128, 0, st>>>(g, kh, F, W64, Gw, Dv, Rc);
    if (resid)
        k_ss_hyb<true><<<blocks_for(g.n, 128), 128, 0, st>>>(g, kh, ph, rk, c_E, F, Gw, Rc, Dv, Q64, out, Qs,
                                                             Fnext, W64next);
    else
        k_ss_hyb<false><<<blocks_for(g.n, 128), 128, 0, st>>>(g, kh, ph, rk, c_E, F, Gw, Rc, Dv, Q64, out, Qs,
                                                              Fnext, W64next);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_bl_prod(const Grid& g, const T* Qf, const T* Wf, T* P, cudaStream_t st) {
    k_bl_prod<T><<<blocks_for(g.n, 256), 256, 0, st>>>(g, Qf, Wf, P);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_bl_d1(const Grid& g, const T* Qf, const T* Wf, const T* P, T* D1, cudaStream_t st) {
    k_bl_d1<T><<<blocks_for(g.n, 256), 256, 0, st>>>(g, Qf, Wf, P, D1);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_bl_d2(const Grid& g, const T* Wf, const T* D1, T* D2, cudaStream_t st) {
    k_bl_d2<T><<<blocks_for(g.n, 256), 256, 0, st>>>(g, Wf, D1, D2);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_bl_res(const Grid& g, const Phys& ph, const RKStage& rk, bool resid, const T* Qf, const T* Wf,
                          const T* D1, const T* D2, const state_t<T>* Q64, state_t<T>* out, state_t<T>* Qs, T* Wnext,
                          cudaStream_t st) {
    if (resid)
        k_bl_res<T, true><<<blocks_for(g.n, 256), 256, 0, st>>>(g, ph, rk, Qf, Wf, D1, D2, Q64, out, Qs, Wnext);
    else
        k_bl_res<T, false><<<blocks_for(g.n, 256), 256, 0, st>>>(g, ph, rk, Qf, Wf, D1, D2, Q64, out, Qs, Wnext);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_sn(const Grid& g, const Phys& ph, const RKStage& rk, bool resid, const T* Qf, const T* Wf,
                      const state_t<T>* Q64, state_t<T>* out, state_t<T>* Qs, T* Wnext, cudaStream_t st) {
    if (resid)
        k_sn<T, true><<<blocks_for(g.n, 128), 128, 0, st>>>(g, ph, rk, Qf, Wf, Q64, out, Qs, Wnext);
    else
        k_sn<T, false><<<blocks_for(g.n, 128), 128, 0, st>>>(g, ph, rk, Qf, Wf, Q64, out, Qs, Wnext);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_rs(const Grid& g, const Phys& ph, const RKStage& rk, bool resid, const T* Qf, const T* Wf,
                      const T* Gw, const state_t<T>* Q64, state_t<T>* out, state_t<T>* Qs, T* Wnext,
                      cudaStream_t st) {
    const dim3 block(kRsPoints, 5);
    if (resid)
        k_rs<T, true><<<blocks_for(g.n, kRsPoints), block, 0, st>>>(g, ph, rk, Qf, Wf, Gw, Q64, out, Qs, Wnext);
    else
        k_rs<T, false><<<blocks_for(g.n, kRsPoints), block, 0, st>>>(g, ph, rk, Qf, Wf, Gw, Q64, out, Qs, Wnext);
    return cudaGetLastError();
}

// binary64 recompute-all runs the global-memory kernel; binary32 and df64 run
// the z-marching kernels (launch_ra_tiled, launch_ra_tma)
template cudaError_t launch_ra<double>(const Grid&, const Coef<double>&, const Phys&, const RKStage&, bool,
                                       const double*, const double*, const double*, double*, double*, double*,
                                       cudaStream_t);
#define FD_INSTANTIATE(T)                                                                                        \
    template cudaError_t launch_ss_grad<T>(const Grid&, const Coef<T>&, const T*, T*, cudaStream_t);            \
    template cudaError_t launch_ss<T>(const Grid&, const Coef<T>&, const Phys&, const RKStage&, bool, const T*,  \
                                      const T*, const T*, const state_t<T>*, state_t<T>*, state_t<T>*, T*,      \
                                      cudaStream_t);                                                            \
    template cudaError_t launch_bl_prod<T>(const Grid&, const T*, const T*, T*, cudaStream_t);                  \
    template cudaError_t launch_bl_d1<T>(const Grid&, const T*, const T*, const T*, T*, cudaStream_t);          \
    template cudaError_t launch_bl_d2<T>(const Grid&, const T*, const T*, T*, cudaStream_t);                    \
    template cudaError_t launch_bl_res<T>(const Grid&, const Phys&, const RKStage&, bool, const T*, const T*,    \
                                          const T*, const T*, const state_t<T>*, state_t<T>*, state_t<T>*, T*,  \
                                          cudaStream_t);                                                        \
    template cudaError_t launch_sn<T>(const Grid&, const Phys&, const RKStage&, bool, const T*, const T*,        \
                                      const state_t<T>*, state_t<T>*, state_t<T>*, T*, cudaStream_t);           \
    template cudaError_t launch_rs<T>(const Grid&, const Phys&, const RKStage&, bool, const T*, const T*,        \
                                      const T*, const state_t<T>*, state_t<T>*, state_t<T>*, T*, cudaStream_t);
FD_INSTANTIATE(double)
FD_INSTANTIATE(float)
FD_INSTANTIATE(df64)
#undef FD_INSTANTIATE
template cudaError_t launch_ra_tiled<float>(const Grid&, const Coef<float>&, const Phys&, const RKStage&, bool,
                                            const float*, const float*, const df64*, df64*, df64*, float*,
                                            cudaStream_t);
template cudaError_t launch_ra_tiled<df64>(const Grid&, const Coef<df64>&, const Phys&, const RKStage&, bool,
                                            const df64*, const df64*, const df64*, df64*, df64*, df64*,
                                            cudaStream_t);

cudaError_t launch_diagnostics_f64(const Grid& g, const double* Q, double* Wv, double* partial, double* out,
                                   cudaStream_t st) {
    k_velocity_f64<<<blocks_for(g.n, 256), 256, 0, st>>>(g, Q, Wv);
    k_diag_partial_f64<<<kDiagBlocks, kDiagThreads, 0, st>>>(g, Q, Wv, partial);
    k_diag_final_f64<<<1, 32, 0, st>>>(partial, kDiagBlocks, 1.0 / (double)g.n, out);
    return cudaGetLastError();
}

cudaError_t launch_check_finite(const double* x, long long m, int* flag, cudaStream_t st) {
    k_check_finite<<<kDiagBlocks, 256, 0, st>>>(x, m, flag);
    return cudaGetLastError();
}

}  // namespace fd
