// fd_internal.h -- launchers shared between the kernel translation units and
// the C-ABI implementation (not part of the public interface).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "fd_core.cuh"

namespace fd {

// Fixed launch shape of the reductions: the partial-sum order, and hence the
// rounding of the diagnostics, depends only on the grid size.
constexpr int kDiagBlocks = 608;   // 4 per SM on a 152-SM GB300
constexpr int kDiagThreads = 256;

// Taylor-Green state of the grid, or (z0, nz_period) of the planes z0 .. z0+nz-1
// (mod nz_period) of a periodic grid of nz_period planes (a slab).
cudaError_t launch_tgv_ic(const Grid& g, const Phys& ph, double hx, double hy, double hz, double* Q,
                          cudaStream_t st, int z0 = 0, int nz_period = 0);
// Primitive variables: binary64 W = (u, v, w, p, T), or the ten binary32
// perturbation fields F = (rho-1, rho u, rho v, rho w, rhoE-rhoE0, u, v, w, p-p0, T-1).
cudaError_t launch_prims_f64(const Grid& g, const Phys& ph, const double* Q, double* W, cudaStream_t st);
cudaError_t launch_prims_f32(const Grid& g, const Phys& ph, const df64* Q, float* F, cudaStream_t st);
cudaError_t launch_prims_df64(const Grid& g, const Phys& ph, const df64* Q, df64* F, cudaStream_t st);
// binary64 <-> double-word conversion of 5 arrays of n values, subtracting /
// adding a per-array shift (df64 mode at the API boundary).
cudaError_t launch_to_df64(const double* src, df64* dst, long long n, const Shift5& sh, cudaStream_t st);
cudaError_t launch_from_df64(const df64* src, double* dst, long long n, const Shift5& sh, cudaStream_t st);

// Kernels of one stage in precision T (double, float or df64), one launch
// each.  Qf / Wf are the five conserved-like and five primitive-like working
// fields, Q64 the state the stage starts from (state_t<T>: binary64, or
// shifted double-words), out the next state (or R when resid), Qs the saved
// register, Wnext the working fields of `out` for the next stage (written by
// the last kernel of a stage unless resid).
//   RA: launch_ra (binary64), launch_ra_tiled (df64, binary32), launch_ra_tma (binary32)
//   SS: launch_ss_grad, launch_ss
//   BL: launch_bl_prod, launch_bl_d1, launch_bl_d2, launch_bl_res
//   SN: launch_sn;  RS: launch_ss_grad, launch_rs
template <class T>
cudaError_t launch_ra(const Grid& g, const Coef<T>& k, const Phys& ph, const RKStage& rk, bool resid, const T* Qf,
                      const T* Wf, const state_t<T>* Q64, state_t<T>* out, state_t<T>* Qs, T* Wnext, cudaStream_t st);
// RA with the fields staged through shared memory (same arithmetic as launch_ra).
// binary32 recompute-all with TMA-staged planes.  Its ten working fields use a
// ghost-padded layout, [10][nz][ny+4][nx+4] with the periodic images in the
// padding (padded_field_points(g) values per field): launch_prims_padded
// writes it from a state, and the kernel writes the next stage's fields in it.
// `map` describes one such buffer (box 36 x 12 x 1 x 10, made by
// encode_field_map); usable when tma_staging_ok(g).  prepare_ra_tma sets the
// kernels' shared-memory size (host set-up, once per device).  A wait that
// runs out (0.5 s) sets *err to 1 (2: the shared ring was misaligned).
bool tma_staging_ok(const Grid& g);
size_t padded_field_points(const Grid& g);
cudaError_t launch_prims_padded(const Grid& g, const Phys& ph, const df64* Q, float* F, cudaStream_t st);
cudaError_t encode_field_map(CUtensorMap* map, const float* F, const Grid& g);
cudaError_t prepare_ra_tma();
// skip_plane >= 0 is a failure-detection test hook: the copy of that plane is
// never issued, so the wait for it runs out (0.5 s) and *err is set.
cudaError_t launch_ra_tma(const CUtensorMap& map, const Grid& g, const Coef<float>& k, const Phys& ph,
                          const RKStage& rk, bool resid, const df64* Q64, df64* out, df64* Qs, float* Wnext,
                          int* err, cudaStream_t st, int skip_plane = -1000000);
template <class T>
cudaError_t launch_ra_tiled(const Grid& g, const Coef<T>& k, const Phys& ph, const RKStage& rk, bool resid,
                            const T* Qf, const T* Wf, const state_t<T>* Q64, state_t<T>* out, state_t<T>* Qs, T* Wnext,
                            cudaStream_t st);
template <class T>
cudaError_t launch_ss_grad(const Grid& g, const Coef<T>& k, const T* Wf, T* Gw, cudaStream_t st);
template <class T>
cudaError_t launch_ss(const Grid& g, const Coef<T>& k, const Phys& ph, const RKStage& rk, bool resid, const T* Qf,
                      const T* Wf, const T* Gw, const state_t<T>* Q64, state_t<T>* out, state_t<T>* Qs, T* Wnext,
                      cudaStream_t st);
// Recompute-all with the primitives recomputed at every tap from the state
// (FD_RECOMPUTE_ALL_INLINE, binary64): no working fields at all.
cudaError_t launch_ra_inline(const Grid& g, const Coef<double>& k, const Phys& ph, const RKStage& rk, bool resid,
                             const double* Q64, double* out, double* Qs, cudaStream_t st);
// Store-some in mixed binary64 / double-word arithmetic (FD_F64_DW): binary64
// state Q / Qs / out, binary64 velocities W64 = (u, v, w) (3 arrays; the
// binary64 pressure is kept only as p - p0 in F), the ten shifted double-word
// working fields F (as in the df64 mode)
// and the nine double-word gradients of launch_ss_grad<df64> (given the df64
// coefficients k) with binary64 div u (Dv, from the binary64 velocities).
// launch_prims_hyb writes F and W64 of a state.
cudaError_t launch_prims_hyb(const Grid& g, const Phys& ph, const double* Q, df64* F, double* W64,
                             cudaStream_t st);
// The fused pass: the gradients, div u and the convective part (one kernel),
// then the rest of the residual and the update (a second).
cudaError_t launch_ss_hyb(const Grid& g, const Coef<df64>& k, const Phys& ph, const RKStage& rk, bool resid,
                          const df64* F, const double* W64, df64* Gw, df64* Rc, double* Dv, const double* Q64,
                          double* out, double* Qs, df64* Fnext, double* W64next, cudaStream_t st);
template <class T>
cudaError_t launch_bl_prod(const Grid& g, const T* Qf, const T* Wf, T* P, cudaStream_t st);
template <class T>
cudaError_t launch_bl_d1(const Grid& g, const T* Qf, const T* Wf, const T* P, T* D1, cudaStream_t st);
template <class T>
cudaError_t launch_bl_d2(const Grid& g, const T* Wf, const T* D1, T* D2, cudaStream_t st);
template <class T>
cudaError_t launch_bl_res(const Grid& g, const Phys& ph, const RKStage& rk, bool resid, const T* Qf, const T* Wf,
                          const T* D1, const T* D2, const state_t<T>* Q64, state_t<T>* out, state_t<T>* Qs, T* Wnext,
                          cudaStream_t st);
// SN: derivatives into thread-local variables, nothing stored.  RS: the nine
// gradients of launch_ss_grad, every other derivative inside each equation.
template <class T>
cudaError_t launch_sn(const Grid& g, const Phys& ph, const RKStage& rk, bool resid, const T* Qf, const T* Wf,
                      const state_t<T>* Q64, state_t<T>* out, state_t<T>* Qs, T* Wnext, cudaStream_t st);
template <class T>
cudaError_t launch_rs(const Grid& g, const Phys& ph, const RKStage& rk, bool resid, const T* Qf, const T* Wf,
                      const T* Gw, const state_t<T>* Q64, state_t<T>* out, state_t<T>* Qs, T* Wnext,
                      cudaStream_t st);
// ---- batched path ----------------------------------------------------------
// One instance of a batch as the kernels see it (device memory, read per tile).
template <class T>
struct BatchInst {
    Grid g;
    Coef<T> k;
    Phys ph;
    state_t<T>* Q[2];  // ping-pong state (binary64, or shifted double-words in the binary32 mode)
    state_t<T>* Qs;    // saved RK register
    CUtensorMap fmap[2];  // binary32 RA with TMA staging: maps of W[0] / W[1] (else unused)
    T* W[2];       // working fields of Q[0] / Q[1] (binary64: 5 primitives; binary32: 10 perturbation fields)
    T* G;          // SS: nine velocity gradients (else null)
    int padded;    // binary32 RA with TMA staging: W[] in the ghost-padded layout
    RKStage rk[3];  // a_s dt, b_s dt of each stage (binary64 and double-word)
};

// A contiguous run of points [start, start + count) of one instance.
struct BatchTile {
    int inst, start, count;
};

// One instance of a batch in the mixed binary64 / double-word store-some
// arithmetic (FD_F64_DW): binary64 state, double-word working fields F,
// binary64 u, v, w (W64), double-word gradients G and binary64 div u (Dv).
// k is the df64 coefficient record with its mean-state terms zeroed (they
// enter in binary64, c_E = -(rhoE0 + p0)).
struct alignas(16) BatchHyb {
    Grid g;
    Coef<df64> k;
    Phys ph;
    RKStage rk[3];
    double c_E;
    double* Q[2];
    double* Qs;
    df64* F[2];
    double* W64[2];
    df64* G;
    double* Dv;
    df64* Rc;  // convective part of the residual (first of the two fused kernels)
};
int batch_hyb_blocks_per_sm(int kernel);  // 0: primitives, 1: fused (second kernel), 2: gradients + convective part
cudaError_t launch_batch_prims_hyb(const BatchHyb* insts, const BatchTile* tiles, int ntiles, int parity, int grid,
                                   cudaStream_t st);
// The two fused kernels of a stage (gradients, div u and the convective part, then the rest and the
// update); grid_conv and grid the persistent grids of the two.
cudaError_t launch_batch_ss_hyb(const BatchHyb* insts, const BatchTile* tiles, int ntiles, int stage, int parity,
                                int grid_conv, int grid, cudaStream_t st);

template <class T>
int batch_blocks_per_sm(bool fused, bool stored_g);

// Batched binary32 recompute-all through shared memory: work items are the
// (x-y tile, z-chunk) pairs of an instance, numbered 0 .. tiled_work_items-1
// in BatchTile::start.  batch_tiled_blocks_per_sm also sets the kernel's
// shared-memory attribute and must run on the device before the first launch.
int tiled_work_items(int nx, int ny, int nz);
template <class T>
int batch_tiled_blocks_per_sm();
// Batched binary32 recompute-all with TMA-staged planes: work items are the
// (32 x 8 tile, zlen-plane z-chunk) pairs of an instance, numbered 0 ..
// tma_work_items-1 in BatchTile::start; two blocks per SM where they fit
// (each ring takes 115 KB of shared memory); prepare_ra_tma must have run on
// the device.  tma_batch_zchunk picks zlen for instances of the given grid
// sizes (nx, ny, nz per instance) and a persistent grid of `blocks`.
int tma_work_items(int nx, int ny, int nz, int zlen);
int tma_batch_zchunk(const int* dims, int count, int blocks);
int batch_tma_blocks_per_sm();  // after prepare_ra_tma
cudaError_t launch_batch_ra_tma(const BatchInst<float>* insts, const BatchTile* tiles, int ntiles, int stage,
                                int parity, int grid, int zlen, int* err, cudaStream_t st);
template <class T>
cudaError_t launch_batch_ra_tiled(const BatchInst<T>* insts, const BatchTile* tiles, int ntiles, int stage,
                                  int parity, int grid, cudaStream_t st);
template <class T>
cudaError_t launch_batch_prims(const BatchInst<T>* insts, const BatchTile* tiles, int ntiles, int parity, int grid,
                               cudaStream_t st);
template <class T>
cudaError_t launch_batch_grad(const BatchInst<T>* insts, const BatchTile* tiles, int ntiles, int parity, int grid,
                              cudaStream_t st);
template <class T>
cudaError_t launch_batch_fused(const BatchInst<T>* insts, const BatchTile* tiles, int ntiles, bool stored_g,
                               int stage, int parity, int grid, cudaStream_t st);

cudaError_t launch_diagnostics_f64(const Grid& g, const double* Q, double* Wv, double* partial, double* out,
                                   cudaStream_t st);
cudaError_t launch_check_finite(const double* x, long long m, int* flag, cudaStream_t st);

}  // namespace fd
