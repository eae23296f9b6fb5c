// fd_api.cu -- implementation of the C ABI declared in include/fdgb300.h.
//
// A handle owns one device allocation, carved into 256-byte-aligned arrays:
//   Q[2]  ping-pong conserved state (5 arrays each): a stage reads Q[cur]
//         through its stencils and writes Q[1-cur], so no thread overwrites
//         a value a neighbour still reads (the race Section 2 avoids by
//         splitting loops in BL);
//   Qs    the saved RK register (Fig. 1, save-state), updated pointwise;
//   W[2]  primitives u, v, w, p, T (stored in every family, Section 2),
//         ping-pong: the last kernel of a stage writes the primitives of the
//         new state into W[1-wcur] while the stage reads W[wcur];
//   work  SS, RS: 9 velocity-gradient arrays (binary64: and the 3 pair sums
//         of the diagonal ones); BL: 18 product + 45 first- and 18
//         second-derivative arrays;
//   Wf[2] binary32 mode: the ten perturbation fields, ping-pong likewise
//         (ghost-padded for the TMA-staged recompute-all kernel; W[0] then
//         only serves as scratch of the diagnostics and the residual);
//   Wd[2] df64 and mixed (FD_F64_DW) modes: the ten perturbation fields as
//         double-words (the mixed mode keeps binary64 u, v, w in W[2]);
//   and the reduction scratch.  In the binary32 and df64 modes Q[2] and Qs
//   hold shifted double-words, converted to and from binary64 at the API.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/fdgb300.h"
#include "fd_host.h"
#include "fd_internal.h"

namespace {

using fd::kRkA;
using fd::kRkB;

thread_local std::string g_err;

int fail_global(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

struct fd_handle {
    int nx = 0, ny = 0, nz = 0, n = 0;
    double Re = 0, Mach = 0, Pr = 0, gamma = 0, dt = 0;
    int algorithm = 0, dtype = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    fd_alloc alloc{};
    bool has_alloc = false;
    void* block = nullptr;
    size_t block_bytes = 0;
    double* Q[2] = {nullptr, nullptr};
    int cur = 0;
    double* Qs = nullptr;
    double* W[2] = {nullptr, nullptr};
    float* Wf[2] = {nullptr, nullptr};  // binary32 mode: perturbation fields (10 arrays each)
    fd::df64* Wd[2] = {nullptr, nullptr};  // df64 mode: perturbation fields (10 arrays each)
    int wcur = 0;                       // W[wcur] / Wf[wcur] hold the primitives of Q[cur] ...
    bool wvalid = false;                // ... when wvalid
    double* G = nullptr;   // SS
    double* P = nullptr;   // BL
    double* Dv = nullptr;  // FD_F64_DW: binary64 div u of the current stage
    fd::df64* Rc = nullptr;  // FD_F64_DW: convective part of the residual
    double* D1 = nullptr;  // BL
    double* D2 = nullptr;  // BL
    float* Gf = nullptr;   // binary32 SS: 9 gradients
    fd::df64* Gd = nullptr;  // df64 SS: 9 gradients
    double* partial = nullptr;
    double* diag = nullptr;
    int* flag = nullptr;
    int* kerr = nullptr;       // set by a kernel whose bounded wait ran out
    bool use_tma = false;      // binary32 RA: planes staged by TMA (fmap[b] describes Wf[b])
    // z-slab decomposition (fd_slab_create): the handle's nz planes are ghost + nz_local
    // + ghost planes of a periodic grid of nz_global planes, starting at z_first - ghost
    int slab_ghost = 0, slab_nz_local = 0, slab_z_first = 0, slab_nz_global = 0;
    CUtensorMap fmap[2]{};
    fd::Grid grid{};
    fd::Phys phys{};
    fd::Coef<double> kd{};  // fused-residual coefficients, binary64 mode
    fd::Coef<float> kf{};   // and binary32 perturbation mode
    fd::Coef<fd::df64> kw{};  // and df64 perturbation mode
    fd::Profiler prof;

    template <class T>
    const fd::Coef<T>& coef() const;
    std::string err;

    int fail(int code, const char* fmt, ...) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        err = buf;
        return code;
    }
    int cuda_fail(cudaError_t e, const char* what) {
        return fail(FD_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    }
};

template <>
const fd::Coef<double>& fd_handle::coef<double>() const {
    return kd;
}
template <>
const fd::Coef<float>& fd_handle::coef<float>() const {
    return kf;
}
template <>
const fd::Coef<fd::df64>& fd_handle::coef<fd::df64>() const {
    return kw;
}

namespace {

int check_args(int nx, int ny, int nz, double Re, double Mach, double Pr, double gamma, double dt, int algorithm,
               int dtype) {
    if (const char* why = fd::check_instance(nx, ny, nz, Re, Mach, Pr, gamma, dt))
        return fail_global(FD_EINVAL, "fd_create: grid %dx%dx%d: %s", nx, ny, nz, why);
    if (algorithm != FD_STORE_ALL && algorithm != FD_STORE_SOME && algorithm != FD_RECOMPUTE_ALL &&
        algorithm != FD_RECOMPUTE_SOME && algorithm != FD_STORE_NONE && algorithm != FD_RECOMPUTE_ALL_INLINE)
        return fail_global(FD_EINVAL, "unknown algorithm %d", algorithm);
    if (algorithm == FD_RECOMPUTE_ALL_INLINE && dtype != FD_F64)
        return fail_global(FD_EINVAL, "FD_RECOMPUTE_ALL_INLINE exists in binary64 (FD_F64) only");
    if (dtype != FD_F64 && dtype != FD_F32_ACCDW && dtype != FD_DF64 && dtype != FD_F64_DW)
        return fail_global(FD_EINVAL, "unknown dtype %d", dtype);
    if (dtype == FD_F64_DW && algorithm != FD_STORE_SOME)
        return fail_global(FD_EINVAL, "dtype FD_F64_DW exists for the store-some family only (algorithm %d)",
                           algorithm);
    return FD_OK;
}

// Byte layout of a handle's single device allocation.
struct Layout {
    size_t q0, q1, qs, w0, w1, g, p, d1, d2, wf0, wf1, gf, wd0, wd1, gd, dv, rc, partial, diag, flag, kerr, total;
};

// SS and RS keep the nine velocity gradients in work arrays.
bool stores_g(int algorithm) { return algorithm == FD_STORE_SOME || algorithm == FD_RECOMPUTE_SOME; }

// wf_points: values per binary32 working field (n, or the ghost-padded size
// of the TMA-staged recompute-all kernel).
Layout plan(long long n, int algorithm, int dtype, size_t wf_points) {
    Layout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off += align256(bytes);
        return at;
    };
    size_t f5 = 5 * n * sizeof(double);
    L.q0 = take(f5);
    L.q1 = take(f5);
    L.qs = take(f5);
    L.w1 = L.g = L.p = L.d1 = L.d2 = L.wf0 = L.wf1 = L.gf = L.wd0 = L.wd1 = L.gd = L.dv = L.rc = (size_t)-1;
    L.w0 = dtype == FD_DF64 || algorithm == FD_RECOMPUTE_ALL_INLINE
               ? (size_t)-1
               : take(dtype == FD_F64_DW ? 3 * n * sizeof(double) : f5);
    if (dtype == FD_F64_DW) {
        // binary64 state; W[2] the binary64 u, v, w; Wd[2] the double-word working fields
        L.w1 = take(3 * n * sizeof(double));
        L.wd0 = take(10 * n * sizeof(fd::df64));
        L.wd1 = take(10 * n * sizeof(fd::df64));
        L.gd = take(fd::kHybGradArrays * n * sizeof(fd::df64));  // G_ii only
        L.dv = take(n * sizeof(double));  // binary64 div u of the stage (gradient pass -> fused kernel)
        L.rc = take(5 * n * sizeof(fd::df64));  // convective part of the residual (first fused kernel)
    } else if (dtype == FD_DF64) {
        // state Q[2], Qs hold double-words (8 bytes per value, like binary64)
        L.wd0 = take(10 * n * sizeof(fd::df64));
        L.wd1 = take(10 * n * sizeof(fd::df64));
        if (stores_g(algorithm)) L.gd = take(fd::kGradArrays<fd::df64> * n * sizeof(fd::df64));
        if (algorithm == FD_STORE_ALL) {
            L.p = take(18 * n * sizeof(fd::df64));
            L.d1 = take(45 * n * sizeof(fd::df64));
            L.d2 = take(18 * n * sizeof(fd::df64));
        }
    } else if (dtype == FD_F64 && algorithm == FD_RECOMPUTE_ALL_INLINE) {
        L.w0 = (size_t)-1;  // no primitive arrays: the state alone (the diagnostics use Qs)
    } else if (dtype == FD_F64) {
        L.w1 = take(f5);
        if (stores_g(algorithm)) L.g = take(fd::kGradArrays<double> * n * sizeof(double));
        if (algorithm == FD_STORE_ALL) {
            L.p = take(18 * n * sizeof(double));
            L.d1 = take(45 * n * sizeof(double));
            L.d2 = take(18 * n * sizeof(double));
        }
    } else {
        L.wf0 = take(10 * wf_points * sizeof(float));
        L.wf1 = take(10 * wf_points * sizeof(float));
        if (stores_g(algorithm)) L.gf = take(fd::kGradArrays<float> * n * sizeof(float));
        if (algorithm == FD_STORE_ALL) {
            L.p = take(18 * n * sizeof(float));
            L.d1 = take(45 * n * sizeof(float));
            L.d2 = take(18 * n * sizeof(float));
        }
    }
    L.partial = take(2 * fd::kDiagBlocks * sizeof(double));
    L.diag = take(2 * sizeof(double));
    L.flag = take(sizeof(int));
    L.kerr = take(sizeof(int));
    L.total = off;
    return L;
}

template <class T>
T* at(void* base, size_t off) {
    return off == (size_t)-1 ? nullptr : reinterpret_cast<T*>(static_cast<char*>(base) + off);
}

void device_free(fd_handle* h) {
    if (!h->block) return;
    if (h->has_alloc)
        h->alloc.free(h->alloc.ctx, h->block, h->block_bytes, h->stream);
    else
        cudaFree(h->block);
    h->block = nullptr;
}

template <class F>
cudaError_t timed(fd_handle* h, int cls, F launch) {
    return h->prof.timed(h->stream, cls, launch);
}

// Kernels of one stage of family `alg` in precision T.
template <class T, class S = fd::state_t<T>>
cudaError_t stage_kernels(fd_handle* h, const fd::RKStage& rk, bool resid, const T* Qf, const T* Wf, T* G, T* P,
                          T* D1, T* D2, const S* Qin, S* Qout, T* Wnext) {
    const fd::Grid& g = h->grid;
    const fd::Phys& ph = h->phys;
    const fd::Coef<T>& k = h->coef<T>();
    cudaStream_t st = h->stream;
    cudaError_t e;
    switch (h->algorithm) {
        case FD_RECOMPUTE_ALL:
            // binary32 and df64: fields staged through shared memory (the
            // global-memory kernel is latency-bound on its tap loads; df64 256^3
            // step 16.2 -> 11.0 ms); binary64 is bound by FP64 issue, where staging
            // does not help.
            return timed(h, FD_KERNEL_FUSED, [&] {
                if constexpr (std::is_same<T, float>::value) {
                    if (h->use_tma)  // Qf is the first of the ten fields of Wf[0] or Wf[1]
                        return fd::launch_ra_tma(h->fmap[Qf == h->Wf[0] ? 0 : 1], g, k, ph, rk, resid, Qin, Qout,
                                                 reinterpret_cast<S*>(h->Qs), Wnext, h->kerr, st);
                    return fd::launch_ra_tiled<T>(g, k, ph, rk, resid, Qf, Wf, Qin, Qout, reinterpret_cast<S*>(h->Qs),
                                                  Wnext, st);
                } else if constexpr (std::is_same<T, fd::df64>::value) {
                    return fd::launch_ra_tiled<T>(g, k, ph, rk, resid, Qf, Wf, Qin, Qout, reinterpret_cast<S*>(h->Qs),
                                                  Wnext, st);
                } else
                    return fd::launch_ra<T>(g, k, ph, rk, resid, Qf, Wf, Qin, Qout, reinterpret_cast<S*>(h->Qs),
                                            Wnext, st);
            });
        case FD_STORE_NONE:
            return timed(h, FD_KERNEL_FUSED, [&] {
                return fd::launch_sn<T>(g, ph, rk, resid, Qf, Wf, Qin, Qout, reinterpret_cast<S*>(h->Qs), Wnext, st);
            });
        case FD_RECOMPUTE_SOME:
            e = timed(h, FD_KERNEL_GRAD, [&] { return fd::launch_ss_grad<T>(g, k, Wf, G, st); });
            if (e != cudaSuccess) return e;
            return timed(h, FD_KERNEL_FUSED, [&] {
                return fd::launch_rs<T>(g, ph, rk, resid, Qf, Wf, G, Qin, Qout, reinterpret_cast<S*>(h->Qs), Wnext,
                                        st);
            });
        case FD_STORE_SOME:
            e = timed(h, FD_KERNEL_GRAD, [&] { return fd::launch_ss_grad<T>(g, k, Wf, G, st); });
            if (e != cudaSuccess) return e;
            return timed(h, FD_KERNEL_FUSED, [&] {
                return fd::launch_ss<T>(g, k, ph, rk, resid, Qf, Wf, G, Qin, Qout, reinterpret_cast<S*>(h->Qs),
                                        Wnext, st);
            });
        default:
            e = timed(h, FD_KERNEL_PRODUCTS, [&] { return fd::launch_bl_prod<T>(g, Qf, Wf, P, st); });
            if (e != cudaSuccess) return e;
            e = timed(h, FD_KERNEL_DERIV1, [&] { return fd::launch_bl_d1<T>(g, Qf, Wf, P, D1, st); });
            if (e != cudaSuccess) return e;
            e = timed(h, FD_KERNEL_DERIV2, [&] { return fd::launch_bl_d2<T>(g, Wf, D1, D2, st); });
            if (e != cudaSuccess) return e;
            return timed(h, FD_KERNEL_FUSED, [&] {
                return fd::launch_bl_res<T>(g, ph, rk, resid, Qf, Wf, D1, D2, Qin, Qout, reinterpret_cast<S*>(h->Qs),
                                            Wnext, st);
            });
    }
}

// One RK stage (s = 0, 1, 2), or the bare residual into `out` when resid.
// The primitives of Q[cur] (Fig. 1, evaluate-u_i,p,T) come from the previous
// stage, which wrote them with its update; only after creation or
// fd_set_state is a separate primitives pass needed.
cudaError_t run_stage(fd_handle* h, int s, bool resid, double* out) {
    const fd::Grid& g = h->grid;
    const fd::Phys& ph = h->phys;
    const fd::RKStage rk = fd::make_stage(s, h->dt);
    const double* Qin = h->Q[h->cur];
    double* Qout = resid ? out : h->Q[1 - h->cur];
    const int wc = h->wcur;
    const long long n = h->n;
    cudaError_t e;
    if (h->dtype == FD_F64 && h->algorithm == FD_RECOMPUTE_ALL_INLINE) {
        return timed(h, FD_KERNEL_FUSED, [&] {
            return fd::launch_ra_inline(g, h->kd, ph, rk, resid, Qin, Qout, h->Qs, h->stream);
        });
    }
    if (h->dtype == FD_F64) {
        if (!h->wvalid) {
            e = timed(h, FD_KERNEL_PRIMS, [&] { return fd::launch_prims_f64(g, ph, Qin, h->W[wc], h->stream); });
            if (e != cudaSuccess) return e;
            h->wvalid = true;
        }
        return stage_kernels<double>(h, rk, resid, Qin, h->W[wc], h->G, h->P, h->D1, h->D2, Qin, Qout,
                                     resid ? nullptr : h->W[1 - wc]);
    }
    if (h->dtype == FD_F64_DW) {  // store-some only (fd_create checks)
        using fd::df64;
        if (!h->wvalid) {
            e = timed(h, FD_KERNEL_PRIMS,
                      [&] { return fd::launch_prims_hyb(g, ph, Qin, h->Wd[wc], h->W[wc], h->stream); });
            if (e != cudaSuccess) return e;
            h->wvalid = true;
        }
        return timed(h, FD_KERNEL_FUSED, [&] {
            return fd::launch_ss_hyb(g, h->kw, ph, rk, resid, h->Wd[wc], h->W[wc], h->Gd, h->Rc, h->Dv, Qin, Qout, h->Qs,
                                     resid ? nullptr : h->Wd[1 - wc], resid ? nullptr : h->W[1 - wc], h->stream);
        });
    }
    if (h->dtype == FD_DF64) {
        using fd::df64;
        const df64* Qd = reinterpret_cast<const df64*>(Qin);
        if (!h->wvalid) {
            e = timed(h, FD_KERNEL_PRIMS, [&] { return fd::launch_prims_df64(g, ph, Qd, h->Wd[wc], h->stream); });
            if (e != cudaSuccess) return e;
            h->wvalid = true;
        }
        return stage_kernels<df64>(h, rk, resid, h->Wd[wc], h->Wd[wc] + 5 * n, h->Gd, reinterpret_cast<df64*>(h->P),
                                   reinterpret_cast<df64*>(h->D1), reinterpret_cast<df64*>(h->D2), Qd,
                                   reinterpret_cast<df64*>(Qout), resid ? nullptr : h->Wd[1 - wc]);
    }
    using fd::df64;
    const df64* Qd = reinterpret_cast<const df64*>(Qin);
    if (!h->wvalid) {
        e = timed(h, FD_KERNEL_PRIMS, [&] {
            return h->use_tma ? fd::launch_prims_padded(g, ph, Qd, h->Wf[wc], h->stream)
                              : fd::launch_prims_f32(g, ph, Qd, h->Wf[wc], h->stream);
        });
        if (e != cudaSuccess) return e;
        h->wvalid = true;
    }
    return stage_kernels<float>(h, rk, resid, h->Wf[wc], h->Wf[wc] + 5 * n, h->Gf, reinterpret_cast<float*>(h->P),
                                reinterpret_cast<float*>(h->D1), reinterpret_cast<float*>(h->D2), Qd,
                                reinterpret_cast<df64*>(Qout), resid ? nullptr : h->Wf[1 - wc]);
}

// binary32 and df64 modes: the state buffers hold shifted double-words; these
// move a binary64 copy of the current state through the saved register Qs,
// which is dead between steps (stage 0 rewrites it).
bool dw_state(int dtype) { return dtype == FD_F32_ACCDW || dtype == FD_DF64; }

fd::Shift5 state_shift(const fd_handle* h) { return fd::Shift5{{1.0, 0.0, 0.0, 0.0, h->phys.rhoE0}}; }

// A kernel whose bounded wait ran out (TMA-staged binary32 RA) leaves a
// nonzero error word; the synchronising calls report it.
int check_kernel_error(fd_handle* h, const char* what) {
    if (!h->use_tma) return FD_OK;
    int v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, h->kerr, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return h->cuda_fail(e, what);
    if (v)
        return h->fail(FD_ECUDA, "%s: %s; the state is not valid", what,
                       v == 2 ? "the TMA ring was not 128-byte aligned" : "a staging wait in a kernel ran out");
    return FD_OK;
}

cudaError_t state_to_binary64(fd_handle* h, double* dst) {
    return fd::launch_from_df64(reinterpret_cast<const fd::df64*>(h->Q[h->cur]), dst, h->n, state_shift(h),
                                h->stream);
}

int create_impl(fd_handle** out, int nx, int ny, int nz, int nz_period, int z0, double Re, double Mach, double Pr,
                double gamma, double dt, int algorithm, int dtype, const fd_alloc* alloc, void* cuda_stream);

}  // namespace

extern "C" {

int fd_create(fd_handle** out, int nx, int ny, int nz, double Re, double Mach, double Pr, double gamma, double dt,
              int algorithm, int dtype, const fd_alloc* alloc, void* cuda_stream) {
    return create_impl(out, nx, ny, nz, 0, 0, Re, Mach, Pr, gamma, dt, algorithm, dtype, alloc, cuda_stream);
}

}  // extern "C"

namespace {

// fd_create, and (nz_period > 0) a slab of nz planes of a periodic grid of
// nz_period planes whose plane 0 is plane z0 (mod nz_period) of that grid.
int create_impl(fd_handle** out, int nx, int ny, int nz, int nz_period, int z0, double Re, double Mach, double Pr,
                double gamma, double dt, int algorithm, int dtype, const fd_alloc* alloc, void* cuda_stream) {
    if (!out) return fail_global(FD_EINVAL, "fd_create: out is NULL");
    *out = nullptr;
    int rc = check_args(nx, ny, nz, Re, Mach, Pr, gamma, dt, algorithm, dtype);
    if (rc != FD_OK) return rc;
    if (alloc && (!alloc->alloc || !alloc->free))
        return fail_global(FD_EINVAL, "fd_create: allocator needs both alloc and free");
    fd_handle* h = new (std::nothrow) fd_handle();
    if (!h) return fail_global(FD_ENOMEM, "fd_create: host allocation failed");
    h->nx = nx;
    h->ny = ny;
    h->nz = nz;
    h->n = nx * ny * nz;
    h->Re = Re;
    h->Mach = Mach;
    h->Pr = Pr;
    h->gamma = gamma;
    h->dt = dt;
    h->algorithm = algorithm;
    h->dtype = dtype;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) {
        delete h;
        return fail_global(FD_ECUDA, "fd_create: cudaGetDevice: %s", cudaGetErrorString(e));
    }
    // binary32 recompute-all stages its planes with TMA where the grid allows it
    // (FDGB300_NO_TMA=1 selects the thread-staged kernel, for comparison); its
    // working fields then use the ghost-padded layout.
    const fd::Grid grid0 = fd::make_grid(nx, ny, nz, nz_period);
    if (dtype == FD_F32_ACCDW && algorithm == FD_RECOMPUTE_ALL && fd::tma_staging_ok(grid0)) {
        const char* off = std::getenv("FDGB300_NO_TMA");
        h->use_tma = !(off && off[0] == '1');
    }
    Layout L = plan(h->n, algorithm, dtype, h->use_tma ? fd::padded_field_points(grid0) : (size_t)h->n);
    h->block_bytes = L.total;
    if (alloc) {
        h->alloc = *alloc;
        h->has_alloc = true;
        h->block = alloc->alloc(alloc->ctx, L.total, cuda_stream);
        if (!h->block) {
            delete h;
            return fail_global(FD_ENOMEM, "fd_create: allocator returned NULL for %zu bytes", L.total);
        }
        if (reinterpret_cast<uintptr_t>(h->block) & 255) {
            alloc->free(alloc->ctx, h->block, L.total, cuda_stream);
            delete h;
            return fail_global(FD_EINVAL, "fd_create: allocator returned a pointer not aligned to 256 bytes");
        }
    } else {
        e = cudaMalloc(&h->block, L.total);
        if (e != cudaSuccess) {
            cudaGetLastError();
            delete h;
            return fail_global(FD_ENOMEM, "fd_create: cudaMalloc(%zu): %s", L.total, cudaGetErrorString(e));
        }
    }
    h->Q[0] = at<double>(h->block, L.q0);
    h->Q[1] = at<double>(h->block, L.q1);
    h->Qs = at<double>(h->block, L.qs);
    h->W[0] = at<double>(h->block, L.w0);
    h->W[1] = at<double>(h->block, L.w1);
    h->Wd[0] = at<fd::df64>(h->block, L.wd0);
    h->Wd[1] = at<fd::df64>(h->block, L.wd1);
    h->Gd = at<fd::df64>(h->block, L.gd);
    h->Dv = at<double>(h->block, L.dv);
    h->Rc = at<fd::df64>(h->block, L.rc);
    if (dtype == FD_F64) {
        h->G = at<double>(h->block, L.g);
        h->P = at<double>(h->block, L.p);
        h->D1 = at<double>(h->block, L.d1);
        h->D2 = at<double>(h->block, L.d2);
    } else {
        h->Wf[0] = at<float>(h->block, L.wf0);
        h->Wf[1] = at<float>(h->block, L.wf1);
        h->Gf = at<float>(h->block, L.gf);
        h->P = at<double>(h->block, L.p);
        h->D1 = at<double>(h->block, L.d1);
        h->D2 = at<double>(h->block, L.d2);
    }
    h->partial = at<double>(h->block, L.partial);
    h->diag = at<double>(h->block, L.diag);
    h->flag = at<int>(h->block, L.flag);
    h->kerr = at<int>(h->block, L.kerr);

    const double hx = 2.0 * fd::kPi / nx, hy = 2.0 * fd::kPi / ny,
                 hz = 2.0 * fd::kPi / (nz_period > 0 ? nz_period : nz);
    h->grid = fd::make_grid(nx, ny, nz, nz_period);
    h->phys = fd::make_phys(Re, Mach, Pr, gamma);
    const fd::Grid& g = h->grid;
    const fd::Phys& ph = h->phys;
    h->kd = fd::make_coef<double>(g, ph, false);
    h->kf = fd::make_coef<float>(g, ph, true);
    h->kw = fd::make_coef<fd::df64>(g, ph, true);

    e = cudaMemsetAsync(h->kerr, 0, sizeof(int), h->stream);
    if (e == cudaSuccess && h->use_tma) {
        // the padding columns no point writes are copied but never read: zero them once
        const size_t wf_bytes = 10 * fd::padded_field_points(g) * sizeof(float);
        e = fd::prepare_ra_tma();
        for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
            e = cudaMemsetAsync(h->Wf[b], 0, wf_bytes, h->stream);
            if (e == cudaSuccess) e = fd::encode_field_map(&h->fmap[b], h->Wf[b], g);
        }
    }
    if (e != cudaSuccess) {
        device_free(h);
        delete h;
        return fail_global(FD_ECUDA, "fd_create: staging set-up: %s", cudaGetErrorString(e));
    }
    if (dw_state(dtype)) {
        e = fd::launch_tgv_ic(g, ph, hx, hy, hz, h->Qs, h->stream, z0, nz_period);
        if (e == cudaSuccess)
            e = fd::launch_to_df64(h->Qs, reinterpret_cast<fd::df64*>(h->Q[0]), h->n, state_shift(h), h->stream);
    } else {
        e = fd::launch_tgv_ic(g, ph, hx, hy, hz, h->Q[0], h->stream, z0, nz_period);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        device_free(h);
        delete h;
        return fail_global(FD_ECUDA, "fd_create: initial condition: %s", cudaGetErrorString(e));
    }
    *out = h;
    return FD_OK;
}

}  // namespace

extern "C" {

int fd_step(fd_handle* h, int n) {
    if (!h) return fail_global(FD_EINVAL, "fd_step: NULL handle");
    if (n < 0) return h->fail(FD_EINVAL, "fd_step: n = %d < 0", n);
    for (int it = 0; it < n; ++it)
        for (int s = 0; s < 3; ++s) {
            cudaError_t e = run_stage(h, s, false, nullptr);
            if (e != cudaSuccess) {
                h->wvalid = false;
                return h->cuda_fail(e, "fd_step: kernel launch");
            }
            h->cur = 1 - h->cur;
            h->wcur = 1 - h->wcur;
        }
    return FD_OK;
}

int fd_get_state_async(fd_handle* h, double* dst, size_t n_elems, int dst_is_device) {
    if (!h) return fail_global(FD_EINVAL, "fd_get_state: NULL handle");
    if (!dst) return h->fail(FD_EINVAL, "fd_get_state: dst is NULL");
    if (n_elems != 5 * (size_t)h->n)
        return h->fail(FD_EINVAL, "fd_get_state: n_elems = %zu, expected %zu", n_elems, 5 * (size_t)h->n);
    cudaError_t e = cudaSuccess;
    const double* src = h->Q[h->cur];
    if (dw_state(h->dtype)) {
        double* tmp = dst_is_device ? dst : h->Qs;
        e = state_to_binary64(h, tmp);
        src = tmp;
    }
    if (e == cudaSuccess && src != dst)
        e = cudaMemcpyAsync(dst, src, n_elems * sizeof(double),
                            dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "fd_get_state");
    return FD_OK;
}

int fd_get_state(fd_handle* h, double* dst, size_t n_elems, int dst_is_device) {
    int rc = fd_get_state_async(h, dst, n_elems, dst_is_device);
    if (rc != FD_OK) return rc;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "fd_get_state");
    return check_kernel_error(h, "fd_get_state");
}

int fd_set_state_async(fd_handle* h, const double* src, size_t n_elems, int src_is_device) {
    if (!h) return fail_global(FD_EINVAL, "fd_set_state: NULL handle");
    if (!src) return h->fail(FD_EINVAL, "fd_set_state: src is NULL");
    if (n_elems != 5 * (size_t)h->n)
        return h->fail(FD_EINVAL, "fd_set_state: n_elems = %zu, expected %zu", n_elems, 5 * (size_t)h->n);
    h->wvalid = false;
    double* dst = dw_state(h->dtype) ? h->Qs : h->Q[h->cur];
    cudaError_t e = cudaMemcpyAsync(dst, src, n_elems * sizeof(double),
                                    src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && dw_state(h->dtype))
        e = fd::launch_to_df64(h->Qs, reinterpret_cast<fd::df64*>(h->Q[h->cur]), h->n, state_shift(h), h->stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "fd_set_state");
    return FD_OK;
}

int fd_set_state(fd_handle* h, const double* src, size_t n_elems, int src_is_device) {
    int rc = fd_set_state_async(h, src, n_elems, src_is_device);
    if (rc != FD_OK) return rc;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "fd_set_state");
    return FD_OK;
}

int fd_diagnostics(fd_handle* h, double* ke, double* enstrophy) {
    if (!h) return fail_global(FD_EINVAL, "fd_diagnostics: NULL handle");
    double out[2];
    // Scratch for the velocities: the working-field buffer the next stage will
    // overwrite (binary64, df64), or W[0], unused by the binary32 stages.  The
    // double-word modes first convert the state to binary64 in Qs (dead
    // between steps).
    double* Wv = h->algorithm == FD_RECOMPUTE_ALL_INLINE          ? h->Qs
                 : h->dtype == FD_F64                             ? h->W[1 - h->wcur]
                 : h->dtype == FD_DF64 || h->dtype == FD_F64_DW ? reinterpret_cast<double*>(h->Wd[1 - h->wcur])
                                                                : h->W[0];
    const double* Q = h->Q[h->cur];
    cudaError_t e = cudaSuccess;
    if (dw_state(h->dtype)) {
        e = state_to_binary64(h, h->Qs);
        Q = h->Qs;
    }
    if (e == cudaSuccess) e = fd::launch_diagnostics_f64(h->grid, Q, Wv, h->partial, h->diag, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, h->diag, sizeof out, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "fd_diagnostics");
    if (int rc = check_kernel_error(h, "fd_diagnostics")) return rc;
    if (ke) *ke = out[0];
    if (enstrophy) *enstrophy = out[1];
    return FD_OK;
}

int fd_residual(fd_handle* h, double* R, size_t n_elems, int dst_is_device) {
    if (!h) return fail_global(FD_EINVAL, "fd_residual: NULL handle");
    if (!R) return h->fail(FD_EINVAL, "fd_residual: R is NULL");
    if (n_elems != 5 * (size_t)h->n)
        return h->fail(FD_EINVAL, "fd_residual: n_elems = %zu, expected %zu", n_elems, 5 * (size_t)h->n);
    // Between steps the saved register Qs is dead (stage 0 rewrites it), so it
    // serves as the device buffer for R.  The double-word modes evaluate R as
    // double-words into a spare buffer (the df64 working fields the next stage
    // overwrites, or W[0], unused by the binary32 stages), then convert it.
    double* out = dst_is_device ? R : h->Qs;
    cudaError_t e;
    if (dw_state(h->dtype)) {
        double* Rw = h->dtype == FD_DF64 ? reinterpret_cast<double*>(h->Wd[1 - h->wcur]) : h->W[0];
        e = run_stage(h, 0, true, Rw);
        if (e == cudaSuccess)  // a residual is a rate: no shift
            e = fd::launch_from_df64(reinterpret_cast<const fd::df64*>(Rw), out, h->n, fd::Shift5{{0, 0, 0, 0, 0}},
                                     h->stream);
    } else {
        e = run_stage(h, 0, true, out);
    }
    if (e == cudaSuccess && !dst_is_device)
        e = cudaMemcpyAsync(R, h->Qs, n_elems * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "fd_residual");
    return check_kernel_error(h, "fd_residual");
}

int fd_check_finite(fd_handle* h) {
    if (!h) return fail_global(FD_EINVAL, "fd_check_finite: NULL handle");
    int flag = 0;
    const double* Q = h->Q[h->cur];
    cudaError_t e = cudaSuccess;
    if (dw_state(h->dtype)) {
        e = state_to_binary64(h, h->Qs);
        Q = h->Qs;
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream);
    if (e == cudaSuccess) e = fd::launch_check_finite(Q, 5LL * h->n, h->flag, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "fd_check_finite");
    if (int rc = check_kernel_error(h, "fd_check_finite")) return rc;
    if (flag) return h->fail(FD_EUNSTABLE, "state holds NaN or infinity");
    return FD_OK;
}

int fd_slab_create(fd_handle** out, int nx, int ny, int nz_global, int z_first, int nz_local, int ghost, double Re,
                   double Mach, double Pr, double gamma, double dt, int algorithm, int dtype, const fd_alloc* alloc,
                   void* cuda_stream) {
    if (!out) return fail_global(FD_EINVAL, "fd_slab_create: out is NULL");
    *out = nullptr;
    if (dtype != FD_F64 && dtype != FD_F64_DW)
        return fail_global(FD_EINVAL, "fd_slab_create: dtype %d; slabs hold binary64 states (FD_F64, FD_F64_DW)",
                           dtype);
    if (nz_global < 5 || nz_local < 1 || z_first < 0 || z_first >= nz_global || nz_local > nz_global)
        return fail_global(FD_EINVAL, "fd_slab_create: planes %d..%d of %d", z_first, z_first + nz_local - 1,
                           nz_global);
    const int need = fd_slab_ghost_planes(algorithm);
    if (need <= 0) return fail_global(FD_EINVAL, "fd_slab_create: unknown algorithm %d", algorithm);
    if (ghost < need || ghost > nz_global)
        return fail_global(FD_EINVAL, "fd_slab_create: ghost = %d, this family needs %d (and at most nz_global)",
                           ghost, need);
    const long long nz = (long long)nz_local + 2LL * ghost;
    if (nz > fd::kMaxPoints) return fail_global(FD_EINVAL, "fd_slab_create: slab too large");
    int rc = create_impl(out, nx, ny, (int)nz, nz_global, z_first - ghost, Re, Mach, Pr, gamma, dt, algorithm, dtype,
                         alloc, cuda_stream);
    if (rc != FD_OK) return rc;
    fd_handle* h = *out;
    h->slab_ghost = ghost;
    h->slab_nz_local = nz_local;
    h->slab_z_first = z_first;
    h->slab_nz_global = nz_global;
    return FD_OK;
}

int fd_slab_ghost_planes(int algorithm) {
    // A stage's result at plane z reads planes z-2 .. z+2 in every family: the
    // stored gradients (SS, RS) and derivative arrays (BL) at plane z read planes
    // z-2 .. z+2, and a z-difference of stored values only ever takes in-plane
    // derivatives (D_z of D_x u + D_y v; D_x, D_y of D_z w at the same plane).
    // Three stages per step: 3 x 2 planes.
    switch (algorithm) {
        case FD_STORE_ALL:
        case FD_STORE_SOME:
        case FD_RECOMPUTE_ALL:
        case FD_RECOMPUTE_SOME:
        case FD_STORE_NONE:
        case FD_RECOMPUTE_ALL_INLINE:
            return 6;
        default:
            return -1;
    }
}

// Stream-ordered copy of `count` planes starting at plane z of the state to or
// from buf, laid out [5][count][ny][nx] (one 2-D copy: 5 rows of count planes,
// pitch = one variable of the state).
static int planes_copy(fd_handle* h, int z, int count, double* buf, int buf_is_device, bool to_state,
                       const char* what) {
    if (!h) return fail_global(FD_EINVAL, "%s: NULL handle", what);
    if (!buf) return h->fail(FD_EINVAL, "%s: buffer is NULL", what);
    if (h->dtype != FD_F64 && h->dtype != FD_F64_DW)
        return h->fail(FD_EINVAL, "%s: the state is not binary64 (dtype %d)", what, h->dtype);
    if (z < 0 || count < 0 || z + count > h->nz)
        return h->fail(FD_EINVAL, "%s: planes %d..%d outside 0..%d", what, z, z + count - 1, h->nz - 1);
    if (count == 0) return FD_OK;
    const size_t plane = (size_t)h->nx * h->ny;
    double* state = h->Q[h->cur] + (size_t)z * plane;
    const size_t width = (size_t)count * plane * sizeof(double), pitch_state = (size_t)h->n * sizeof(double);
    cudaError_t e;
    if (to_state) {
        h->wvalid = false;  // the working fields of the replaced planes are stale
        e = cudaMemcpy2DAsync(state, pitch_state, buf, width, width, 5,
                              buf_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream);
    } else {
        e = cudaMemcpy2DAsync(buf, width, state, pitch_state, width, 5,
                              buf_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream);
    }
    if (e != cudaSuccess) return h->cuda_fail(e, what);
    return FD_OK;
}

int fd_get_planes_async(fd_handle* h, int z, int count, double* dst, int dst_is_device) {
    return planes_copy(h, z, count, dst, dst_is_device, false, "fd_get_planes_async");
}

int fd_set_planes_async(fd_handle* h, int z, int count, const double* src, int src_is_device) {
    return planes_copy(h, z, count, const_cast<double*>(src), src_is_device, true, "fd_set_planes_async");
}

int fd_selftest_wait_timeout(int* err_word) {
    if (!err_word) return fail_global(FD_EINVAL, "fd_selftest_wait_timeout: err_word is NULL");
    *err_word = 0;
    fd_handle* h = nullptr;
    int rc = fd_create(&h, 32, 8, 8, 1600.0, 0.1, 0.71, 1.4, 1e-3, FD_RECOMPUTE_ALL, FD_F32_ACCDW, nullptr, nullptr);
    if (rc != FD_OK) return rc;
    if (!h->use_tma) {
        fd_destroy(h);
        return fail_global(FD_EINVAL, "fd_selftest_wait_timeout: TMA staging is turned off");
    }
    const fd::df64* Qin = reinterpret_cast<const fd::df64*>(h->Q[h->cur]);
    fd::df64* Qout = reinterpret_cast<fd::df64*>(h->Q[1 - h->cur]);
    cudaError_t e = fd::launch_prims_padded(h->grid, h->phys, Qin, h->Wf[h->wcur], h->stream);
    if (e == cudaSuccess)  // plane 2 of the single z-chunk is never copied
        e = fd::launch_ra_tma(h->fmap[h->wcur], h->grid, h->kf, h->phys, fd::make_stage(0, h->dt), false, Qin, Qout,
                              reinterpret_cast<fd::df64*>(h->Qs), h->Wf[1 - h->wcur], h->kerr, h->stream, 2);
    if (e == cudaSuccess) e = cudaMemcpyAsync(err_word, h->kerr, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    fd_destroy(h);
    if (e != cudaSuccess) return fail_global(FD_ECUDA, "fd_selftest_wait_timeout: %s", cudaGetErrorString(e));
    return FD_OK;
}

size_t fd_device_bytes(const fd_handle* h) { return h ? h->block_bytes : 0; }

int fd_profile(fd_handle* h, int enable) {
    if (!h) return fail_global(FD_EINVAL, "fd_profile: NULL handle");
    cudaError_t e = h->prof.enable(enable != 0, h->stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "fd_profile");
    return FD_OK;
}

int fd_profile_read(fd_handle* h, int kernel_class, double* total_ms, long long* launches) {
    if (!h) return fail_global(FD_EINVAL, "fd_profile_read: NULL handle");
    if (kernel_class < 0 || kernel_class >= FD_KERNEL_CLASSES)
        return h->fail(FD_EINVAL, "fd_profile_read: kernel class %d out of range", kernel_class);
    cudaError_t e = h->prof.fold(h->stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "fd_profile_read");
    if (total_ms) *total_ms = h->prof.total_ms[kernel_class];
    if (launches) *launches = h->prof.count[kernel_class];
    return FD_OK;
}

int fd_destroy(fd_handle* h) {
    if (!h) return FD_OK;
    cudaStreamSynchronize(h->stream);
    h->prof.destroy();
    device_free(h);
    delete h;
    return FD_OK;
}

const char* fd_last_error(const fd_handle* h) { return h ? h->err.c_str() : g_err.c_str(); }

}  // extern "C"
