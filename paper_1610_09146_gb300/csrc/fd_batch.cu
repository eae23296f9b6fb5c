// fd_batch.cu -- many independent Taylor-Green instances advanced together
// (the batched path of include/fdgb300.h).
//
// Device memory (one allocation, 256-byte-aligned pieces):
//   instance table  BatchInst<T>[count]   grid, coefficients, buffer pointers
//   tile lists      BatchTile[...]        one list per family (SS, RA) and one
//                                         over all instances (primitives pass)
//   per instance    Q[2], Qs state (binary64, or shifted double-words in the
//                   binary32 mode), W[2] working fields, G (SS)
//   diagnostics     partial sums and 2 x count results
// A step is three stages; each stage launches, per family present, the
// persistent kernels of fd_kernels.cu (SS: gradients then fused; RA: fused).
// The two families touch disjoint instances, so the captured step graph runs
// them on two branches (fork/join) and their tails overlap.  All instances
// flip their ping-pong parity together, so two graphs exist: one for a step
// that starts at parity 0 and one for parity 1.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/fdgb300.h"
#include "fd_host.h"
#include "fd_internal.h"

namespace {

thread_local std::string g_batch_err;

int fail_global(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_batch_err = buf;
    return code;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

constexpr int kThreads = 256;
constexpr int kDefaultTile = 1024;

struct InstHost {
    fd_instance_desc d;
    int n;
    bool padded;                   // TMA-staged binary32 RA: ghost-padded working fields
    size_t q0, q1, qs, w0, w1, g;  // byte offsets in the allocation
    // FD_F64_DW: w0 / w1 hold the double-word fields F; binary64 u, v, w, p and div u here
    size_t w64_0 = (size_t)-1, w64_1 = (size_t)-1, dv = (size_t)-1, rc = (size_t)-1;
};

// The binary32 mode keeps a double-word state; binary64 and the mixed mode a binary64 one.
bool dw_state(int dtype) { return dtype == FD_F32_ACCDW; }

}  // namespace

struct fd_batch {
    int count = 0, dtype = 0, device = 0;
    cudaStream_t stream = nullptr;
    fd_alloc alloc{};
    bool has_alloc = false;
    void* block = nullptr;
    size_t block_bytes = 0;
    std::vector<InstHost> inst;
    void* d_inst = nullptr;                       // BatchInst<T>[count]
    fd::BatchTile *d_ss = nullptr, *d_ra = nullptr, *d_all = nullptr;
    int n_ss = 0, n_ra = 0, n_all = 0;
    int grid_ss_fused = 0, grid_ra_fused = 0, grid_grad = 0, grid_prims = 0;
    double* partial = nullptr;
    double* diag = nullptr;
    int* kerr = nullptr;  // set by a kernel whose bounded wait ran out
    bool ra_tma = false;  // binary32 RA instances staged by TMA (all of them qualify)
    int tma_zlen = 64;    // planes per TMA work item
    int parity = 0;
    bool wvalid = false;
    cudaStream_t cap[2] = {nullptr, nullptr};      // capture streams
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    fd::Profiler prof;
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
    int cuda_fail(cudaError_t e, const char* what) { return fail(FD_ECUDA, "%s: %s", what, cudaGetErrorString(e)); }
    char* base() const { return static_cast<char*>(block); }
};

namespace {

// binary32 mode: the state holds shifted double-words (rho - 1, rho u_i,
// rho E - rhoE0); a binary64 copy passes through the instance's saved
// register Qs, which is dead between steps (stage 0 rewrites it).
fd::Shift5 state_shift(const InstHost& h) {
    return fd::Shift5{{1.0, 0.0, 0.0, 0.0, fd::make_phys(h.d.Re, h.d.Mach, h.d.Pr, h.d.gamma).rhoE0}};
}

cudaError_t to_binary64(const fd_batch* b, const InstHost& h, double* dst) {
    const char* q = b->base() + (b->parity ? h.q1 : h.q0);
    return fd::launch_from_df64(reinterpret_cast<const fd::df64*>(q), dst, h.n, state_shift(h), b->stream);
}

template <class T>
void fill_inst(const fd_batch* b, std::vector<fd::BatchInst<T>>& out) {
    out.resize(b->count);
    for (int i = 0; i < b->count; ++i) {
        const InstHost& h = b->inst[i];
        fd::BatchInst<T>& I = out[i];
        std::memset(&I, 0, sizeof I);
        I.g = fd::make_grid(h.d.nx, h.d.ny, h.d.nz);
        I.ph = fd::make_phys(h.d.Re, h.d.Mach, h.d.Pr, h.d.gamma);
        I.k = fd::make_coef<T>(I.g, I.ph, sizeof(T) == sizeof(float));
        I.Q[0] = reinterpret_cast<fd::state_t<T>*>(b->base() + h.q0);
        I.Q[1] = reinterpret_cast<fd::state_t<T>*>(b->base() + h.q1);
        I.Qs = reinterpret_cast<fd::state_t<T>*>(b->base() + h.qs);
        I.W[0] = reinterpret_cast<T*>(b->base() + h.w0);
        I.W[1] = reinterpret_cast<T*>(b->base() + h.w1);
        I.G = h.g == (size_t)-1 ? nullptr : reinterpret_cast<T*>(b->base() + h.g);
        I.padded = h.padded ? 1 : 0;
        for (int s = 0; s < 3; ++s) I.rk[s] = fd::make_stage(s, h.d.dt);
    }
}

// Instance records of a mixed (FD_F64_DW) batch.
void fill_hyb(const fd_batch* b, std::vector<fd::BatchHyb>& out) {
    out.resize(b->count);
    for (int i = 0; i < b->count; ++i) {
        const InstHost& h = b->inst[i];
        fd::BatchHyb& I = out[i];
        std::memset(&I, 0, sizeof I);
        I.g = fd::make_grid(h.d.nx, h.d.ny, h.d.nz);
        I.ph = fd::make_phys(h.d.Re, h.d.Mach, h.d.Pr, h.d.gamma);
        I.k = fd::make_coef<fd::df64>(I.g, I.ph, true);
        I.k.c_rho = fd::df64(0.0f, 0.0f);  // the mean-state terms enter in binary64
        I.k.c_E = fd::df64(0.0f, 0.0f);
        I.c_E = -(I.ph.rhoE0 + I.ph.p0);
        for (int s = 0; s < 3; ++s) I.rk[s] = fd::make_stage(s, h.d.dt);
        I.Q[0] = reinterpret_cast<double*>(b->base() + h.q0);
        I.Q[1] = reinterpret_cast<double*>(b->base() + h.q1);
        I.Qs = reinterpret_cast<double*>(b->base() + h.qs);
        I.F[0] = reinterpret_cast<fd::df64*>(b->base() + h.w0);
        I.F[1] = reinterpret_cast<fd::df64*>(b->base() + h.w1);
        I.W64[0] = reinterpret_cast<double*>(b->base() + h.w64_0);
        I.W64[1] = reinterpret_cast<double*>(b->base() + h.w64_1);
        I.G = reinterpret_cast<fd::df64*>(b->base() + h.g);
        I.Dv = reinterpret_cast<double*>(b->base() + h.dv);
        I.Rc = reinterpret_cast<fd::df64*>(b->base() + h.rc);
    }
}

// Tensor maps of the working fields of the TMA-staged binary32 RA instances.
cudaError_t fill_maps(const fd_batch* b, std::vector<fd::BatchInst<float>>& out) {
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < b->count && e == cudaSuccess; ++i)
        if (b->inst[i].padded)
            for (int w = 0; w < 2 && e == cudaSuccess; ++w) e = fd::encode_field_map(&out[i].fmap[w], out[i].W[w], out[i].g);
    return e;
}

// Work items: point ranges of tile_points each, or (tiled) the x-y tile /
// z-chunk pairs of the shared-memory recompute-all kernel, thread-staged or
// (b->ra_tma) TMA-staged.
void make_tiles(const fd_batch* b, int family, bool tiled, std::vector<fd::BatchTile>& out) {
    for (int i = 0; i < b->count; ++i) {
        const InstHost& h = b->inst[i];
        if (family >= 0 && h.d.algorithm != family) continue;
        if (tiled) {
            const int m = b->ra_tma ? fd::tma_work_items(h.d.nx, h.d.ny, h.d.nz, b->tma_zlen)
                                    : fd::tiled_work_items(h.d.nx, h.d.ny, h.d.nz);
            for (int t = 0; t < m; ++t) out.push_back({i, t, 0});
            continue;
        }
        int tp = h.d.tile_points > 0 ? h.d.tile_points : kDefaultTile;
        for (int s = 0; s < h.n; s += tp) out.push_back({i, s, std::min(tp, h.n - s)});
    }
}

// Kernels of stage s at parity p for the instances of one family.
template <class T>
cudaError_t enqueue_family(fd_batch* b, bool ss, int s, int p, cudaStream_t st) {
    auto* I = static_cast<const fd::BatchInst<T>*>(b->d_inst);
    if (ss) {
        if (!b->n_ss) return cudaSuccess;
        cudaError_t e = b->prof.timed(st, FD_KERNEL_GRAD, [&] {
            return fd::launch_batch_grad<T>(I, b->d_ss, b->n_ss, p, b->grid_grad, st);
        });
        if (e != cudaSuccess) return e;
        return b->prof.timed(st, FD_KERNEL_FUSED, [&] {
            return fd::launch_batch_fused<T>(I, b->d_ss, b->n_ss, true, s, p, b->grid_ss_fused, st);
        });
    }
    if (!b->n_ra) return cudaSuccess;
    return b->prof.timed(st, FD_KERNEL_FUSED, [&] {
        if constexpr (sizeof(T) == sizeof(float)) {  // binary32: fields staged through shared memory
            if (b->ra_tma)
                return fd::launch_batch_ra_tma(I, b->d_ra, b->n_ra, s, p, b->grid_ra_fused, b->tma_zlen, b->kerr,
                                               st);
            return fd::launch_batch_ra_tiled<T>(I, b->d_ra, b->n_ra, s, p, b->grid_ra_fused, st);
        }
        return fd::launch_batch_fused<T>(I, b->d_ra, b->n_ra, false, s, p, b->grid_ra_fused, st);
    });
}

// One RK3 step starting at parity p.  With two streams the SS family runs on
// st0 and RA on st1 between a fork and a join; with one stream in sequence.
template <class T>
cudaError_t enqueue_step(fd_batch* b, int p, cudaStream_t st0, cudaStream_t st1) {
    cudaError_t e;
    bool two = st1 != nullptr && b->n_ss && b->n_ra;
    if (two) {
        if ((e = cudaEventRecord(b->fork, st0)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(st1, b->fork, 0)) != cudaSuccess) return e;
    }
    for (int s = 0, q = p; s < 3; ++s, q ^= 1) {
        if ((e = enqueue_family<T>(b, true, s, q, st0)) != cudaSuccess) return e;
        if ((e = enqueue_family<T>(b, false, s, q, two ? st1 : st0)) != cudaSuccess) return e;
    }
    if (two) {
        if ((e = cudaEventRecord(b->join, st1)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(st0, b->join, 0)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Mixed store-some batch (FD_F64_DW): three stages of the two fused kernels
// (the first also forms the gradients).
cudaError_t enqueue_step_hyb(fd_batch* b, int p, cudaStream_t st) {
    auto* I = static_cast<const fd::BatchHyb*>(b->d_inst);
    cudaError_t e;
    for (int s = 0, q = p; s < 3; ++s, q ^= 1) {
        e = b->prof.timed(st, FD_KERNEL_FUSED, [&] {
            return fd::launch_batch_ss_hyb(I, b->d_ss, b->n_ss, s, q, b->grid_ra_fused, b->grid_ss_fused, st);
        });
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t step_direct(fd_batch* b, int p) {
    if (b->dtype == FD_F64_DW) return enqueue_step_hyb(b, p, b->stream);
    return b->dtype == FD_F64 ? enqueue_step<double>(b, p, b->stream, nullptr)
                              : enqueue_step<float>(b, p, b->stream, nullptr);
}

cudaError_t build_graphs(fd_batch* b) {
    cudaError_t e;
    if (!b->cap[0]) {
        for (auto& c : b->cap)
            if ((e = cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming)) != cudaSuccess) return e;
    }
    for (int p = 0; p < 2; ++p) {
        cudaGraph_t g = nullptr;
        if ((e = cudaStreamBeginCapture(b->cap[0], cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
        cudaError_t le = b->dtype == FD_F64_DW ? enqueue_step_hyb(b, p, b->cap[0])
                         : b->dtype == FD_F64  ? enqueue_step<double>(b, p, b->cap[0], b->cap[1])
                                               : enqueue_step<float>(b, p, b->cap[0], b->cap[1]);
        e = cudaStreamEndCapture(b->cap[0], &g);
        if (le == cudaSuccess && e == cudaSuccess) e = cudaGraphInstantiate(&b->exec[p], g, 0);
        if (g) cudaGraphDestroy(g);
        if (le != cudaSuccess) return le;
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

void release(fd_batch* b) {
    if (b->stream || b->block) cudaStreamSynchronize(b->stream);
    for (auto& x : b->exec)
        if (x) cudaGraphExecDestroy(x);
    for (auto& c : b->cap)
        if (c) cudaStreamDestroy(c);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->join) cudaEventDestroy(b->join);
    b->prof.destroy();
    if (b->block) {
        if (b->has_alloc)
            b->alloc.free(b->alloc.ctx, b->block, b->block_bytes, b->stream);
        else
            cudaFree(b->block);
    }
    b->block = nullptr;
}

// A TMA-staged kernel whose bounded wait ran out leaves a nonzero error word;
// the synchronising calls report it.
int check_kernel_error(fd_batch* b, const char* what) {
    if (!b->ra_tma) return FD_OK;
    int v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, b->kerr, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return b->cuda_fail(e, what);
    if (v)
        return b->fail(FD_ECUDA, "%s: %s; the states are not valid", what,
                       v == 2 ? "the TMA ring was not 128-byte aligned" : "a staging wait in a kernel ran out");
    return FD_OK;
}

int ensure_prims(fd_batch* b) {
    if (b->wvalid) return FD_OK;
    cudaError_t e = b->prof.timed(b->stream, FD_KERNEL_PRIMS, [&] {
        if (b->dtype == FD_F64_DW)
            return fd::launch_batch_prims_hyb(static_cast<const fd::BatchHyb*>(b->d_inst), b->d_all, b->n_all,
                                              b->parity, b->grid_prims, b->stream);
        if (b->dtype == FD_F64)
            return fd::launch_batch_prims<double>(static_cast<const fd::BatchInst<double>*>(b->d_inst), b->d_all,
                                                  b->n_all, b->parity, b->grid_prims, b->stream);
        return fd::launch_batch_prims<float>(static_cast<const fd::BatchInst<float>*>(b->d_inst), b->d_all,
                                             b->n_all, b->parity, b->grid_prims, b->stream);
    });
    if (e != cudaSuccess) return b->cuda_fail(e, "fd_batch: primitives");
    b->wvalid = true;
    return FD_OK;
}

template <class T>
int grid_for(int sms, bool fused, bool stored_g) {
    return sms * fd::batch_blocks_per_sm<T>(fused, stored_g);
}

}  // namespace

extern "C" {

int fd_batch_create(fd_batch** out, const fd_instance_desc* desc, int count, int dtype, const fd_alloc* alloc,
                    void* cuda_stream) {
    if (!out) return fail_global(FD_EINVAL, "fd_batch_create: out is NULL");
    *out = nullptr;
    if (!desc || count < 1) return fail_global(FD_EINVAL, "fd_batch_create: need count >= 1 descriptors");
    if (dtype != FD_F64 && dtype != FD_F32_ACCDW && dtype != FD_F64_DW)
        return fail_global(FD_EINVAL, "fd_batch_create: dtype %d", dtype);
    if (alloc && (!alloc->alloc || !alloc->free))
        return fail_global(FD_EINVAL, "fd_batch_create: allocator needs both alloc and free");
    for (int i = 0; i < count; ++i) {
        const fd_instance_desc& d = desc[i];
        if (const char* why = fd::check_instance(d.nx, d.ny, d.nz, d.Re, d.Mach, d.Pr, d.gamma, d.dt))
            return fail_global(FD_EINVAL, "fd_batch_create: instance %d: %s", i, why);
        if (d.algorithm != FD_STORE_SOME && d.algorithm != FD_RECOMPUTE_ALL)
            return fail_global(FD_EINVAL, "fd_batch_create: instance %d: algorithm %d is not batched", i, d.algorithm);
        if (d.tile_points != 0 && d.tile_points < 32)
            return fail_global(FD_EINVAL, "fd_batch_create: instance %d: tile_points %d < 32", i, d.tile_points);
        if (dtype == FD_F64_DW && d.algorithm != FD_STORE_SOME)
            return fail_global(FD_EINVAL, "fd_batch_create: instance %d: FD_F64_DW batches are store-some only", i);
    }
    fd_batch* b = new (std::nothrow) fd_batch();
    if (!b) return fail_global(FD_ENOMEM, "fd_batch_create: host allocation failed");
    b->count = count;
    b->dtype = dtype;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    if (dtype == FD_F32_ACCDW) {  // TMA staging when every RA instance allows it
        const char* off_env = std::getenv("FDGB300_NO_TMA");
        b->ra_tma = !(off_env && off_env[0] == '1');
        for (int i = 0; i < count; ++i)
            if (desc[i].algorithm == FD_RECOMPUTE_ALL &&
                !fd::tma_staging_ok(fd::make_grid(desc[i].nx, desc[i].ny, desc[i].nz)))
                b->ra_tma = false;
        if (b->ra_tma) {  // work-item length for the persistent grid (two blocks per SM)
            std::vector<int> dims;
            for (int i = 0; i < count; ++i)
                if (desc[i].algorithm == FD_RECOMPUTE_ALL) dims.insert(dims.end(), {desc[i].nx, desc[i].ny, desc[i].nz});
            int dev = 0, sms = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            b->tma_zlen = fd::tma_batch_zchunk(dims.data(), (int)dims.size() / 3, 2 * (sms > 0 ? sms : 152));
        }
    }
    cudaError_t e = cudaGetDevice(&b->device);
    if (e != cudaSuccess) {
        delete b;
        return fail_global(FD_ECUDA, "fd_batch_create: cudaGetDevice: %s", cudaGetErrorString(e));
    }
    const bool hyb = dtype == FD_F64_DW;
    const size_t tsize = dtype == FD_F64 ? sizeof(double) : (hyb ? sizeof(fd::df64) : sizeof(float));
    const size_t wfields = dtype == FD_F64 ? 5 : 10;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off += align256(bytes);
        return at;
    };
    const size_t inst_bytes = hyb                 ? sizeof(fd::BatchHyb)
                              : dtype == FD_F64 ? sizeof(fd::BatchInst<double>)
                                                : sizeof(fd::BatchInst<float>);
    size_t o_inst = take(inst_bytes * count);
    b->inst.resize(count);
    for (int i = 0; i < count; ++i) {
        InstHost& h = b->inst[i];
        h.d = desc[i];
        h.n = desc[i].nx * desc[i].ny * desc[i].nz;
        size_t f5 = 5 * (size_t)h.n * sizeof(double);
        h.q0 = take(f5);
        h.q1 = take(f5);
        h.qs = take(f5);
        h.padded = b->ra_tma && desc[i].algorithm == FD_RECOMPUTE_ALL;
        const size_t wpts = h.padded ? fd::padded_field_points(fd::make_grid(h.d.nx, h.d.ny, h.d.nz)) : (size_t)h.n;
        h.w0 = take(wfields * wpts * tsize);
        h.w1 = take(wfields * wpts * tsize);
        const size_t garrays = dtype == FD_F64 ? fd::kGradArrays<double>
                               : hyb           ? (size_t)fd::kHybGradArrays
                                               : fd::kGradArrays<float>;
        h.g = desc[i].algorithm == FD_STORE_SOME ? take(garrays * (size_t)h.n * tsize) : (size_t)-1;
        if (hyb) {
            h.w64_0 = take(3 * (size_t)h.n * sizeof(double));
            h.w64_1 = take(3 * (size_t)h.n * sizeof(double));
            h.dv = take((size_t)h.n * sizeof(double));
            h.rc = take(5 * (size_t)h.n * sizeof(fd::df64));
        }
    }
    std::vector<fd::BatchTile> t_ss, t_ra, t_all;
    make_tiles(b, FD_STORE_SOME, false, t_ss);
    make_tiles(b, FD_RECOMPUTE_ALL, dtype == FD_F32_ACCDW, t_ra);
    make_tiles(b, -1, false, t_all);
    size_t o_ss = take(std::max<size_t>(1, t_ss.size()) * sizeof(fd::BatchTile));
    size_t o_ra = take(std::max<size_t>(1, t_ra.size()) * sizeof(fd::BatchTile));
    size_t o_all = take(t_all.size() * sizeof(fd::BatchTile));
    size_t o_part = take(2 * fd::kDiagBlocks * sizeof(double));
    size_t o_diag = take(2 * (size_t)count * sizeof(double));
    size_t o_err = take(sizeof(int));
    b->block_bytes = off;
    if (alloc) {
        b->alloc = *alloc;
        b->has_alloc = true;
        b->block = alloc->alloc(alloc->ctx, off, cuda_stream);
        if (!b->block) {
            delete b;
            return fail_global(FD_ENOMEM, "fd_batch_create: allocator returned NULL for %zu bytes", off);
        }
    } else if ((e = cudaMalloc(&b->block, off)) != cudaSuccess) {
        cudaGetLastError();
        b->block = nullptr;
        delete b;
        return fail_global(FD_ENOMEM, "fd_batch_create: cudaMalloc(%zu): %s", off, cudaGetErrorString(e));
    }
    b->d_inst = b->base() + o_inst;
    b->d_ss = reinterpret_cast<fd::BatchTile*>(b->base() + o_ss);
    b->d_ra = reinterpret_cast<fd::BatchTile*>(b->base() + o_ra);
    b->d_all = reinterpret_cast<fd::BatchTile*>(b->base() + o_all);
    b->n_ss = (int)t_ss.size();
    b->n_ra = (int)t_ra.size();
    b->n_all = (int)t_all.size();
    b->partial = reinterpret_cast<double*>(b->base() + o_part);
    b->diag = reinterpret_cast<double*>(b->base() + o_diag);
    b->kerr = reinterpret_cast<int*>(b->base() + o_err);

    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    if (sms <= 0) sms = 152;
    if (hyb) {  // (the RA slot holds the grid of the first fused kernel: a mixed batch has no RA)
        b->grid_ss_fused = sms * fd::batch_hyb_blocks_per_sm(1);
        b->grid_ra_fused = sms * fd::batch_hyb_blocks_per_sm(2);
        b->grid_grad = b->grid_ss_fused;  // (no gradient pass of its own)
    } else if (dtype == FD_F64) {
        b->grid_ss_fused = grid_for<double>(sms, true, true);
        b->grid_ra_fused = grid_for<double>(sms, true, false);
        b->grid_grad = grid_for<double>(sms, false, false);
    } else {
        b->grid_ss_fused = grid_for<float>(sms, true, true);
        if (b->ra_tma) {
            e = fd::prepare_ra_tma();
            b->grid_ra_fused = sms * fd::batch_tma_blocks_per_sm();  // 115 KB ring per block
        } else {
            b->grid_ra_fused = sms * fd::batch_tiled_blocks_per_sm<float>();
        }
        b->grid_grad = grid_for<float>(sms, false, false);
    }
    b->grid_prims = hyb ? sms * fd::batch_hyb_blocks_per_sm(0) : b->grid_grad;

    // Instance table and tile lists (host staging is pageable; copies complete
    // before the synchronisation below).
    if (hyb) {
        std::vector<fd::BatchHyb> I;
        fill_hyb(b, I);
        e = cudaMemcpyAsync(b->d_inst, I.data(), I.size() * sizeof I[0], cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    } else if (dtype == FD_F64) {
        std::vector<fd::BatchInst<double>> I;
        fill_inst<double>(b, I);
        e = cudaMemcpyAsync(b->d_inst, I.data(), I.size() * sizeof I[0], cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    } else {
        std::vector<fd::BatchInst<float>> I;
        fill_inst<float>(b, I);
        if (e == cudaSuccess) e = fill_maps(b, I);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->d_inst, I.data(), I.size() * sizeof I[0], cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    }
    auto up = [&](fd::BatchTile* dst, const std::vector<fd::BatchTile>& v) {
        if (v.empty() || e != cudaSuccess) return;
        e = cudaMemcpyAsync(dst, v.data(), v.size() * sizeof v[0], cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    };
    up(b->d_ss, t_ss);
    up(b->d_ra, t_ra);
    up(b->d_all, t_all);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->kerr, 0, sizeof(int), b->stream);
    // padded working fields: the padding columns no point writes are copied but never read
    for (int i = 0; i < count && e == cudaSuccess; ++i) {
        const InstHost& h = b->inst[i];
        if (!h.padded) continue;
        const size_t bytes = 10 * fd::padded_field_points(fd::make_grid(h.d.nx, h.d.ny, h.d.nz)) * sizeof(float);
        e = cudaMemsetAsync(b->base() + h.w0, 0, bytes, b->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->base() + h.w1, 0, bytes, b->stream);
    }
    // Taylor-Green initial state of every instance (Section 3).
    for (int i = 0; i < count && e == cudaSuccess; ++i) {
        const InstHost& h = b->inst[i];
        fd::Grid g = fd::make_grid(h.d.nx, h.d.ny, h.d.nz);
        fd::Phys ph = fd::make_phys(h.d.Re, h.d.Mach, h.d.Pr, h.d.gamma);
        double* ic = reinterpret_cast<double*>(b->base() + (dw_state(dtype) ? h.qs : h.q0));
        e = fd::launch_tgv_ic(g, ph, 2.0 * fd::kPi / h.d.nx, 2.0 * fd::kPi / h.d.ny, 2.0 * fd::kPi / h.d.nz, ic,
                              b->stream);
        if (e == cudaSuccess && dw_state(dtype))
            e = fd::launch_to_df64(ic, reinterpret_cast<fd::df64*>(b->base() + h.q0), h.n, state_shift(h), b->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        release(b);
        delete b;
        return fail_global(FD_ECUDA, "fd_batch_create: set-up: %s", cudaGetErrorString(e));
    }
    *out = b;
    return FD_OK;
}

int fd_batch_step(fd_batch* b, int n) {
    if (!b) return fail_global(FD_EINVAL, "fd_batch_step: NULL batch");
    if (n < 0) return b->fail(FD_EINVAL, "fd_batch_step: n = %d < 0", n);
    if (n == 0) return FD_OK;
    int rc = ensure_prims(b);
    if (rc != FD_OK) return rc;
    cudaError_t e;
    if (b->prof.on) {
        for (int it = 0; it < n; ++it) {
            if ((e = step_direct(b, b->parity)) != cudaSuccess) return b->cuda_fail(e, "fd_batch_step");
            b->parity ^= 1;
        }
        return FD_OK;
    }
    if (!b->exec[0] && (e = build_graphs(b)) != cudaSuccess) return b->cuda_fail(e, "fd_batch_step: graph capture");
    for (int it = 0; it < n; ++it) {
        if ((e = cudaGraphLaunch(b->exec[b->parity], b->stream)) != cudaSuccess)
            return b->cuda_fail(e, "fd_batch_step: graph launch");
        b->parity ^= 1;
    }
    return FD_OK;
}

int fd_batch_get_state(fd_batch* b, int i, double* dst, size_t n_elems, int dst_is_device) {
    if (!b) return fail_global(FD_EINVAL, "fd_batch_get_state: NULL batch");
    if (i < 0 || i >= b->count) return b->fail(FD_EINVAL, "fd_batch_get_state: instance %d out of range", i);
    if (!dst) return b->fail(FD_EINVAL, "fd_batch_get_state: dst is NULL");
    const InstHost& h = b->inst[i];
    if (n_elems != 5 * (size_t)h.n)
        return b->fail(FD_EINVAL, "fd_batch_get_state: n_elems = %zu, expected %zu", n_elems, 5 * (size_t)h.n);
    const char* src = b->base() + (b->parity ? h.q1 : h.q0);
    cudaError_t e = cudaSuccess;
    if (dw_state(b->dtype)) {
        double* tmp = dst_is_device ? dst : reinterpret_cast<double*>(b->base() + h.qs);
        e = to_binary64(b, h, tmp);
        src = reinterpret_cast<const char*>(tmp);
    }
    if (e == cudaSuccess && src != reinterpret_cast<const char*>(dst))
        e = cudaMemcpyAsync(dst, src, n_elems * sizeof(double),
                            dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return b->cuda_fail(e, "fd_batch_get_state");
    return check_kernel_error(b, "fd_batch_get_state");
}

int fd_batch_set_state(fd_batch* b, int i, const double* src, size_t n_elems, int src_is_device) {
    if (!b) return fail_global(FD_EINVAL, "fd_batch_set_state: NULL batch");
    if (i < 0 || i >= b->count) return b->fail(FD_EINVAL, "fd_batch_set_state: instance %d out of range", i);
    if (!src) return b->fail(FD_EINVAL, "fd_batch_set_state: src is NULL");
    const InstHost& h = b->inst[i];
    if (n_elems != 5 * (size_t)h.n)
        return b->fail(FD_EINVAL, "fd_batch_set_state: n_elems = %zu, expected %zu", n_elems, 5 * (size_t)h.n);
    b->wvalid = false;
    char* q = b->base() + (b->parity ? h.q1 : h.q0);
    char* dst = dw_state(b->dtype) ? b->base() + h.qs : q;
    cudaError_t e = cudaMemcpyAsync(dst, src, n_elems * sizeof(double),
                                    src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && dw_state(b->dtype))
        e = fd::launch_to_df64(reinterpret_cast<const double*>(dst), reinterpret_cast<fd::df64*>(q), h.n,
                               state_shift(h), b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return b->cuda_fail(e, "fd_batch_set_state");
    return FD_OK;
}

int fd_batch_diagnostics(fd_batch* b, double* ke, double* enstrophy) {
    if (!b) return fail_global(FD_EINVAL, "fd_batch_diagnostics: NULL batch");
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < b->count && e == cudaSuccess; ++i) {
        const InstHost& h = b->inst[i];
        fd::Grid g = fd::make_grid(h.d.nx, h.d.ny, h.d.nz);
        const double* Q = reinterpret_cast<const double*>(b->base() + (b->parity ? h.q1 : h.q0));
        if (dw_state(b->dtype)) {
            double* tmp = reinterpret_cast<double*>(b->base() + h.qs);
            e = to_binary64(b, h, tmp);
            Q = tmp;
        }
        // Scratch for the velocities: the working-field buffer the next stage
        // overwrites (at least 3 x n doubles in either precision).
        double* Wv = reinterpret_cast<double*>(b->base() + (b->parity ? h.w0 : h.w1));
        if (e == cudaSuccess) e = fd::launch_diagnostics_f64(g, Q, Wv, b->partial, b->diag + 2 * i, b->stream);
    }
    std::vector<double> out(2 * (size_t)b->count);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out.data(), b->diag, out.size() * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return b->cuda_fail(e, "fd_batch_diagnostics");
    if (int rc = check_kernel_error(b, "fd_batch_diagnostics")) return rc;
    for (int i = 0; i < b->count; ++i) {
        if (ke) ke[i] = out[2 * i];
        if (enstrophy) enstrophy[i] = out[2 * i + 1];
    }
    return FD_OK;
}

int fd_batch_count(const fd_batch* b) { return b ? b->count : 0; }

size_t fd_batch_device_bytes(const fd_batch* b) { return b ? b->block_bytes : 0; }

int fd_batch_profile(fd_batch* b, int enable) {
    if (!b) return fail_global(FD_EINVAL, "fd_batch_profile: NULL batch");
    cudaError_t e = b->prof.enable(enable != 0, b->stream);
    if (e != cudaSuccess) return b->cuda_fail(e, "fd_batch_profile");
    return FD_OK;
}

int fd_batch_profile_read(fd_batch* b, int kernel_class, double* total_ms, long long* launches) {
    if (!b) return fail_global(FD_EINVAL, "fd_batch_profile_read: NULL batch");
    if (kernel_class < 0 || kernel_class >= FD_KERNEL_CLASSES)
        return b->fail(FD_EINVAL, "fd_batch_profile_read: kernel class %d out of range", kernel_class);
    cudaError_t e = b->prof.fold(b->stream);
    if (e != cudaSuccess) return b->cuda_fail(e, "fd_batch_profile_read");
    if (total_ms) *total_ms = b->prof.total_ms[kernel_class];
    if (launches) *launches = b->prof.count[kernel_class];
    return FD_OK;
}

int fd_batch_destroy(fd_batch* b) {
    if (!b) return FD_OK;
    release(b);
    delete b;
    return FD_OK;
}

const char* fd_batch_last_error(const fd_batch* b) { return b ? b->err.c_str() : g_batch_err.c_str(); }

}  // extern "C"
