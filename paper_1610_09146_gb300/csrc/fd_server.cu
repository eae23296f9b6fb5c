// fd_server.cu -- continuous-batching server for Taylor-Green solves (the
// serving path of include/fdgb300.h).
//
// Memory: one device arena, sized at creation, split by a first-fit
// free-list allocator with coalescing; an admitted solve takes one block for
// its Q[2], Qs, W[2] (and G for store-some), laid out as in a batch.  The
// instance tables and tile lists live in separate device buffers that grow
// geometrically.
//
// Scheduling: FIFO queue, first-fit admission by footprint and a cap on
// active solves.  All active solves share one ping-pong parity: a newly
// admitted solve writes its initial state into Q[parity], so every tick runs
// one RK3 step of every active solve with the batched kernels, one group per
// (dtype, family).  One tick stays in flight: a tick enqueues its work and
// the diagnostics of the solves it finishes, then waits for the previous
// tick's work only, and retires that tick's finished solves, so the device
// runs tick k while the host plans tick k+1 (a tick that leaves no solve
// active waits for its own work and retires at once).  A retired solve's
// state stays readable (fd_server_get_state) until the first tick after its
// result was polled, which returns its memory to the arena.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/fdgb300.h"
#include "fd_host.h"
#include "fd_internal.h"

namespace {

thread_local std::string g_server_err;

int fail_global(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_server_err = buf;
    return code;
}

constexpr size_t kAlign = 256;
constexpr int kDefaultTile = 1024;
size_t align256(size_t b) { return (b + kAlign - 1) & ~(kAlign - 1); }

// First-fit allocator over [0, capacity) with coalescing of free neighbours.
class Arena {
   public:
    explicit Arena(size_t cap = 0) : cap_(cap) {
        if (cap) free_[0] = cap;
    }
    bool alloc(size_t bytes, size_t* off) {
        bytes = align256(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                size_t rest = it->second - bytes, at = it->first + bytes;
                free_.erase(it);
                if (rest) free_[at] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = align256(bytes);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }
    size_t capacity() const { return cap_; }

   private:
    size_t cap_ = 0, used_ = 0;
    std::map<size_t, size_t> free_;  // offset -> size
};

struct Layout {
    size_t q0, q1, qs, w0, w1, g, total;
    bool padded;  // binary32 RA staged by TMA: ghost-padded working fields
    // FD_F64_DW: w0 / w1 hold the double-word fields; binary64 u, v, w, p and div u here
    size_t w64_0 = (size_t)-1, w64_1 = (size_t)-1, dv = (size_t)-1, rc = (size_t)-1;
};

// Instance group of a request: 0 binary64, 1 binary32, 2 mixed binary64 / double-word.
int group_of(int dtype) { return dtype == FD_F64 ? 0 : (dtype == FD_F32_ACCDW ? 1 : 2); }

// tma: whether TMA staging may be used (a binary32 RA solve on a grid that
// allows it then gets the ghost-padded working-field layout, a little larger).
Layout layout_of(const fd_request& r, bool tma) {
    const size_t n = (size_t)r.nx * r.ny * r.nz;
    const bool hyb = r.dtype == FD_F64_DW;
    const size_t t = r.dtype == FD_F64 ? sizeof(double) : (hyb ? sizeof(fd::df64) : sizeof(float));
    const size_t wf = r.dtype == FD_F64 ? 5 : 10;
    Layout L{};
    const fd::Grid g = fd::make_grid(r.nx, r.ny, r.nz);
    L.padded = tma && r.dtype == FD_F32_ACCDW && r.algorithm == FD_RECOMPUTE_ALL && fd::tma_staging_ok(g);
    const size_t wpts = L.padded ? fd::padded_field_points(g) : n;
    size_t off = 0;
    auto take = [&](size_t b) {
        size_t at = off;
        off += align256(b);
        return at;
    };
    L.q0 = take(5 * n * sizeof(double));
    L.q1 = take(5 * n * sizeof(double));
    L.qs = take(5 * n * sizeof(double));
    L.w0 = take(wf * wpts * t);
    L.w1 = take(wf * wpts * t);
    const size_t garrays = r.dtype == FD_F64 ? fd::kGradArrays<double>
                           : hyb             ? (size_t)fd::kHybGradArrays
                                             : fd::kGradArrays<float>;
    L.g = r.algorithm == FD_STORE_SOME ? take(garrays * n * t) : (size_t)-1;
    if (hyb) {
        L.w64_0 = take(3 * n * sizeof(double));
        L.w64_1 = take(3 * n * sizeof(double));
        L.dv = take(n * sizeof(double));
        L.rc = take(5 * n * sizeof(fd::df64));
    }
    L.total = off;
    return L;
}

const char* check_request(const fd_request* r) {
    if (!r) return "request is NULL";
    if (const char* why = fd::check_instance(r->nx, r->ny, r->nz, r->Re, r->Mach, r->Pr, r->gamma, r->dt)) return why;
    if (r->steps < 1) return "steps must be >= 1";
    if (r->dtype != FD_F64 && r->dtype != FD_F32_ACCDW && r->dtype != FD_F64_DW) return "unknown dtype";
    if (r->algorithm != FD_STORE_SOME && r->algorithm != FD_RECOMPUTE_ALL) return "algorithm must be SS or RA";
    if (r->dtype == FD_F64_DW && r->algorithm != FD_STORE_SOME) return "FD_F64_DW requests are store-some only";
    if (r->tile_points != 0 && r->tile_points < 32) return "tile_points must be 0 or >= 32";
    return nullptr;
}

struct Active {
    fd_request r;
    Layout L;
    size_t off;  // arena offset of the block
    int n;
    int done = 0;
    bool fresh = true;  // initial state written this tick, primitives pending
    bool cancelled = false;
    int slot = -1;      // index in its dtype's instance table
    int k = 1;          // steps per tick (odd; see plan_steps)
};

// A finished solve: its arena block (and so its final state, in Q[parity])
// is kept for fd_server_get_state until the first tick after its result was
// polled.
struct Finished {
    fd_request r;
    Layout L;
    size_t off;
    int n;
    int parity;
    bool polled = false;
    int done = 0;  // steps taken
};

// The solves one tick finished, waiting for that tick's work: the event
// recorded after it, and the host slot its diagnostics and the staging-error
// word are copied to (pinned; two slots, as two ticks can be outstanding).
struct Pending {
    std::vector<Finished> solves;
    cudaEvent_t ev = nullptr;
    double* host_res = nullptr;  // 2 per solve: KE, enstrophy
    int* host_err = nullptr;
    bool armed = false, check_err = false;
    long long tick = 0;
};

// Time slicing.  A tick advances every active solve by an odd number of steps
// k: the dearest step of the active set gets one, and a cheaper solve gets as
// many as fit in that step's time (at most kMaxSteps, never past its request),
// so a small solve is not held to the pace of the largest one.  Odd counts
// flip every solve's ping-pong parity once per tick, so all solves keep one
// parity; round r of a tick advances the solves with k > r, which are a prefix
// of tile lists ordered by k.  Step costs are estimated from the measured
// rates of the two precisions (binary64 ~6e8, binary32 ~6e9 point-steps/s).
constexpr int kMaxSteps = 31;

double step_cost(const fd_request& r) {
    const double per_point = r.dtype == FD_F64 ? 1.7e-9 : (r.dtype == FD_F64_DW ? 7.0e-10 : 1.6e-10);
    return (double)r.nx * r.ny * r.nz * per_point;
}

}  // namespace

struct fd_server {
    cudaStream_t stream = nullptr;
    fd_alloc alloc{};
    bool has_alloc = false;
    int device = 0, max_active = 0, sms = 152;
    void* arena_ptr = nullptr;
    Arena arena;
    // small fixed buffers: diagnostics partial sums and per-slot results
    void* fixed = nullptr;
    size_t fixed_bytes = 0;
    double* partial = nullptr;
    double* results = nullptr;  // 2 * max_active
    int* kerr = nullptr;        // set by a kernel whose bounded wait ran out
    bool tma_allowed = true;    // FDGB300_NO_TMA=1 at creation turns TMA staging off
    int tma_blocks = 1;         // resident TMA-staged blocks per SM
    int tma_zlen = 64;          // planes per TMA work item (set by rebuild)
    // growable buffers for tables and tiles
    void* tab = nullptr;
    size_t tab_bytes = 0;
    std::deque<fd_request> queue;
    std::vector<Active> active;
    std::vector<fd_result> done;
    std::vector<Finished> finished;  // retired solves whose state is still kept
    Pending pending[2];              // by tick parity: finished, not yet retired
    void* host_pinned = nullptr;     // both slots' results and error words
    bool dirty = true;
    int parity = 0;
    long long submitted = 0, completed = 0, ticks = 0;
    // current device views (valid after a rebuild)
    void* inst[3] = {nullptr, nullptr, nullptr};  // tables of the groups: binary64, binary32, mixed
    // [group][family: 0 SS, 1 RA, 2 RA staged by TMA (binary32, padded layout)], ordered by k
    fd::BatchTile* tiles[3][3] = {};
    // ntiles[d][f][r]: tiles of the solves with k > r (a prefix of tiles[d][f])
    int ntiles[3][3][kMaxSteps] = {};
    int rounds = 1;  // max k over the active set
    fd::BatchTile* fresh_tiles[3] = {nullptr, nullptr, nullptr};
    int nfresh[3] = {0, 0, 0};
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
    char* base() const { return static_cast<char*>(arena_ptr); }

    void* dev_alloc(size_t bytes) {
        if (has_alloc) return alloc.alloc(alloc.ctx, bytes, stream);
        void* p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return p;
    }
    void dev_free(void* p, size_t bytes) {
        if (!p) return;
        if (has_alloc)
            alloc.free(alloc.ctx, p, bytes, stream);
        else
            cudaFree(p);
    }
};

namespace {

template <class T>
fd::BatchInst<T> record(const fd_server* s, const Active& a) {
    fd::BatchInst<T> I;
    std::memset(&I, 0, sizeof I);
    I.g = fd::make_grid(a.r.nx, a.r.ny, a.r.nz);
    I.ph = fd::make_phys(a.r.Re, a.r.Mach, a.r.Pr, a.r.gamma);
    I.k = fd::make_coef<T>(I.g, I.ph, sizeof(T) == sizeof(float));
    char* b = s->base() + a.off;
    I.Q[0] = reinterpret_cast<fd::state_t<T>*>(b + a.L.q0);
    I.Q[1] = reinterpret_cast<fd::state_t<T>*>(b + a.L.q1);
    I.Qs = reinterpret_cast<fd::state_t<T>*>(b + a.L.qs);
    I.W[0] = reinterpret_cast<T*>(b + a.L.w0);
    I.W[1] = reinterpret_cast<T*>(b + a.L.w1);
    I.G = a.L.g == (size_t)-1 ? nullptr : reinterpret_cast<T*>(b + a.L.g);
    I.padded = a.L.padded ? 1 : 0;
    for (int st = 0; st < 3; ++st) I.rk[st] = fd::make_stage(st, a.r.dt);
    return I;
}

fd::BatchHyb record_hyb(const fd_server* s, const Active& a) {
    fd::BatchHyb I;
    std::memset(&I, 0, sizeof I);
    I.g = fd::make_grid(a.r.nx, a.r.ny, a.r.nz);
    I.ph = fd::make_phys(a.r.Re, a.r.Mach, a.r.Pr, a.r.gamma);
    I.k = fd::make_coef<fd::df64>(I.g, I.ph, true);
    I.k.c_rho = fd::df64(0.0f, 0.0f);  // the mean-state terms enter in binary64
    I.k.c_E = fd::df64(0.0f, 0.0f);
    I.c_E = -(I.ph.rhoE0 + I.ph.p0);
    for (int st = 0; st < 3; ++st) I.rk[st] = fd::make_stage(st, a.r.dt);
    char* b = s->base() + a.off;
    I.Q[0] = reinterpret_cast<double*>(b + a.L.q0);
    I.Q[1] = reinterpret_cast<double*>(b + a.L.q1);
    I.Qs = reinterpret_cast<double*>(b + a.L.qs);
    I.F[0] = reinterpret_cast<fd::df64*>(b + a.L.w0);
    I.F[1] = reinterpret_cast<fd::df64*>(b + a.L.w1);
    I.W64[0] = reinterpret_cast<double*>(b + a.L.w64_0);
    I.W64[1] = reinterpret_cast<double*>(b + a.L.w64_1);
    I.G = reinterpret_cast<fd::df64*>(b + a.L.g);
    I.Dv = reinterpret_cast<double*>(b + a.L.dv);
    I.Rc = reinterpret_cast<fd::df64*>(b + a.L.rc);
    return I;
}

void append_tiles(const Active& a, std::vector<fd::BatchTile>& v, bool tiled = false, int tma_zlen = 0) {
    if (tiled) {  // x-y tile / z-chunk work items of the shared-memory recompute-all kernel
        const int m = tma_zlen ? fd::tma_work_items(a.r.nx, a.r.ny, a.r.nz, tma_zlen)
                               : fd::tiled_work_items(a.r.nx, a.r.ny, a.r.nz);
        for (int t = 0; t < m; ++t) v.push_back({a.slot, t, 0});
        return;
    }
    int tp = a.r.tile_points > 0 ? a.r.tile_points : kDefaultTile;
    for (int st = 0; st < a.n; st += tp) v.push_back({a.slot, st, std::min(tp, a.n - st)});
}

// Rebuild the instance tables and tile lists of the active set and upload
// them (stream-ordered after every earlier launch that reads them).
cudaError_t rebuild(fd_server* s) {
    std::vector<fd::BatchInst<double>> I64;
    std::vector<fd::BatchInst<float>> I32;
    std::vector<fd::BatchHyb> IH;
    std::vector<fd::BatchTile> t[3][3], f[3];
    cudaError_t e;
    {  // work-item length of the TMA-staged solves for this active set
        std::vector<int> dims;
        for (auto& a : s->active)
            if (a.L.padded) dims.insert(dims.end(), {a.r.nx, a.r.ny, a.r.nz});
        s->tma_zlen = fd::tma_batch_zchunk(dims.data(), (int)dims.size() / 3, s->sms * s->tma_blocks);
    }
    // tiles in order of decreasing k, so that the solves a round advances are a prefix
    std::vector<Active*> order;
    for (auto& a : s->active) order.push_back(&a);
    std::stable_sort(order.begin(), order.end(), [](const Active* x, const Active* y) { return x->k > y->k; });
    int count[3][3][kMaxSteps] = {};
    s->rounds = 1;
    for (Active* ap : order) {
        Active& a = *ap;
        const int d = group_of(a.r.dtype);
        if (d == 0) {
            a.slot = (int)I64.size();
            I64.push_back(record<double>(s, a));
        } else if (d == 2) {
            a.slot = (int)IH.size();
            IH.push_back(record_hyb(s, a));
        } else {
            a.slot = (int)I32.size();
            I32.push_back(record<float>(s, a));
            if (a.L.padded)
                for (int w = 0; w < 2; ++w)
                    if ((e = fd::encode_field_map(&I32.back().fmap[w], I32.back().W[w], I32.back().g)) != cudaSuccess)
                        return e;
        }
        const bool ss = a.r.algorithm == FD_STORE_SOME;
        const int fam = ss ? 0 : (a.L.padded ? 2 : 1);
        append_tiles(a, t[d][fam], !ss && d == 1, a.L.padded ? s->tma_zlen : 0);
        for (int r = 0; r < a.k; ++r) count[d][fam][r] = (int)t[d][fam].size();
        s->rounds = std::max(s->rounds, a.k);
        if (a.fresh) append_tiles(a, f[d]);
    }
    size_t off = 0;
    auto take = [&](size_t b) {
        size_t at = off;
        off += align256(std::max<size_t>(b, 1));
        return at;
    };
    size_t o64 = take(I64.size() * sizeof(fd::BatchInst<double>));
    size_t o32 = take(I32.size() * sizeof(fd::BatchInst<float>));
    size_t oh = take(IH.size() * sizeof(fd::BatchHyb));
    size_t ot[3][3], of[3];
    for (int d = 0; d < 3; ++d) {
        for (int k = 0; k < 3; ++k) ot[d][k] = take(t[d][k].size() * sizeof(fd::BatchTile));
        of[d] = take(f[d].size() * sizeof(fd::BatchTile));
    }
    if (off > s->tab_bytes) {
        if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess) return e;
        s->dev_free(s->tab, s->tab_bytes);
        size_t nb = std::max(off, 2 * s->tab_bytes);
        s->tab = s->dev_alloc(nb);
        s->tab_bytes = s->tab ? nb : 0;
        if (!s->tab) return cudaErrorMemoryAllocation;
    }
    char* b = static_cast<char*>(s->tab);
    auto up = [&](size_t at, const void* src, size_t bytes) {
        if (!bytes) return cudaSuccess;
        return cudaMemcpyAsync(b + at, src, bytes, cudaMemcpyHostToDevice, s->stream);
    };
    if ((e = up(o64, I64.data(), I64.size() * sizeof I64[0])) != cudaSuccess) return e;
    if ((e = up(o32, I32.data(), I32.size() * sizeof I32[0])) != cudaSuccess) return e;
    if ((e = up(oh, IH.data(), IH.size() * sizeof(fd::BatchHyb))) != cudaSuccess) return e;
    s->inst[0] = b + o64;
    s->inst[1] = b + o32;
    s->inst[2] = b + oh;
    for (int d = 0; d < 3; ++d) {
        for (int k = 0; k < 3; ++k) {
            if ((e = up(ot[d][k], t[d][k].data(), t[d][k].size() * sizeof(fd::BatchTile))) != cudaSuccess) return e;
            s->tiles[d][k] = reinterpret_cast<fd::BatchTile*>(b + ot[d][k]);
            for (int r = 0; r < kMaxSteps; ++r) s->ntiles[d][k][r] = count[d][k][r];
        }
        if ((e = up(of[d], f[d].data(), f[d].size() * sizeof(fd::BatchTile))) != cudaSuccess) return e;
        s->fresh_tiles[d] = reinterpret_cast<fd::BatchTile*>(b + of[d]);
        s->nfresh[d] = (int)f[d].size();
    }
    // Host vectors are pageable: the copies above have consumed them on return.
    return cudaSuccess;
}

template <class T>
cudaError_t run_group(fd_server* s, int d, int round) {
    auto* I = static_cast<const fd::BatchInst<T>*>(s->inst[d]);
    cudaError_t e;
    const int gg = s->sms * fd::batch_blocks_per_sm<T>(false, false);
    const int* nt[3] = {&s->ntiles[d][0][round], &s->ntiles[d][1][round], &s->ntiles[d][2][round]};
    if (round == 0 && s->nfresh[d]) {
        if ((e = fd::launch_batch_prims<T>(I, s->fresh_tiles[d], s->nfresh[d], s->parity, gg, s->stream)) !=
            cudaSuccess)
            return e;
    }
    const bool tiled = sizeof(T) == sizeof(float);  // binary32 RA: shared-memory kernels
    const int gs = s->sms * fd::batch_blocks_per_sm<T>(true, true);
    const int gr = s->sms * (tiled ? fd::batch_tiled_blocks_per_sm<T>() : fd::batch_blocks_per_sm<T>(true, false));
    const int gt = s->sms * s->tma_blocks;
    // round r starts at parity parity ^ (r & 1): every solve it advances has taken r steps this tick
    for (int st = 0, p = s->parity ^ (round & 1); st < 3; ++st, p ^= 1) {
        if (*nt[0]) {
            if ((e = fd::launch_batch_grad<T>(I, s->tiles[d][0], *nt[0], p, gg, s->stream)) != cudaSuccess) return e;
            if ((e = fd::launch_batch_fused<T>(I, s->tiles[d][0], *nt[0], true, st, p, gs, s->stream)) != cudaSuccess)
                return e;
        }
        if (*nt[1]) {
            if constexpr (sizeof(T) == sizeof(float))
                e = fd::launch_batch_ra_tiled<T>(I, s->tiles[d][1], *nt[1], st, p, gr, s->stream);
            else
                e = fd::launch_batch_fused<T>(I, s->tiles[d][1], *nt[1], false, st, p, gr, s->stream);
            if (e != cudaSuccess) return e;
        }
        if constexpr (sizeof(T) == sizeof(float)) {
            if (*nt[2]) {
                e = fd::launch_batch_ra_tma(I, s->tiles[d][2], *nt[2], st, p, gt, s->tma_zlen, s->kerr, s->stream);
                if (e != cudaSuccess) return e;
            }
        }
    }
    return cudaSuccess;
}

// The mixed (FD_F64_DW) group: store-some only, the two fused kernels per stage (the first also
// forms the gradients).
cudaError_t run_group_hyb(fd_server* s, int round) {
    auto* I = static_cast<const fd::BatchHyb*>(s->inst[2]);
    cudaError_t e;
    const int n = s->ntiles[2][0][round];
    if (round == 0 && s->nfresh[2]) {
        const int gp = s->sms * fd::batch_hyb_blocks_per_sm(0);
        if ((e = fd::launch_batch_prims_hyb(I, s->fresh_tiles[2], s->nfresh[2], s->parity, gp, s->stream)) !=
            cudaSuccess)
            return e;
    }
    if (!n) return cudaSuccess;
    const int gs = s->sms * fd::batch_hyb_blocks_per_sm(1), gc = s->sms * fd::batch_hyb_blocks_per_sm(2);
    for (int st = 0, p = s->parity ^ (round & 1); st < 3; ++st, p ^= 1) {
        if ((e = fd::launch_batch_ss_hyb(I, s->tiles[2][0], n, st, p, gc, gs, s->stream)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Retire the solves of pending slot i: wait for the tick that finished them,
// check the staging-error word of that tick, and turn them into results (in
// the order the tick finished them) whose states stay kept.
int retire(fd_server* s, int i) {
    Pending& P = s->pending[i];
    if (!P.armed) return FD_OK;
    P.armed = false;
    cudaError_t e = cudaEventSynchronize(P.ev);
    if (e != cudaSuccess) return s->cuda_fail(e, "fd_server_tick");
    if (P.check_err && *P.host_err) {
        const int v = *P.host_err;
        P.solves.clear();
        return s->fail(FD_ECUDA, "fd_server_tick: %s; the states are not valid",
                       v == 2 ? "the TMA ring was not 128-byte aligned" : "a staging wait in a kernel ran out");
    }
    for (size_t k = 0; k < P.solves.size(); ++k) {
        const Finished& f = P.solves[k];
        const double ke = P.host_res[2 * k], en = P.host_res[2 * k + 1];
        const int st = std::isfinite(ke) && std::isfinite(en) ? FD_OK : FD_EUNSTABLE;
        s->done.push_back({f.r.tag, st, f.done, ke, en});
        s->finished.push_back(f);
        s->completed++;
    }
    P.solves.clear();
    return FD_OK;
}

// Retire every outstanding tick, oldest first.
int retire_all(fd_server* s) {
    int first = s->pending[0].tick <= s->pending[1].tick ? 0 : 1;
    int rc = retire(s, first);
    if (rc == FD_OK) rc = retire(s, first ^ 1);
    return rc;
}

void release_all(fd_server* s) {
    if (s->stream || s->arena_ptr) cudaStreamSynchronize(s->stream);
    s->dev_free(s->tab, s->tab_bytes);
    s->dev_free(s->fixed, s->fixed_bytes);
    s->dev_free(s->arena_ptr, s->arena.capacity());
    s->tab = s->fixed = s->arena_ptr = nullptr;
    for (auto& P : s->pending) {
        if (P.ev) cudaEventDestroy(P.ev);
        P.ev = nullptr;
    }
    if (s->host_pinned) cudaFreeHost(s->host_pinned);
    s->host_pinned = nullptr;
}

}  // namespace

extern "C" {

size_t fd_server_footprint(const fd_request* req) { return check_request(req) ? 0 : layout_of(*req, true).total; }

int fd_server_create(fd_server** out, size_t arena_bytes, int max_active, const fd_alloc* alloc, void* cuda_stream) {
    if (!out) return fail_global(FD_EINVAL, "fd_server_create: out is NULL");
    *out = nullptr;
    if (arena_bytes < kAlign || max_active < 1)
        return fail_global(FD_EINVAL, "fd_server_create: need arena_bytes >= 256 and max_active >= 1");
    if (alloc && (!alloc->alloc || !alloc->free))
        return fail_global(FD_EINVAL, "fd_server_create: allocator needs both alloc and free");
    fd_server* s = new (std::nothrow) fd_server();
    if (!s) return fail_global(FD_ENOMEM, "fd_server_create: host allocation failed");
    s->stream = static_cast<cudaStream_t>(cuda_stream);
    s->max_active = max_active;
    if (alloc) {
        s->alloc = *alloc;
        s->has_alloc = true;
    }
    cudaGetDevice(&s->device);
    cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device);
    if (s->sms <= 0) s->sms = 152;
    arena_bytes = arena_bytes & ~(kAlign - 1);
    s->arena_ptr = s->dev_alloc(arena_bytes);
    if (!s->arena_ptr) {
        delete s;
        return fail_global(FD_ENOMEM, "fd_server_create: arena of %zu bytes could not be allocated", arena_bytes);
    }
    s->arena = Arena(arena_bytes);
    s->fixed_bytes = align256(2 * fd::kDiagBlocks * sizeof(double)) + align256(2 * (size_t)max_active * sizeof(double)) +
                     align256(sizeof(int));
    s->fixed = s->dev_alloc(s->fixed_bytes);
    if (!s->fixed) {
        release_all(s);
        delete s;
        return fail_global(FD_ENOMEM, "fd_server_create: diagnostics buffers could not be allocated");
    }
    s->partial = static_cast<double*>(s->fixed);
    s->results = reinterpret_cast<double*>(static_cast<char*>(s->fixed) + align256(2 * fd::kDiagBlocks * sizeof(double)));
    s->kerr = reinterpret_cast<int*>(reinterpret_cast<char*>(s->results) + align256(2 * (size_t)max_active * sizeof(double)));
    const char* off_env = std::getenv("FDGB300_NO_TMA");
    s->tma_allowed = !(off_env && off_env[0] == '1');
    // two pending slots: 2 results per solve, then an error word, each slot
    const size_t slot_bytes = align256(2 * (size_t)max_active * sizeof(double) + sizeof(int));
    cudaError_t e = cudaMallocHost(&s->host_pinned, 2 * slot_bytes);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        Pending& P = s->pending[i];
        P.host_res = reinterpret_cast<double*>(static_cast<char*>(s->host_pinned) + i * slot_bytes);
        P.host_err = reinterpret_cast<int*>(P.host_res + 2 * (size_t)max_active);
        *P.host_err = 0;
        e = cudaEventCreateWithFlags(&P.ev, cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        release_all(s);
        delete s;
        return fail_global(FD_ENOMEM, "fd_server_create: host result buffers: %s", cudaGetErrorString(e));
    }
    e = cudaMemsetAsync(s->kerr, 0, sizeof(int), s->stream);
    if (e == cudaSuccess && s->tma_allowed) {
        e = fd::prepare_ra_tma();
        s->tma_blocks = fd::batch_tma_blocks_per_sm();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        release_all(s);
        delete s;
        return fail_global(FD_ECUDA, "fd_server_create: set-up: %s", cudaGetErrorString(e));
    }
    *out = s;
    return FD_OK;
}

int fd_server_submit(fd_server* s, const fd_request* req) {
    if (!s) return fail_global(FD_EINVAL, "fd_server_submit: NULL server");
    if (const char* why = check_request(req)) return s->fail(FD_EINVAL, "fd_server_submit: %s", why);
    size_t need = layout_of(*req, s->tma_allowed).total;
    if (need > s->arena.capacity())
        return s->fail(FD_EBUSY, "fd_server_submit: footprint %zu bytes exceeds the arena (%zu)", need,
                       s->arena.capacity());
    s->queue.push_back(*req);
    s->submitted++;
    return FD_OK;
}

int fd_server_cancel(fd_server* s, long long tag) {
    if (!s) return fail_global(FD_EINVAL, "fd_server_cancel: NULL server");
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
        if (it->tag == tag) {
            s->done.push_back({tag, FD_EBUSY, 0, 0.0, 0.0});
            s->queue.erase(it);
            return FD_OK;
        }
    for (auto& a : s->active)
        if (a.r.tag == tag && !a.cancelled) {
            a.cancelled = true;
            return FD_OK;
        }
    return s->fail(FD_EINVAL, "fd_server_cancel: no pending request with tag %lld", tag);
}

int fd_server_tick(fd_server* s, int* active_out) {
    if (!s) return fail_global(FD_EINVAL, "fd_server_tick: NULL server");
    s->ticks++;
    cudaError_t e = cudaSuccess;
    // 0. finished solves whose results were polled since the last tick free their blocks
    for (size_t i = 0; i < s->finished.size();) {
        if (s->finished[i].polled) {
            s->arena.release(s->finished[i].off, s->finished[i].L.total);
            s->finished.erase(s->finished.begin() + i);
        } else {
            ++i;
        }
    }
    // 1. cancelled active solves leave without diagnostics
    for (size_t i = 0; i < s->active.size();) {
        Active& a = s->active[i];
        if (a.cancelled) {
            s->done.push_back({a.r.tag, FD_EBUSY, a.done, 0.0, 0.0});
            s->arena.release(a.off, a.L.total);
            s->active.erase(s->active.begin() + i);
            s->dirty = true;
        } else {
            ++i;
        }
    }
    // 2. admission: first fit in submission order
    for (auto it = s->queue.begin(); it != s->queue.end() && (int)s->active.size() < s->max_active;) {
        Layout L = layout_of(*it, s->tma_allowed);
        size_t off = 0;
        if (!s->arena.alloc(L.total, &off)) {
            ++it;
            continue;
        }
        Active a;
        a.r = *it;
        a.L = L;
        a.off = off;
        a.n = it->nx * it->ny * it->nz;
        fd::Grid g = fd::make_grid(a.r.nx, a.r.ny, a.r.nz);
        fd::Phys ph = fd::make_phys(a.r.Re, a.r.Mach, a.r.Pr, a.r.gamma);
        // binary32 solves keep a shifted double-word state (rho - 1, rho u_i,
        // rho E - rhoE0): the binary64 initial condition passes through Qs.
        char* Q = s->base() + off + (s->parity ? L.q1 : L.q0);
        const bool dw = a.r.dtype == FD_F32_ACCDW;  // double-word state
        double* ic = reinterpret_cast<double*>(dw ? s->base() + off + L.qs : Q);
        e = fd::launch_tgv_ic(g, ph, 2.0 * fd::kPi / a.r.nx, 2.0 * fd::kPi / a.r.ny, 2.0 * fd::kPi / a.r.nz, ic,
                              s->stream);
        if (e == cudaSuccess && dw)
            e = fd::launch_to_df64(ic, reinterpret_cast<fd::df64*>(Q), a.n, fd::Shift5{{1.0, 0.0, 0.0, 0.0, ph.rhoE0}},
                                   s->stream);
        if (L.padded) {  // padding columns no point writes are copied but never read: zero them
            const size_t bytes = 10 * fd::padded_field_points(g) * sizeof(float);
            if (e == cudaSuccess) e = cudaMemsetAsync(s->base() + off + L.w0, 0, bytes, s->stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(s->base() + off + L.w1, 0, bytes, s->stream);
        }
        if (e != cudaSuccess) {
            s->arena.release(off, L.total);
            return s->cuda_fail(e, "fd_server_tick: initial condition");
        }
        s->active.push_back(a);
        it = s->queue.erase(it);
        s->dirty = true;
    }
    if (active_out) *active_out = (int)s->active.size();
    if (s->active.empty()) return retire_all(s);  // nothing to overlap with
    // 3. steps per solve, tables, then k RK3 steps of every active solve
    double dearest = 0;
    for (auto& a : s->active) dearest = std::max(dearest, step_cost(a.r));
    bool any_fresh = false;
    for (auto& a : s->active) {
        any_fresh |= a.fresh;
        const int left = a.r.steps - a.done;
        int k = (int)std::min<double>({(double)kMaxSteps, (double)left, std::floor(dearest / step_cost(a.r))});
        k = std::max(1, k);
        if (k % 2 == 0) --k;
        if (k != a.k) {
            a.k = k;
            s->dirty = true;
        }
    }
    if (s->dirty || any_fresh) {
        if ((e = rebuild(s)) != cudaSuccess) return s->cuda_fail(e, "fd_server_tick: tables");
        s->dirty = false;
    }
    for (int r = 0; r < s->rounds; ++r) {
        if ((e = run_group<double>(s, 0, r)) != cudaSuccess) return s->cuda_fail(e, "fd_server_tick: binary64 group");
        if ((e = run_group<float>(s, 1, r)) != cudaSuccess) return s->cuda_fail(e, "fd_server_tick: binary32 group");
        if ((e = run_group_hyb(s, r)) != cudaSuccess) return s->cuda_fail(e, "fd_server_tick: mixed group");
    }
    s->parity ^= 1;
    s->nfresh[0] = s->nfresh[1] = s->nfresh[2] = 0;
    for (auto& a : s->active) {
        a.fresh = false;
        a.done += a.k;
    }
    // 4. diagnostics of the solves this tick finishes (scratch: the working
    //    fields the next stage would overwrite) and the staging-error word,
    //    copied to this tick's pending slot; then wait for the previous tick
    //    only and retire its solves, so the work just enqueued keeps the device
    //    busy while the caller plans the next tick.
    const int slot = (int)(s->ticks & 1);
    Pending& P = s->pending[slot];
    if (P.armed) {  // left by a tick that failed before it retired this slot
        const int rc = retire(s, slot);
        if (rc != FD_OK) return rc;
    }
    std::vector<int> fin;
    for (int i = 0; i < (int)s->active.size(); ++i)
        if (s->active[i].done >= s->active[i].r.steps) fin.push_back(i);
    for (size_t k = 0; k < fin.size() && e == cudaSuccess; ++k) {
        const Active& a = s->active[fin[k]];
        fd::Grid g = fd::make_grid(a.r.nx, a.r.ny, a.r.nz);
        char* b = s->base() + a.off;
        const double* Q = reinterpret_cast<const double*>(b + (s->parity ? a.L.q1 : a.L.q0));
        if (a.r.dtype == FD_F32_ACCDW) {  // double-word state to binary64 in the retiring solve's Qs
            double* tmp = reinterpret_cast<double*>(b + a.L.qs);
            fd::Phys ph = fd::make_phys(a.r.Re, a.r.Mach, a.r.Pr, a.r.gamma);
            e = fd::launch_from_df64(reinterpret_cast<const fd::df64*>(Q), tmp, a.n,
                                     fd::Shift5{{1.0, 0.0, 0.0, 0.0, ph.rhoE0}}, s->stream);
            Q = tmp;
        }
        double* Wv = reinterpret_cast<double*>(b + (s->parity ? a.L.w0 : a.L.w1));
        if (e == cudaSuccess) e = fd::launch_diagnostics_f64(g, Q, Wv, s->partial, s->results + 2 * k, s->stream);
    }
    if (e == cudaSuccess && !fin.empty())
        e = cudaMemcpyAsync(P.host_res, s->results, 2 * fin.size() * sizeof(double), cudaMemcpyDeviceToHost,
                            s->stream);
    P.check_err = s->ntiles[1][2][0] != 0;
    if (e == cudaSuccess && P.check_err)
        e = cudaMemcpyAsync(P.host_err, s->kerr, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaEventRecord(P.ev, s->stream);
    if (e != cudaSuccess) return s->cuda_fail(e, "fd_server_tick");
    P.armed = true;
    P.tick = s->ticks;
    for (size_t k = fin.size(); k-- > 0;) {
        const Active& a = s->active[fin[k]];
        Finished f{a.r, a.L, a.off, a.n, s->parity, false, a.done};
        P.solves.insert(P.solves.begin(), f);
        s->active.erase(s->active.begin() + fin[k]);
        s->dirty = true;
    }
    int rc = retire(s, slot ^ 1);
    if (rc == FD_OK && s->active.empty()) rc = retire(s, slot);
    return rc;
}

int fd_server_poll(fd_server* s, fd_result* out, int max, int* n_out) {
    if (!s) return fail_global(FD_EINVAL, "fd_server_poll: NULL server");
    if (max < 0 || (max > 0 && !out)) return s->fail(FD_EINVAL, "fd_server_poll: bad output buffer");
    int n = std::min<int>(max, (int)s->done.size());
    for (int i = 0; i < n; ++i) {
        out[i] = s->done[i];
        // the solve's block returns to the arena at the next tick
        for (auto& f : s->finished)
            if (f.r.tag == out[i].tag && !f.polled) {
                f.polled = true;
                break;
            }
    }
    s->done.erase(s->done.begin(), s->done.begin() + n);
    if (n_out) *n_out = n;
    return FD_OK;
}

int fd_server_get_state(fd_server* s, long long tag, double* dst, size_t n_elems, int dst_is_device) {
    if (!s) return fail_global(FD_EINVAL, "fd_server_get_state: NULL server");
    if (!dst) return s->fail(FD_EINVAL, "fd_server_get_state: dst is NULL");
    const Finished* f = nullptr;
    for (const auto& x : s->finished)
        if (x.r.tag == tag) {
            f = &x;
            break;
        }
    // finished by an outstanding tick (the copy below waits for its work)
    const int first = s->pending[0].tick <= s->pending[1].tick ? 0 : 1;
    for (int i : {first, first ^ 1})
        for (const auto& x : s->pending[i].solves)
            if (!f && x.r.tag == tag) f = &x;
    if (!f) return s->fail(FD_EINVAL, "fd_server_get_state: no kept state of a finished solve with tag %lld", tag);
    if (n_elems != 5 * (size_t)f->n)
        return s->fail(FD_EINVAL, "fd_server_get_state: n_elems = %zu, expected %zu", n_elems, 5 * (size_t)f->n);
    char* b = s->base() + f->off;
    const double* src = reinterpret_cast<const double*>(b + (f->parity ? f->L.q1 : f->L.q0));
    cudaError_t e = cudaSuccess;
    if (f->r.dtype == FD_F32_ACCDW) {  // shifted double-word state to binary64 through the solve's dead Qs
        double* tmp = reinterpret_cast<double*>(b + f->L.qs);
        const fd::Phys ph = fd::make_phys(f->r.Re, f->r.Mach, f->r.Pr, f->r.gamma);
        e = fd::launch_from_df64(reinterpret_cast<const fd::df64*>(src), tmp, f->n,
                                 fd::Shift5{{1.0, 0.0, 0.0, 0.0, ph.rhoE0}}, s->stream);
        src = tmp;
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dst, src, n_elems * sizeof(double),
                            dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return s->cuda_fail(e, "fd_server_get_state");
    return FD_OK;
}

int fd_server_get_stats(const fd_server* s, fd_server_stats* out) {
    if (!s || !out) return fail_global(FD_EINVAL, "fd_server_get_stats: NULL argument");
    out->queued = (int)s->queue.size();
    out->active = (int)s->active.size();
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->ticks = s->ticks;
    out->arena_bytes = s->arena.capacity();
    out->arena_used = s->arena.used();
    return FD_OK;
}

int fd_server_destroy(fd_server* s) {
    if (!s) return FD_OK;
    release_all(s);
    delete s;
    return FD_OK;
}

const char* fd_server_last_error(const fd_server* s) { return s ? s->err.c_str() : g_server_err.c_str(); }

}  // extern "C"
