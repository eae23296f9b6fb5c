// fd_noalloc.cu -- fd_residual_noalloc: the store-some residual for a
// caller-owned device state, with its scratch in a fixed device array, so the
// call itself never allocates device (or host) memory.
//
// Who needs this: callers that may not call cudaMalloc at the moment they
// need a residual -- an external time integrator evaluating R(Q) inside a
// region where allocation is forbidden (a stream-capture in progress, a
// real-time loop with a fixed memory budget, a process whose memory is held by
// another framework's pool).  fd_residual needs a handle, and fd_create
// allocates; this entry point needs neither.
//
// The scratch holds the primitives u, v, w, p, T (5 arrays), the nine
// velocity gradients and the three pair sums of the diagonal ones (12 arrays)
// of at most FD_NOALLOC_MAX_POINTS points.  It is a file-scope __device__
// array, so every GPU that loads the library keeps it (17 x 262144 x 8 bytes
// = 35.7 MB) until the process exits.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/fdgb300.h"
#include "fd_host.h"
#include "fd_internal.h"

namespace {

constexpr int kScratchArrays = 17;  // u, v, w, p, T + nine du_i/dx_j + three pair sums
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kScratchArrays * (size_t)FD_NOALLOC_MAX_POINTS];

// Device address of g_noalloc_scratch per device, looked up with that device
// current.  In host code the symbol's name is only a host-side stand-in, never
// a device address.  The address belongs to the context the module was loaded
// into: each cached address is kept beside that context (cuCtxGetCurrent,
// through the runtime's driver entry point) and looked up again when the
// device's current context is a different one, e.g. after cudaDeviceReset.
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};

cudaError_t current_context(CUcontext* ctx) {
    using GetCurrent = CUresult (*)(CUcontext*);
    static GetCurrent get = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<GetCurrent>(p);
    }();
    if (!get) return cudaErrorNotSupported;
    return get(ctx) == CUDA_SUCCESS ? cudaSuccess : cudaErrorDeviceUninitialized;
}

cudaError_t scratch_for_current_device(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    CUcontext ctx = nullptr;
    if ((e = current_context(&ctx)) != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!ctx || !g_scratch_ptr[dev] || g_scratch_ctx[dev] != ctx) {
        // the lookup also makes the device's primary context current when no
        // context is yet, so the context is read again after it
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        if ((e = current_context(&ctx)) != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double*>(p);
        g_scratch_ctx[dev] = ctx;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int fd_residual_noalloc(const double* Q, double* R, int nx, int ny, int nz, double Re, double Mach,
                                   double Pr, double gamma, void* cuda_stream) {
    if (!Q || !R) return FD_EINVAL;
    if (nx < 5 || ny < 5 || nz < 5) return FD_EINVAL;
    if ((long long)nx * ny * nz > FD_NOALLOC_MAX_POINTS) return FD_EINVAL;
    if (!(Re > 0) || !(Mach > 0) || !(Pr > 0) || !(gamma > 1)) return FD_EINVAL;
    double* scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess) return FD_ECUDA;

    const fd::Grid g = fd::make_grid(nx, ny, nz);
    const fd::Phys ph = fd::make_phys(Re, Mach, Pr, gamma);
    const fd::Coef<double> k = fd::make_coef<double>(g, ph, false);

    // The scratch is rewritten in full before it is read on every call (the
    // primitives from Q, then the gradients from the primitives), so nothing
    // in it has to start at zero; what the previous call left there is unused.
    const size_t n = (size_t)g.n;
    double* W = scratch;          // u, v, w, p, T
    double* G = scratch + 5 * n;  // du_i/dx_j at (3 i + j) * n, pair sums at (9 + i) * n
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const fd::RKStage rk{0.0, 0.0, 0};
    if (fd::launch_prims_f64(g, ph, Q, W, st) != cudaSuccess) return FD_ECUDA;
    if (fd::launch_ss_grad<double>(g, k, W, G, st) != cudaSuccess) return FD_ECUDA;
    if (fd::launch_ss<double>(g, k, ph, rk, true, Q, W, G, Q, R, nullptr, nullptr, st) != cudaSuccess)
        return FD_ECUDA;
    return FD_OK;
}
