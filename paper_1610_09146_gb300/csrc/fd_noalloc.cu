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
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/fdgb300.h"
#include "fd_internal.h"

namespace {

constexpr int kScratchArrays = 17;  // u, v, w, p, T + nine du_i/dx_j + three pair sums
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kScratchArrays * (size_t)FD_NOALLOC_MAX_POINTS];

// Device address of g_noalloc_scratch per device, looked up once per device
// (with that device current).  In host code the symbol's name is only a
// host-side stand-in, never a device address.
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

cudaError_t scratch_for_current_device(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double*>(p);
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

    const double kPi = 3.14159265358979323846;
    fd::Grid g{};
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.n = nx * ny * nz;
    const int ns[3] = {nx, ny, nz};
    for (int a = 0; a < 3; ++a) {
        double h = 2.0 * kPi / ns[a];
        g.inv12h[a] = 1.0 / (12.0 * h);
        g.inv12h2[a] = 1.0 / (12.0 * h * h);
        g.inv12hf[a] = (float)g.inv12h[a];
        g.inv12h2f[a] = (float)g.inv12h2[a];
    }
    fd::Phys ph{};
    ph.gamma = gamma;
    ph.gm1 = gamma - 1.0;
    ph.gM2 = gamma * Mach * Mach;
    ph.nu = 1.0 / Re;
    ph.kappa = 1.0 / ((gamma - 1.0) * Mach * Mach * Pr * Re);
    ph.p0 = 1.0 / (gamma * Mach * Mach);
    ph.rhoE0 = ph.p0 / (gamma - 1.0);
    fd::Coef<double> k{};
    for (int j = 0; j < 3; ++j) {
        double s1 = g.inv12h[j], s2 = g.inv12h2[j];
        k.s1[j] = s1;
        k.c1[j] = -0.5 * s1;
        k.cp[j] = -s1;
        k.ks2[j] = ph.kappa * s2;
        k.vmix1[j] = ph.nu / 3.0 * s1;
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            k.vs2[i][j] = ph.nu * g.inv12h2[j] * (i == j ? 4.0 / 3.0 : 1.0);
            k.vmix[i][j] = ph.nu / 3.0 * g.inv12h[i] * g.inv12h[j];
        }
    k.nu = ph.nu;

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
