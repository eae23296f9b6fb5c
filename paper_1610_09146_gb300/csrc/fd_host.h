// fd_host.h -- host-side set-up shared by the single-instance and batched
// paths: grid spacings, flow constants with their negative powers (Section 2:
// rationals and inverse constants are evaluated once at start-up), the fused
// residual's coefficients, and the Runge-Kutta coefficients.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "fd_core.cuh"

namespace fd {

constexpr double kPi = 3.14159265358979323846;
// Two-register low-storage RK3 (read of Section 2 / Fig. 1): a, b per stage.
constexpr double kRkA[3] = {2.0 / 3.0, 5.0 / 12.0, 3.0 / 5.0};
constexpr double kRkB[3] = {1.0 / 4.0, 3.0 / 20.0, 0.0};

// Periodic grid x_i = i * 2 pi / n per axis (Section 3).  nz_period > 0: the
// z spacing is that of a periodic grid of nz_period planes, of which these nz
// are a slab (the z-slab decomposition).
inline Grid make_grid(int nx, int ny, int nz, int nz_period = 0) {
    Grid g{};
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.n = nx * ny * nz;
    const int ns[3] = {nx, ny, nz_period > 0 ? nz_period : nz};
    for (int a = 0; a < 3; ++a) {
        double h = 2.0 * kPi / ns[a];
        g.inv12h[a] = 1.0 / (12.0 * h);
        g.inv12h2[a] = 1.0 / (12.0 * h * h);
        g.inv12hf[a] = (float)g.inv12h[a];
        g.inv12h2f[a] = (float)g.inv12h2[a];
        g.inv12h_w[a] = df64(g.inv12h[a]);
        g.inv12h2_w[a] = df64(g.inv12h2[a]);
    }
    return g;
}

inline Phys make_phys(double Re, double Mach, double Pr, double gamma) {
    Phys ph{};
    ph.gamma = gamma;
    ph.gm1 = gamma - 1.0;
    ph.gM2 = gamma * Mach * Mach;
    ph.nu = 1.0 / Re;
    ph.kappa = 1.0 / ((gamma - 1.0) * Mach * Mach * Pr * Re);
    ph.p0 = 1.0 / (gamma * Mach * Mach);
    ph.rhoE0 = ph.p0 / (gamma - 1.0);
    ph.gm1_w = df64(ph.gm1);
    ph.gM2_w = df64(ph.gM2);
    ph.rhoE0_w = df64(ph.rhoE0);
    ph.nu_w = df64(ph.nu);
    ph.kappa_w = df64(ph.kappa);
    ph.cE_w = df64(ph.rhoE0 + ph.p0);
    return ph;
}

// The RK constants of stage s for a time step dt.
inline RKStage make_stage(int s, double dt) {
    RKStage rk{};
    rk.adt = kRkA[s] * dt;
    rk.bdt = kRkB[s] * dt;
    rk.stage = s;
    rk.adt_w = df64(rk.adt);
    rk.bdt_w = df64(rk.bdt);
    return rk;
}

// Constants of the fused residual (see fd::Coef); `shifted` selects the
// perturbation form of the binary32 and df64 modes.
template <class T>
Coef<T> make_coef(const Grid& g, const Phys& ph, bool shifted) {
    Coef<T> k{};
    for (int j = 0; j < 3; ++j) {
        double s1 = g.inv12h[j], s2 = g.inv12h2[j];
        k.s1[j] = (T)s1;
        k.c1[j] = (T)(-0.5 * s1);
        k.cp[j] = (T)(-s1);
        k.ks2[j] = (T)(ph.kappa * s2);
        k.vmix1[j] = (T)(ph.nu / 3.0 * s1);
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            k.vs2[i][j] = (T)(ph.nu * g.inv12h2[j] * (i == j ? 4.0 / 3.0 : 1.0));
            k.vmix[i][j] = (T)(ph.nu / 3.0 * g.inv12h[i] * g.inv12h[j]);
        }
    // tap weights of the binary64 residual (exact multiples of the above but
    // the centre sums, which are rounded once here)
    if constexpr (kTapWeighted<T>) {
        for (int j = 0; j < 3; ++j) {
            k.c8[j] = -4.0 * g.inv12h[j];
            k.k16[j] = 16.0 * ph.kappa * g.inv12h2[j];
        }
        k.kc = -30.0 * ph.kappa * (g.inv12h2[0] + g.inv12h2[1] + g.inv12h2[2]);
        for (int i = 0; i < 3; ++i) {
            double sum = 0.0;
            for (int j = 0; j < 3; ++j) {
                const double v = ph.nu * g.inv12h2[j] * (i == j ? 4.0 / 3.0 : 1.0);
                k.v16[i][j] = 16.0 * v;
                sum += v;
            }
            k.vc[i] = -30.0 * sum;
        }
    }
    k.nu = (T)ph.nu;
    k.c_rho = shifted ? (T)-1.0 : (T)0.0;
    k.c_E = shifted ? (T)(-(ph.rhoE0 + ph.p0)) : (T)0.0;
    return k;
}

// Argument checks shared by fd_create and the batch / server calls; returns
// nullptr when valid, else a static description of the first problem.
inline const char* check_instance(int nx, int ny, int nz, double Re, double Mach, double Pr, double gamma,
                                  double dt) {
    if (nx < 5 || ny < 5 || nz < 5) return "every axis needs at least 5 points";
    // the kernels address the ten working fields of an instance with 32-bit
    // offsets (f n + c, f <= 9); the store-all work arrays use 64-bit ones
    if ((long long)nx * ny * nz > kMaxPoints) return "nx*ny*nz must be at most 214748364 (598^3)";
    if (!(Re > 0) || !(Mach > 0) || !(Pr > 0) || !(dt > 0) || !std::isfinite(Re) || !std::isfinite(Mach) ||
        !std::isfinite(Pr) || !std::isfinite(dt))
        return "Re, Mach, Pr and dt must be positive and finite";
    if (!(gamma > 1) || !std::isfinite(gamma)) return "gamma must be > 1";
    return nullptr;
}

// Per-kernel timing: CUDA events recorded around each launch on the caller's
// stream, folded into per-class totals when the ring fills or on read.
struct Profiler {
    static constexpr int kCap = 2048;
    static constexpr int kClasses = 6;  // FD_KERNEL_CLASSES
    bool on = false;
    std::vector<cudaEvent_t> ev;  // 2 * kCap events, created on first enable
    std::vector<int> cls;         // kernel class of each pending pair
    int used = 0;
    double total_ms[kClasses] = {};
    long long count[kClasses] = {};

    cudaError_t enable(bool en, cudaStream_t st) {
        if (en && ev.empty()) {
            ev.assign(2 * kCap, nullptr);
            cls.assign(kCap, 0);
            for (auto& e : ev) {
                cudaError_t rc = cudaEventCreate(&e);
                if (rc != cudaSuccess) return rc;
            }
        }
        cudaError_t rc = fold(st);
        if (rc != cudaSuccess) return rc;
        for (int c = 0; c < kClasses; ++c) {
            total_ms[c] = 0.0;
            count[c] = 0;
        }
        on = en;
        return cudaSuccess;
    }

    cudaError_t fold(cudaStream_t st) {
        if (used == 0) return cudaSuccess;
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
        for (int i = 0; i < used; ++i) {
            float ms = 0.f;
            e = cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]);
            if (e != cudaSuccess) return e;
            total_ms[cls[i]] += ms;
            count[cls[i]] += 1;
        }
        used = 0;
        return cudaSuccess;
    }

    // Launch one kernel (the callable returns its launch status), bracketed by
    // a pair of events when timing is on.
    template <class F>
    cudaError_t timed(cudaStream_t st, int c, F launch) {
        if (!on) return launch();
        if (used == kCap) {
            cudaError_t e = fold(st);
            if (e != cudaSuccess) return e;
        }
        cudaEvent_t a = ev[2 * used], b = ev[2 * used + 1];
        cudaError_t e = cudaEventRecord(a, st);
        if (e != cudaSuccess) return e;
        e = launch();
        if (e != cudaSuccess) return e;
        e = cudaEventRecord(b, st);
        if (e != cudaSuccess) return e;
        cls[used++] = c;
        return cudaSuccess;
    }

    void destroy() {
        for (auto e : ev)
            if (e) cudaEventDestroy(e);
        ev.clear();
    }
};

}  // namespace fd
