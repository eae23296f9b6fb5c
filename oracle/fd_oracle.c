/*
 * fd_oracle.c -- plain FP64 CPU oracle for one low-storage RK3 step of the
 * 3-D compressible Navier-Stokes residual with 4th-order central differences
 * on a periodic [0, 2*pi]^3 grid (Jammy, Jacobs & Sandham, "Performance
 * evaluation of explicit finite difference algorithms with varying amounts of
 * computational and memory intensity", arXiv 1610.09146, Sections 2 and 3).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent checker of the CUDA
 * path: only the tests, the smoke check of the package entry and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant with the CUDA path, and the product path never calls it.
 *
 * It is written to be read against the paper, not to be fast: every operator
 * is a separate pass over whole grid arrays, products inside a derivative are
 * formed into a work array first and then differenced (the "store-all" way of
 * Section 2, paragraph BL), and the only parallelism is an OpenMP loop over
 * z-planes (results do not depend on the thread count: every output point is
 * computed by one thread and every reduction is summed in a fixed order).
 * Build with -O2 -ffp-contract=off so that no fused multiply-add changes the
 * rounding between x86 and Arm.
 *
 * Readings of points the paper leaves open (all stated where used):
 *  - stencil weights: standard 5-point central 4th-order first and second
 *    derivatives (Section 2 names the order only);
 *  - mixed second derivatives d2/dxi dxk (i != k) are the first-derivative
 *    operator applied twice; pure second derivatives use the 5-point formula;
 *  - the skew-symmetric convective form (Eq. skewscalar) is applied with
 *    phi = 1, u_i, E to the fluxes rho*u_j, rho*u_i*u_j, rho*E*u_j; the
 *    pressure work d(u_j p)/dx_j stays in conservative form;
 *  - the viscous divergences are expanded by the product rule into second
 *    derivatives of u (Section 2, last sentence before Fig. 1);
 *  - the low-storage RK3 is the two-register scheme
 *      Q <- Qs + a_s dt R(Q),  Qs <- Qs + b_s dt R(Q),
 *    a = (2/3, 5/12, 3/5), b = (1/4, 3/20, -), with Qs = Q at save-state
 *    (Fig. 1); its Butcher weights are b = (1/4, 3/20, 3/5), c = (0, 2/3, 2/3);
 *  - grid points x_i = i * 2*pi / n, i = 0..n-1, periodic in all directions;
 *  - kinetic energy and enstrophy are density-weighted volume means with
 *    reference density 1 (Section 3 defers to DeBonis 2013).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

/* Grid sizes, grid spacings and the flow constants of Section 3.  On the
 * paper's domain h = 2*pi / n per axis; a different h lets a caller evaluate
 * the scheme on a small periodic block cut out of a larger grid. */
typedef struct {
    int nx, ny, nz;
    double hx, hy, hz;
    double Re, Mach, Pr, gamma, dt;
} or_params;

/* ---- grid helpers ------------------------------------------------------ */

static long npts(int nx, int ny, int nz) { return (long)nx * ny * nz; }

static int wrap(int i, int n) { return ((i % n) + n) % n; }

static long at(int nx, int ny, int x, int y, int z) {
    return ((long)z * ny + y) * nx + x;
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---- Section 2: fourth-order central differences on the periodic grid --- */

/* First derivative along `axis` (0 = x, 1 = y, 2 = z) with spacing h:
 *   D f_i = [8 (f_{i+1} - f_{i-1}) - (f_{i+2} - f_{i-2})] / (12 h),
 * indices wrapped periodically (Section 3 boundary conditions). */
void or_d1(const double* f, int nx, int ny, int nz, int axis, double h, double* out) {
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double fm2, fm1, fp1, fp2;
                if (axis == 0) {
                    fm2 = f[at(nx, ny, wrap(x - 2, nx), y, z)];
                    fm1 = f[at(nx, ny, wrap(x - 1, nx), y, z)];
                    fp1 = f[at(nx, ny, wrap(x + 1, nx), y, z)];
                    fp2 = f[at(nx, ny, wrap(x + 2, nx), y, z)];
                } else if (axis == 1) {
                    fm2 = f[at(nx, ny, x, wrap(y - 2, ny), z)];
                    fm1 = f[at(nx, ny, x, wrap(y - 1, ny), z)];
                    fp1 = f[at(nx, ny, x, wrap(y + 1, ny), z)];
                    fp2 = f[at(nx, ny, x, wrap(y + 2, ny), z)];
                } else {
                    fm2 = f[at(nx, ny, x, y, wrap(z - 2, nz))];
                    fm1 = f[at(nx, ny, x, y, wrap(z - 1, nz))];
                    fp1 = f[at(nx, ny, x, y, wrap(z + 1, nz))];
                    fp2 = f[at(nx, ny, x, y, wrap(z + 2, nz))];
                }
                out[at(nx, ny, x, y, z)] =
                    (8.0 * (fp1 - fm1) - (fp2 - fm2)) / (12.0 * h);
            }
}

/* Pure second derivative along `axis` with spacing h:
 *   D2 f_i = [-f_{i-2} + 16 f_{i-1} - 30 f_i + 16 f_{i+1} - f_{i+2}] / (12 h^2). */
void or_d2(const double* f, int nx, int ny, int nz, int axis, double h, double* out) {
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double fm2, fm1, fp1, fp2;
                double f0 = f[at(nx, ny, x, y, z)];
                if (axis == 0) {
                    fm2 = f[at(nx, ny, wrap(x - 2, nx), y, z)];
                    fm1 = f[at(nx, ny, wrap(x - 1, nx), y, z)];
                    fp1 = f[at(nx, ny, wrap(x + 1, nx), y, z)];
                    fp2 = f[at(nx, ny, wrap(x + 2, nx), y, z)];
                } else if (axis == 1) {
                    fm2 = f[at(nx, ny, x, wrap(y - 2, ny), z)];
                    fm1 = f[at(nx, ny, x, wrap(y - 1, ny), z)];
                    fp1 = f[at(nx, ny, x, wrap(y + 1, ny), z)];
                    fp2 = f[at(nx, ny, x, wrap(y + 2, ny), z)];
                } else {
                    fm2 = f[at(nx, ny, x, y, wrap(z - 2, nz))];
                    fm1 = f[at(nx, ny, x, y, wrap(z - 1, nz))];
                    fp1 = f[at(nx, ny, x, y, wrap(z + 1, nz))];
                    fp2 = f[at(nx, ny, x, y, wrap(z + 2, nz))];
                }
                out[at(nx, ny, x, y, z)] =
                    (-fm2 + 16.0 * fm1 - 30.0 * f0 + 16.0 * fp1 - fp2) / (12.0 * h * h);
            }
}

/* ---- Section 3: Taylor-Green vortex initial condition ------------------- */

/* u = sin x cos y cos z, v = -cos x sin y cos z, w = 0,
 * p = 1/(gamma M^2) + (cos 2x + cos 2y)(cos 2z + 2)/16, rho = gamma M^2 p,
 * rho E = p/(gamma-1) + rho |u|^2 / 2 (DeBonis 2013, cited in Section 3).
 * Q is [var][z][y][x], var = rho, rho u, rho v, rho w, rho E. */
void or_tgv_ic(int nx, int ny, int nz, double gamma, double mach, double* Q) {
    long n = npts(nx, ny, nz);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double x = i * (2.0 * OR_PI / nx);
                double y = j * (2.0 * OR_PI / ny);
                double z = k * (2.0 * OR_PI / nz);
                double u = sin(x) * cos(y) * cos(z);
                double v = -cos(x) * sin(y) * cos(z);
                double w = 0.0;
                double p = 1.0 / (gamma * mach * mach) +
                           (cos(2.0 * x) + cos(2.0 * y)) * (cos(2.0 * z) + 2.0) / 16.0;
                double rho = gamma * mach * mach * p;
                long q = at(nx, ny, i, j, k);
                Q[0 * n + q] = rho;
                Q[1 * n + q] = rho * u;
                Q[2 * n + q] = rho * v;
                Q[3 * n + q] = rho * w;
                Q[4 * n + q] = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w);
            }
}

/* ---- Section 2, Eqs. 6-7: primitive variables ---------------------------- */

/* u_i = (rho u_i)/rho, p = (gamma-1)(rho E - rho u_j u_j / 2),
 * T = gamma M^2 p / rho.  prim is [5][n]: u, v, w, p, T. */
void or_primitives(int nx, int ny, int nz, double gamma, double mach,
                   const double* Q, double* prim) {
    long n = npts(nx, ny, nz);
#pragma omp parallel for schedule(static)
    for (long q = 0; q < n; ++q) {
        double rho = Q[q];
        double u = Q[1 * n + q] / rho;
        double v = Q[2 * n + q] / rho;
        double w = Q[3 * n + q] / rho;
        double p = (gamma - 1.0) * (Q[4 * n + q] - 0.5 * rho * (u * u + v * v + w * w));
        prim[0 * n + q] = u;
        prim[1 * n + q] = v;
        prim[2 * n + q] = w;
        prim[3 * n + q] = p;
        prim[4 * n + q] = gamma * mach * mach * p / rho;
    }
}

/* ---- Section 2, Eqs. 1-5 with Eq. skewscalar: the residual -------------- */

/* R = right-hand sides of the mass, momentum and energy equations, [5][n]:
 *
 *  R_rho   = -1/2 sum_j [ D_j(rho u_j) + u_j D_j rho + rho D_j u_j ]
 *  R_rhoui = -1/2 sum_j [ D_j(rho u_i u_j) + u_j D_j(rho u_i) + rho u_i D_j u_j ]
 *            - D_i p + sum_j D_j tau_ij
 *  R_rhoE  = -1/2 sum_j [ D_j(rho E u_j) + u_j D_j(rho E) + rho E D_j u_j ]
 *            - sum_j D_j(u_j p) + sum_j D_j q_j + sum_j D_j(u_i tau_ij)
 *
 * with tau_ij = (1/Re)(D_j u_i + D_i u_j - 2/3 delta_ij D_k u_k) (Eq. 4),
 * q_j = D_j T / ((gamma-1) M^2 Pr Re) (Eq. 5), and the viscous divergences
 * expanded into second derivatives:
 *   sum_j D_j tau_ij = (1/Re)[ sum_j D2_j u_i + 1/3 sum_k D_ik u_k ],
 *   sum_j D_j q_j    = sum_j D2_j T / ((gamma-1) M^2 Pr Re),
 *   sum_j D_j(u_i tau_ij) = tau_ij D_j u_i + u_i sum_j D_j tau_ij,
 * where D_ii u_i is the pure second derivative D2_i and D_ik (i != k) is
 * D_i applied to D_k u_k. */
void or_residual(const or_params* P, const double* Q, double* R) {
    int nx = P->nx, ny = P->ny, nz = P->nz;
    long n = npts(nx, ny, nz);
    const double h[3] = {P->hx, P->hy, P->hz};
    double nu = 1.0 / P->Re;
    double kappa = 1.0 / ((P->gamma - 1.0) * P->Mach * P->Mach * P->Pr * P->Re);

    double* prim = malloc(sizeof(double) * 5 * n);
    double* G = malloc(sizeof(double) * 9 * n);   /* G[3*i+j] = D_j u_i */
    double* work = malloc(sizeof(double) * n);    /* product work array */
    double* d = malloc(sizeof(double) * n);       /* derivative work array */
    double* d2 = malloc(sizeof(double) * n);      /* second derivative work array */
    double* visc = malloc(sizeof(double) * n);    /* sum_j D_j tau_ij for one i */

    /* evaluate-u_i,p,T (Fig. 1) */
    or_primitives(nx, ny, nz, P->gamma, P->Mach, Q, prim);
    const double* u[3] = {prim, prim + n, prim + 2 * n};
    const double* p = prim + 3 * n;
    const double* T = prim + 4 * n;

    /* velocity gradients G_ij = D_j u_i */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) or_d1(u[i], nx, ny, nz, j, h[j], G + (3 * i + j) * n);

    memset(R, 0, sizeof(double) * 5 * n);

    /* 1. skew-symmetric convective terms (Eq. skewscalar), phi = 1, u_i, E:
     *    rho*phi is the conservative variable Q[f] itself. */
    for (int f = 0; f < 5; ++f) {
        const double* rphi = Q + f * n;
        double* Rf = R + f * n;
        for (int j = 0; j < 3; ++j) {
            const double* divj = G + (3 * j + j) * n; /* D_j u_j */
            for (long q = 0; q < n; ++q) work[q] = rphi[q] * u[j][q];
            or_d1(work, nx, ny, nz, j, h[j], d);   /* D_j(rho phi u_j) */
            or_d1(rphi, nx, ny, nz, j, h[j], d2);  /* D_j(rho phi)     */
            for (long q = 0; q < n; ++q)
                Rf[q] -= 0.5 * (d[q] + u[j][q] * d2[q] + rphi[q] * divj[q]);
        }
    }

    /* 2. pressure gradient in the momentum equations: -D_i p (Eq. 2) */
    for (int i = 0; i < 3; ++i) {
        or_d1(p, nx, ny, nz, i, h[i], d);
        double* Rm = R + (1 + i) * n;
        for (long q = 0; q < n; ++q) Rm[q] -= d[q];
    }

    /* 3. pressure work in the energy equation: -D_j(u_j p) (Eq. 3) */
    for (int j = 0; j < 3; ++j) {
        for (long q = 0; q < n; ++q) work[q] = u[j][q] * p[q];
        or_d1(work, nx, ny, nz, j, h[j], d);
        double* RE = R + 4 * n;
        for (long q = 0; q < n; ++q) RE[q] -= d[q];
    }

    /* 4. viscous stress divergence (Eq. 4, expanded) in momentum, and the
     *    work term u_i * sum_j D_j tau_ij in energy (Eq. 3) */
    for (int i = 0; i < 3; ++i) {
        memset(visc, 0, sizeof(double) * n);
        for (int j = 0; j < 3; ++j) { /* sum_j D2_j u_i */
            or_d2(u[i], nx, ny, nz, j, h[j], d2);
            for (long q = 0; q < n; ++q) visc[q] += d2[q];
        }
        for (int k = 0; k < 3; ++k) { /* 1/3 sum_k D_ik u_k */
            if (k == i)
                or_d2(u[i], nx, ny, nz, i, h[i], d2);
            else
                or_d1(G + (3 * k + k) * n, nx, ny, nz, i, h[i], d2);
            for (long q = 0; q < n; ++q) visc[q] += d2[q] / 3.0;
        }
        double* Rm = R + (1 + i) * n;
        double* RE = R + 4 * n;
        for (long q = 0; q < n; ++q) {
            Rm[q] += nu * visc[q];
            RE[q] += u[i][q] * (nu * visc[q]);
        }
    }

    /* 5. viscous dissipation tau_ij D_j u_i in energy (Eq. 3 with Eq. 4) */
    {
        double* RE = R + 4 * n;
        for (long q = 0; q < n; ++q) {
            double dk = G[0 * n + q] + G[4 * n + q] + G[8 * n + q];
            double s = 0.0;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    double tau = nu * (G[(3 * i + j) * n + q] + G[(3 * j + i) * n + q] -
                                       (i == j ? 2.0 / 3.0 * dk : 0.0));
                    s += tau * G[(3 * i + j) * n + q];
                }
            RE[q] += s;
        }
    }

    /* 6. heat flux divergence sum_j D_j q_j (Eq. 5) */
    for (int j = 0; j < 3; ++j) {
        or_d2(T, nx, ny, nz, j, h[j], d2);
        double* RE = R + 4 * n;
        for (long q = 0; q < n; ++q) RE[q] += kappa * d2[q];
    }

    free(prim); free(G); free(work); free(d); free(d2); free(visc);
}

/* ---- Section 2 / Fig. 1: low-storage three-stage Runge-Kutta ------------- */

/* Two-register coefficients: Q <- Qs + A[s] dt R, Qs <- Qs + B[s] dt R. */
static const double OR_RK_A[3] = {2.0 / 3.0, 5.0 / 12.0, 3.0 / 5.0};
static const double OR_RK_B[3] = {1.0 / 4.0, 3.0 / 20.0, 0.0};

void or_rk_coefficients(double* a, double* b) {
    for (int s = 0; s < 3; ++s) { a[s] = OR_RK_A[s]; b[s] = OR_RK_B[s]; }
}

/* advance-solution-in-time for stage s (0, 1, 2) given the residual R. */
void or_rk_update(long n, int s, double dt, const double* R, double* Q, double* Qs) {
#pragma omp parallel for schedule(static)
    for (long q = 0; q < n; ++q) {
        double qs = Qs[q];
        Q[q] = qs + OR_RK_A[s] * dt * R[q];
        if (s < 2) Qs[q] = qs + OR_RK_B[s] * dt * R[q];
    }
}

typedef void (*or_rhs_fn)(void* ctx, const double* Q, double* R);

/* One time step of Fig. 1 for a generic right-hand side over n unknowns:
 * save-state, then three stages of (residual, update).  Qs and R are
 * caller-provided work arrays of n doubles. */
void or_lsrk3_step(long n, double dt, double* Q, double* Qs, double* R,
                   or_rhs_fn rhs, void* ctx) {
    memcpy(Qs, Q, sizeof(double) * n); /* save-state */
    for (int s = 0; s < 3; ++s) {
        rhs(ctx, Q, R);
        or_rk_update(n, s, dt, R, Q, Qs);
    }
}

static void ns_rhs(void* ctx, const double* Q, double* R) {
    or_residual((const or_params*)ctx, Q, R);
}

/* Run `nsteps` full RK3 steps of the Navier-Stokes system in place on Q
 * ([5][nz][ny][nx]).  Periodic boundary conditions are implied by the
 * wrapped stencils.  Returns 0, or -1 if memory could not be allocated. */
int or_run(const or_params* P, double* Q, int nsteps) {
    long n5 = 5 * npts(P->nx, P->ny, P->nz);
    double* Qs = malloc(sizeof(double) * n5);
    double* R = malloc(sizeof(double) * n5);
    if (!Qs || !R) { free(Qs); free(R); return -1; }
    for (int it = 0; it < nsteps; ++it)
        or_lsrk3_step(n5, P->dt, Q, Qs, R, ns_rhs, (void*)P);
    free(Qs); free(R);
    return 0;
}

/* ---- Section 3: kinetic energy and enstrophy ----------------------------- */

/* ke  = (1/N) sum rho |u|^2 / 2
 * ens = (1/N) sum rho |omega|^2 / 2, omega = curl u with the first-derivative
 * operator above.  Sums are taken per z-plane, then over planes in order. */
void or_diagnostics(int nx, int ny, int nz, const double* Q, double* ke, double* ens) {
    long n = npts(nx, ny, nz);
    long plane = (long)nx * ny;
    double* uvw = malloc(sizeof(double) * 3 * n);
    double* G = malloc(sizeof(double) * 9 * n);
    double* ske = malloc(sizeof(double) * nz);
    double* sen = malloc(sizeof(double) * nz);
    const double h[3] = {2.0 * OR_PI / nx, 2.0 * OR_PI / ny, 2.0 * OR_PI / nz};
    for (long q = 0; q < n; ++q) {
        uvw[q] = Q[n + q] / Q[q];
        uvw[n + q] = Q[2 * n + q] / Q[q];
        uvw[2 * n + q] = Q[3 * n + q] / Q[q];
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) or_d1(uvw + i * n, nx, ny, nz, j, h[j], G + (3 * i + j) * n);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z) {
        double a = 0.0, b = 0.0;
        for (long q = z * plane; q < (z + 1) * plane; ++q) {
            double rho = Q[q];
            double u = uvw[q], v = uvw[n + q], w = uvw[2 * n + q];
            double ox = G[(3 * 2 + 1) * n + q] - G[(3 * 1 + 2) * n + q]; /* Dy w - Dz v */
            double oy = G[(3 * 0 + 2) * n + q] - G[(3 * 2 + 0) * n + q]; /* Dz u - Dx w */
            double oz = G[(3 * 1 + 0) * n + q] - G[(3 * 0 + 1) * n + q]; /* Dx v - Dy u */
            a += 0.5 * rho * (u * u + v * v + w * w);
            b += 0.5 * rho * (ox * ox + oy * oy + oz * oz);
        }
        ske[z] = a;
        sen[z] = b;
    }
    double a = 0.0, b = 0.0;
    for (int z = 0; z < nz; ++z) { a += ske[z]; b += sen[z]; }
    *ke = a / (double)n;
    *ens = b / (double)n;
    free(uvw); free(G); free(ske); free(sen);
}
