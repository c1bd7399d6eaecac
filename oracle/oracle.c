/*
 * FP64 CPU oracle for RBF semi-Lagrangian transport on the unit sphere
 * (Shankar & Wright, "Mesh-free semi-Lagrangian methods for transport on a sphere
 * using radial basis functions").
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously-correct reference that
 * the CUDA path is checked against. Only the tests, the smoke check and the bench's CPU
 * baseline may load it. It shares no code, header, table or constant with the CUDA library.
 *
 * Compiled with -ffp-contract=off so that every product and sum is rounded on its own:
 * the squared distance used as the k-NN key is exactly ((dx*dx + dy*dy) + dz*dz).
 *
 * Every function cites the passage of the paper it follows. Readings of the paper where it
 * is silent or ambiguous are listed in the design notes; the ones that shape this file:
 *  - RK4 with an orthogonal projection onto S^2 at every stage and of the result (Sec. 3.2);
 *  - PHS kernel r^p (p odd), real orthonormal spherical harmonics ordered degree-major,
 *    order m = -l..l (Sec. 2.2, Eq. rbf_poly);
 *  - Gaussian elimination with partial pivoting; a pivot tie goes to the smaller row index;
 *  - k-NN key (d^2, index) compared lexicographically.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

void orc_set_threads(int n) {
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
#else
    (void)n;
#endif
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ velocity fields */
/* kind 0: solid-body rotation u = omega (a x x); prm = {a_x, a_y, a_z, omega}
 *         (Williamson test case 1 is this field with a = (0, -sin alpha, -cos alpha), Sec. 4.1).
 * kind 1: reversing deformation, stream function psi = kappa y^2 cos(pi t / T_f);
 *         u = x cross grad(psi) = g (-z, 0, x), g = 2 kappa y cos(pi t / T_f); prm = {kappa, T_f}.
 *         Tangent and divergence-free on S^2 (the transport equation, Sec. 1). */
void orc_velocity(int kind, const double *prm, const double *x, double t, double *u) {
    if (kind == 0) {
        double w0 = prm[3] * prm[0], w1 = prm[3] * prm[1], w2 = prm[3] * prm[2];
        u[0] = w1 * x[2] - w2 * x[1];
        u[1] = w2 * x[0] - w0 * x[2];
        u[2] = w0 * x[1] - w1 * x[0];
    } else if (kind == 1) {
        double g = 2.0 * prm[0] * x[1] * cos(ORC_PI * t / prm[1]);
        u[0] = -g * x[2];
        u[1] = 0.0;
        u[2] = g * x[0];
    } else {
        /* Deformational flow of Sec. 4.2 (prm = {kappa, T}) in the paper's spherical form,
         * lambda = longitude, theta = latitude, lp = lambda - 2 pi t / T:
         *   u = kappa cos(pi t / T) sin^2(lp) sin(2 theta) + (2 pi / T) cos(theta)
         *   v = kappa cos(pi t / T) sin(2 lp) cos(theta)
         * converted to Cartesian with e_lambda = (-sin l, cos l, 0) and
         * e_theta = (-sin th cos l, -sin th sin l, cos th). */
        const double T = prm[1];
        const double lam = atan2(x[1], x[0]);
        const double th = atan2(x[2], sqrt(x[0] * x[0] + x[1] * x[1]));
        const double k = prm[0] * cos(ORC_PI * t / T);
        const double lp = lam - 2.0 * ORC_PI * t / T;
        const double uu = k * sin(lp) * sin(lp) * sin(2.0 * th) + 2.0 * ORC_PI / T * cos(th);
        const double vv = k * sin(2.0 * lp) * cos(th);
        const double sl = sin(lam), cl = cos(lam), st = sin(th), ct = cos(th);
        u[0] = -uu * sl - vv * st * cl;
        u[1] = uu * cl - vv * st * sl;
        u[2] = vv * ct;
    }
}

static void project(double *y) {
    double r = sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
    y[0] /= r; y[1] /= r; y[2] /= r;
}

/* Departure points (Eq. sl_ode, Sec. 3.2): integrate d xi/dt = u backward from
 * (x_j, t1) over one step dt with classical RK4, h = -dt, projecting every stage point
 * and the result orthogonally onto S^2. X, Xi: N x 3 row-major. */
void orc_trace_rk4(int kind, const double *prm, const double *X, int64_t N, double t1,
                   double dt, double *Xi) {
    const double h = -dt;
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < N; ++j) {
        const double *x = X + 3 * j;
        double k1[3], k2[3], k3[3], k4[3], y[3];
        orc_velocity(kind, prm, x, t1, k1);
        for (int d = 0; d < 3; ++d) y[d] = x[d] + 0.5 * h * k1[d];
        project(y);
        orc_velocity(kind, prm, y, t1 + 0.5 * h, k2);
        for (int d = 0; d < 3; ++d) y[d] = x[d] + 0.5 * h * k2[d];
        project(y);
        orc_velocity(kind, prm, y, t1 + 0.5 * h, k3);
        for (int d = 0; d < 3; ++d) y[d] = x[d] + h * k3[d];
        project(y);
        orc_velocity(kind, prm, y, t1 + h, k4);
        double *xi = Xi + 3 * j;
        for (int d = 0; d < 3; ++d)
            xi[d] = x[d] + (h / 6.0) * (k1[d] + 2.0 * k2[d] + 2.0 * k3[d] + k4[d]);
        project(xi);
    }
}

/* The same step with Fehlberg's fifth-order Runge-Kutta formula (the paper's final integrator
 * choice, Sec. 3.2): six stages, nodes c = (0, 1/4, 3/8, 12/13, 1, 1/2), the published
 * coupling coefficients a_ij and the fifth-order weights b = (16/135, 0, 6656/12825,
 * 28561/56430, -9/50, 2/55). Stage point i is x + h sum_j a_ij k_j, projected onto S^2 before
 * u is evaluated there at t1 + c_i h; the result x + h sum_i b_i k_i is projected too. */
void orc_trace_rk5(int kind, const double *prm, const double *X, int64_t N, double t1,
                   double dt, double *Xi) {
    static const double c[6] = {0.0, 1.0 / 4.0, 3.0 / 8.0, 12.0 / 13.0, 1.0, 1.0 / 2.0};
    static const double a[6][5] = {
        {0, 0, 0, 0, 0},
        {1.0 / 4.0, 0, 0, 0, 0},
        {3.0 / 32.0, 9.0 / 32.0, 0, 0, 0},
        {1932.0 / 2197.0, -7200.0 / 2197.0, 7296.0 / 2197.0, 0, 0},
        {439.0 / 216.0, -8.0, 3680.0 / 513.0, -845.0 / 4104.0, 0},
        {-8.0 / 27.0, 2.0, -3544.0 / 2565.0, 1859.0 / 4104.0, -11.0 / 40.0}};
    static const double b[6] = {16.0 / 135.0, 0.0, 6656.0 / 12825.0, 28561.0 / 56430.0, -9.0 / 50.0, 2.0 / 55.0};
    const double h = -dt;
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < N; ++j) {
        const double *x = X + 3 * j;
        double k[6][3], y[3];
        for (int i = 0; i < 6; ++i) {
            for (int d = 0; d < 3; ++d) {
                double s = 0.0;
                for (int q = 0; q < i; ++q) s += a[i][q] * k[q][d];
                y[d] = x[d] + h * s;
            }
            if (i > 0) project(y);
            orc_velocity(kind, prm, y, t1 + c[i] * h, k[i]);
        }
        double *xi = Xi + 3 * j;
        for (int d = 0; d < 3; ++d) {
            double s = 0.0;
            for (int i = 0; i < 6; ++i) s += b[i] * k[i][d];
            xi[d] = x[d] + h * s;
        }
        project(xi);
    }
}

/* ------------------------------------------------------------------ brute-force k-NN */
/* The kd-tree of Sec. 3.3 returns the k nearest nodes; here every node is tested.
 * Key (d2, j) with d2 = ((qx-xx)^2 + (qy-xy)^2) + (qz-xz)^2, each operation rounded.
 * Output idx[q*k + r] ascending by key. d2out may be NULL. */
static inline double sqdist(const double *a, const double *b) {
    double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    double s = dx * dx;
    s = s + dy * dy;
    s = s + dz * dz;
    return s;
}

static inline int key_less(double da, int32_t ia, double db, int32_t ib) {
    return da < db || (da == db && ia < ib);
}

void orc_knn(const double *X, int64_t N, const double *Q, int64_t Nq, int k, int32_t *idx,
             double *d2out) {
#pragma omp parallel
    {
        double *bd = (double *)malloc(sizeof(double) * (size_t)k);
        int32_t *bi = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
#pragma omp for schedule(static)
        for (int64_t q = 0; q < Nq; ++q) {
            int cnt = 0;
            for (int64_t j = 0; j < N; ++j) {
                double d = sqdist(Q + 3 * q, X + 3 * j);
                int32_t jj = (int32_t)j;
                if (cnt == k && !key_less(d, jj, bd[k - 1], bi[k - 1])) continue;
                int pos = cnt < k ? cnt : k - 1; /* insertion sort into the sorted list */
                while (pos > 0 && key_less(d, jj, bd[pos - 1], bi[pos - 1])) {
                    bd[pos] = bd[pos - 1]; bi[pos] = bi[pos - 1]; --pos;
                }
                bd[pos] = d; bi[pos] = jj;
                if (cnt < k) ++cnt;
            }
            for (int r = 0; r < k; ++r) {
                idx[q * k + r] = r < cnt ? bi[r] : -1;
                if (d2out) d2out[q * k + r] = r < cnt ? bd[r] : INFINITY;
            }
        }
        free(bd); free(bi);
    }
}

/* ------------------------------------------------------------------ spherical harmonics */
/* Real orthonormal spherical harmonics of degree <= L at the unit vector x, written as
 * polynomials in (x, y, z) (Sec. 2.2: the augmentation basis {p_i}, (L+1)^2 functions).
 * Y[l*l + l + m], m = -l..l. With z = cos(theta) and x + iy = sin(theta) e^{i phi}:
 *   Y_l^0  = N_l0 Q_l^0(z)
 *   Y_l^m  = sqrt2 N_lm Q_l^m(z) Re (x+iy)^m,   Y_l^-m = sqrt2 N_lm Q_l^m(z) Im (x+iy)^m
 * where P_l^m(z) = (1-z^2)^{m/2} Q_l^m(z) (no Condon-Shortley phase),
 * N_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), Q_m^m = (2m-1)!!, Q_{m+1}^m = (2m+1) z Q_m^m,
 * (l-m) Q_l^m = (2l-1) z Q_{l-1}^m - (l+m-1) Q_{l-2}^m. */
void orc_sh_eval(int L, const double *x, double *Y) {
    double cm = 1.0, sm = 0.0; /* Re, Im of (x+iy)^m */
    for (int m = 0; m <= L; ++m) {
        if (m > 0) {
            double c2 = cm * x[0] - sm * x[1];
            double s2 = cm * x[1] + sm * x[0];
            cm = c2; sm = s2;
        }
        double qmm = 1.0;
        for (int i = 1; i <= m; ++i) qmm *= (double)(2 * i - 1);
        double qlm2 = 0.0, qlm1 = 0.0;
        for (int l = m; l <= L; ++l) {
            double qlm;
            if (l == m) qlm = qmm;
            else if (l == m + 1) qlm = (double)(2 * m + 1) * x[2] * qmm;
            else qlm = ((double)(2 * l - 1) * x[2] * qlm1 - (double)(l + m - 1) * qlm2) / (double)(l - m);
            /* (l-m)!/(l+m)! */
            double ratio = 1.0;
            for (int i = l - m + 1; i <= l + m; ++i) ratio /= (double)i;
            double nlm = sqrt((2.0 * l + 1.0) / (4.0 * ORC_PI) * ratio);
            if (m == 0) {
                Y[l * l + l] = nlm * qlm;
            } else {
                Y[l * l + l + m] = sqrt(2.0) * nlm * qlm * cm;
                Y[l * l + l - m] = sqrt(2.0) * nlm * qlm * sm;
            }
            qlm2 = qlm1; qlm1 = qlm;
        }
    }
}

/* ------------------------------------------------------------------ dense GEPP */
/* Gaussian elimination with partial pivoting on the m x m row-major A with nrhs right-hand
 * sides B (m x nrhs row-major), in place; B becomes the solution. The pivot is the entry of
 * largest magnitude in the column, the smaller row index on a tie. Returns 0, or -1 on an
 * exactly zero or non-finite pivot. (Sec. 3.3: the stencil systems are solved by LU.) */
int orc_gepp_solve(double *A, int m, double *B, int nrhs) {
    for (int k = 0; k < m; ++k) {
        int p = k;
        double best = fabs(A[(size_t)k * m + k]);
        for (int i = k + 1; i < m; ++i) {
            double v = fabs(A[(size_t)i * m + k]);
            if (v > best) { best = v; p = i; }
        }
        if (!(best > 0.0) || !isfinite(best)) return -1;
        if (p != k) {
            for (int j = 0; j < m; ++j) {
                double t = A[(size_t)k * m + j]; A[(size_t)k * m + j] = A[(size_t)p * m + j]; A[(size_t)p * m + j] = t;
            }
            for (int r = 0; r < nrhs; ++r) {
                double t = B[(size_t)k * nrhs + r]; B[(size_t)k * nrhs + r] = B[(size_t)p * nrhs + r]; B[(size_t)p * nrhs + r] = t;
            }
        }
        double piv = A[(size_t)k * m + k];
        for (int i = k + 1; i < m; ++i) {
            double l = A[(size_t)i * m + k] / piv;
            if (l == 0.0) continue;
            for (int j = k + 1; j < m; ++j) A[(size_t)i * m + j] -= l * A[(size_t)k * m + j];
            for (int r = 0; r < nrhs; ++r) B[(size_t)i * nrhs + r] -= l * B[(size_t)k * nrhs + r];
        }
    }
    for (int i = m - 1; i >= 0; --i) {
        for (int r = 0; r < nrhs; ++r) {
            double s = B[(size_t)i * nrhs + r];
            for (int j = i + 1; j < m; ++j) s -= A[(size_t)i * m + j] * B[(size_t)j * nrhs + r];
            B[(size_t)i * nrhs + r] = s / A[(size_t)i * m + i];
        }
    }
    return 0;
}

/* LU factorisation with partial pivoting, in place (row-major, L unit-lower below the
 * diagonal, U on and above); piv[k] = row swapped with k at step k. Returns 0 or -1. */
int orc_lu_factor(double *A, int64_t m, int32_t *piv) {
    for (int64_t k = 0; k < m; ++k) {
        int64_t p = k;
        double best = fabs(A[k * m + k]);
        for (int64_t i = k + 1; i < m; ++i) {
            double v = fabs(A[i * m + k]);
            if (v > best) { best = v; p = i; }
        }
        piv[k] = (int32_t)p;
        if (!(best > 0.0) || !isfinite(best)) return -1;
        if (p != k)
            for (int64_t j = 0; j < m; ++j) {
                double t = A[k * m + j]; A[k * m + j] = A[p * m + j]; A[p * m + j] = t;
            }
        double piv_v = A[k * m + k];
#pragma omp parallel for schedule(static) if (m - k > 256)
        for (int64_t i = k + 1; i < m; ++i) {
            double l = A[i * m + k] / piv_v;
            A[i * m + k] = l;
            if (l == 0.0) continue;
            for (int64_t j = k + 1; j < m; ++j) A[i * m + j] -= l * A[k * m + j];
        }
    }
    return 0;
}

/* Solve with the factor of orc_lu_factor: B (m x nrhs row-major) overwritten with A^-1 B. */
void orc_lu_solve(const double *LU, const int32_t *piv, int64_t m, double *B, int nrhs) {
    for (int64_t k = 0; k < m; ++k)
        if (piv[k] != k)
            for (int r = 0; r < nrhs; ++r) {
                double t = B[k * nrhs + r]; B[k * nrhs + r] = B[(int64_t)piv[k] * nrhs + r]; B[(int64_t)piv[k] * nrhs + r] = t;
            }
#pragma omp parallel for schedule(static)
    for (int r = 0; r < nrhs; ++r) {
        for (int64_t i = 0; i < m; ++i) {
            double s = B[i * nrhs + r];
            for (int64_t j = 0; j < i; ++j) s -= LU[i * m + j] * B[j * nrhs + r];
            B[i * nrhs + r] = s;
        }
        for (int64_t i = m - 1; i >= 0; --i) {
            double s = B[i * nrhs + r];
            for (int64_t j = i + 1; j < m; ++j) s -= LU[i * m + j] * B[j * nrhs + r];
            B[i * nrhs + r] = s / LU[i * m + i];
        }
    }
}

/* Cholesky A = L L^T of the symmetric m x m matrix, lower triangle overwritten (the global
 * method's factorisation, Sec. 3.3). Returns 0, or -1 at the first non-positive pivot. */
int orc_cholesky(double *A, int64_t m) {
    for (int64_t j = 0; j < m; ++j) {
        double d = A[j * m + j];
        for (int64_t k = 0; k < j; ++k) d -= A[j * m + k] * A[j * m + k];
        if (!(d > 0.0)) return -1;
        d = sqrt(d);
        A[j * m + j] = d;
#pragma omp parallel for schedule(static) if (m - j > 256)
        for (int64_t i = j + 1; i < m; ++i) {
            double s = A[i * m + j];
            for (int64_t k = 0; k < j; ++k) s -= A[i * m + k] * A[j * m + k];
            A[i * m + j] = s / d;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ radial kernels */
/* kind 0: polyharmonic spline r^p, p odd (Sec. 2.4), as r * (r^2)^((p-1)/2);
 * kind 1: Gaussian exp(-(eps r)^2); kind 2: inverse multiquadric (1 + (eps r)^2)^(-1/2). */
static inline double kernel_of_d2(int kind, double prm, double d2) {
    if (kind == 0) {
        int p = (int)prm;
        double r = sqrt(d2), v = r;
        for (int i = 0; i < (p - 1) / 2; ++i) v *= d2;
        return v;
    } else if (kind == 1) {
        return exp(-(prm * prm) * d2);
    } else {
        return 1.0 / sqrt(1.0 + (prm * prm) * d2);
    }
}

double orc_kernel(int kind, double prm, double r) { return kernel_of_d2(kind, prm, r * r); }

/* ------------------------------------------------------------------ local stencil weights */
/* Interpolation weights of the augmented local RBF interpolant (Eqs. rbf_poly and
 * rbf_poly_linsys) on the stencil I[0..n) at the point xi:
 *   [[A, P], [P^T, 0]] w~ = [phi(|xi - x_Ij|)_j ; p(xi)],  w = w~[0:n],
 * A_ij = phi(|x_Ii - x_Ij|), P_ij = p_j(x_Ii). Because the saddle-point matrix is symmetric,
 * s(xi) = b^T c~ = sum_j w_j q_Ij, with c~ the coefficients of Eq. rbf_poly_linsys.
 * Returns 0, or -1 if the elimination met a zero pivot. */
int orc_stencil_weights(const double *X, const int32_t *I, int n, int L, int kkind, double kprm,
                        const double *xi, double *w) {
    int M = (L + 1) * (L + 1), m = n + M;
    double *A = (double *)calloc((size_t)m * m, sizeof(double));
    double *b = (double *)malloc(sizeof(double) * (size_t)m);
    double *Y = (double *)malloc(sizeof(double) * (size_t)M);
    for (int i = 0; i < n; ++i) {
        const double *xa = X + 3 * (int64_t)I[i];
        for (int j = 0; j < n; ++j)
            A[(size_t)i * m + j] = kernel_of_d2(kkind, kprm, sqdist(xa, X + 3 * (int64_t)I[j]));
        orc_sh_eval(L, xa, Y);
        for (int c = 0; c < M; ++c) {
            A[(size_t)i * m + n + c] = Y[c];
            A[(size_t)(n + c) * m + i] = Y[c];
        }
        b[i] = kernel_of_d2(kkind, kprm, sqdist(xi, xa));
    }
    orc_sh_eval(L, xi, Y);
    for (int c = 0; c < M; ++c) b[n + c] = Y[c];
    int rc = orc_gepp_solve(A, m, b, 1);
    for (int i = 0; i < n; ++i) w[i] = b[i];
    free(A); free(b); free(Y);
    return rc;
}

/* ------------------------------------------------------------------ extended-precision referee */
/* The same stencil system (Eqs. rbf_poly and rbf_poly_linsys) assembled and solved in long double,
 * as a referee for FP64 weights whose system is too ill-conditioned for FP64 to fix them
 * (condition numbers near 1e18 at n = 84, ell = 4). The node coordinates are the FP64 inputs,
 * converted exactly; the kernel r^p, the harmonics and Gaussian elimination with partial
 * pivoting are the double-precision steps above written in long double. long double is IEEE
 * binary128 (113-bit significand) on aarch64 Linux and x87 extended (64 bits) on x86-64:
 * orc_long_double_digits reports which. PHS kernel only. */
int orc_long_double_digits(void) { return LDBL_MANT_DIG; }

static void sh_eval_ld(int L, const long double *x, long double *Y) {
    long double cm = 1.0L, sm = 0.0L;
    for (int m = 0; m <= L; ++m) {
        if (m > 0) {
            long double c2 = cm * x[0] - sm * x[1];
            long double s2 = cm * x[1] + sm * x[0];
            cm = c2; sm = s2;
        }
        long double qmm = 1.0L;
        for (int i = 1; i <= m; ++i) qmm *= (long double)(2 * i - 1);
        long double qlm2 = 0.0L, qlm1 = 0.0L;
        for (int l = m; l <= L; ++l) {
            long double qlm;
            if (l == m) qlm = qmm;
            else if (l == m + 1) qlm = (long double)(2 * m + 1) * x[2] * qmm;
            else qlm = ((long double)(2 * l - 1) * x[2] * qlm1 - (long double)(l + m - 1) * qlm2) / (long double)(l - m);
            long double ratio = 1.0L;
            for (int i = l - m + 1; i <= l + m; ++i) ratio /= (long double)i;
            long double nlm = sqrtl((2.0L * l + 1.0L) / (4.0L * acosl(-1.0L)) * ratio);
            if (m == 0) {
                Y[l * l + l] = nlm * qlm;
            } else {
                Y[l * l + l + m] = sqrtl(2.0L) * nlm * qlm * cm;
                Y[l * l + l - m] = sqrtl(2.0L) * nlm * qlm * sm;
            }
            qlm2 = qlm1; qlm1 = qlm;
        }
    }
}

static long double phs_ld(int p, const long double *a, const long double *b) {
    long double d2 = 0.0L;
    for (int c = 0; c < 3; ++c) d2 += (a[c] - b[c]) * (a[c] - b[c]);
    long double v = sqrtl(d2);
    for (int i = 0; i < (p - 1) / 2; ++i) v *= d2;
    return v;
}

/* Weights of Nq stencils: I (Nq x n), points Xi (Nq x 3), PHS power p; W (Nq x n) receives the
 * long-double weights rounded to double. Returns the number of singular stencils (NaN rows). */
int64_t orc_stencil_weights_ld(const double *X, const int32_t *I, int64_t Nq, int n, int L, int p,
                               const double *Xi, double *W) {
    const int M = (L + 1) * (L + 1), m = n + M;
    int64_t nsing = 0;
#pragma omp parallel reduction(+ : nsing)
    {
        long double *A = (long double *)malloc(sizeof(long double) * (size_t)m * m);
        long double *b = (long double *)malloc(sizeof(long double) * (size_t)m);
        long double *C = (long double *)malloc(sizeof(long double) * 3 * (size_t)(n + 1));
        long double *Y = (long double *)malloc(sizeof(long double) * (size_t)M);
#pragma omp for schedule(dynamic, 1)
        for (int64_t s = 0; s < Nq; ++s) {
            const int32_t *S = I + s * n;
            for (int j = 0; j < n; ++j)
                for (int c = 0; c < 3; ++c) C[3 * j + c] = (long double)X[3 * (int64_t)S[j] + c];
            for (int c = 0; c < 3; ++c) C[3 * n + c] = (long double)Xi[3 * s + c];
            memset(A, 0, sizeof(long double) * (size_t)m * m);
            for (int i = 0; i < n; ++i) {
                for (int j = 0; j < n; ++j) A[(size_t)i * m + j] = i == j ? 0.0L : phs_ld(p, C + 3 * i, C + 3 * j);
                sh_eval_ld(L, C + 3 * i, Y);
                for (int c = 0; c < M; ++c) {
                    A[(size_t)i * m + n + c] = Y[c];
                    A[(size_t)(n + c) * m + i] = Y[c];
                }
                b[i] = phs_ld(p, C + 3 * n, C + 3 * i);
            }
            sh_eval_ld(L, C + 3 * n, Y);
            for (int c = 0; c < M; ++c) b[n + c] = Y[c];
            int bad = 0;
            for (int k = 0; k < m && !bad; ++k) {
                int q = k;
                long double best = fabsl(A[(size_t)k * m + k]);
                for (int i = k + 1; i < m; ++i) {
                    long double v = fabsl(A[(size_t)i * m + k]);
                    if (v > best) { best = v; q = i; }
                }
                if (!(best > 0.0L) || !isfinite(best)) { bad = 1; break; }
                if (q != k) {
                    for (int j = 0; j < m; ++j) {
                        long double t = A[(size_t)k * m + j]; A[(size_t)k * m + j] = A[(size_t)q * m + j]; A[(size_t)q * m + j] = t;
                    }
                    long double t = b[k]; b[k] = b[q]; b[q] = t;
                }
                long double piv = A[(size_t)k * m + k];
                for (int i = k + 1; i < m; ++i) {
                    long double l = A[(size_t)i * m + k] / piv;
                    if (l == 0.0L) continue;
                    for (int j = k + 1; j < m; ++j) A[(size_t)i * m + j] -= l * A[(size_t)k * m + j];
                    b[i] -= l * b[k];
                }
            }
            if (!bad)
                for (int i = m - 1; i >= 0; --i) {
                    long double t = b[i];
                    for (int j = i + 1; j < m; ++j) t -= A[(size_t)i * m + j] * b[j];
                    b[i] = t / A[(size_t)i * m + i];
                }
            for (int j = 0; j < n; ++j) W[s * n + j] = bad ? NAN : (double)b[j];
            nsing += bad;
        }
        free(A); free(b); free(C); free(Y);
    }
    return nsing;
}

/* ------------------------------------------------------------------ one local SL step */
/* Algorithm 1, one step of the local method: departure points Xi are given; for each point,
 * the stencil is either the n nearest nodes of xi (mode 0, direct) or the stencil of the
 * nearest node of xi, i.e. that node and its n-1 nearest neighbours (mode 1, centre; Sec. 3.3);
 * weights from orc_stencil_weights; q_new[i][t] = sum_j w_j q[I_j][t] summed in stencil order.
 * q, qnew: N x T row-major. I_out (Nq x n) and W_out (Nq x n) may be NULL.
 * Returns the number of singular stencils. */
int64_t orc_local_apply(const double *X, int64_t N, int n, int L, int kkind, double kprm,
                        int mode, const double *Xi, int64_t Nq, const double *q, int T,
                        double *qnew, int32_t *I_out, double *W_out) {
    int64_t nsing = 0;
#pragma omp parallel reduction(+ : nsing)
    {
        int32_t *I = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        double *w = (double *)malloc(sizeof(double) * (size_t)n);
        int32_t ctr;
#pragma omp for schedule(dynamic, 16)
        for (int64_t i = 0; i < Nq; ++i) {
            const double *xi = Xi + 3 * i;
            if (mode == 0) {
                orc_knn(X, N, xi, 1, n, I, NULL);
            } else {
                orc_knn(X, N, xi, 1, 1, &ctr, NULL);
                orc_knn(X, N, X + 3 * (int64_t)ctr, 1, n, I, NULL);
            }
            if (orc_stencil_weights(X, I, n, L, kkind, kprm, xi, w) != 0) ++nsing;
            for (int t = 0; t < T; ++t) {
                double s = 0.0;
                for (int j = 0; j < n; ++j) s += w[j] * q[(int64_t)I[j] * T + t];
                qnew[i * T + t] = s;
            }
            if (I_out) memcpy(I_out + i * n, I, sizeof(int32_t) * (size_t)n);
            if (W_out) memcpy(W_out + i * n, w, sizeof(double) * (size_t)n);
        }
        free(I); free(w);
    }
    return nsing;
}

/* ------------------------------------------------------------------ global RBF */
/* A_X[i][j] = phi(|x_i - x_j|) (Eq. rbf_linsys). */
void orc_global_matrix(const double *X, int64_t N, int kkind, double kprm, double *A) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = 0; j < N; ++j)
            A[i * N + j] = kernel_of_d2(kkind, kprm, sqdist(X + 3 * i, X + 3 * j));
}

/* Kernel matrix between point and node sets: Phi[i][j] = phi(|p_i - x_j|) (Eq. srbfinterp). */
void orc_kernel_matrix(const double *P, int64_t Nq, const double *X, int64_t N, int kkind,
                       double kprm, double *Phi) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < Nq; ++i)
        for (int64_t j = 0; j < N; ++j)
            Phi[i * N + j] = kernel_of_d2(kkind, kprm, sqdist(P + 3 * i, X + 3 * j));
}

/* Evaluate the global interpolant (Eq. srbfinterp) at Nq points:
 * out[i][t] = sum_j phi(|p_i - x_j|) C[j][t], j ascending. */
void orc_global_eval(const double *P, int64_t Nq, const double *X, int64_t N, int kkind,
                     double kprm, const double *C, int T, double *out) {
#pragma omp parallel
    {
        double *acc = (double *)malloc(sizeof(double) * (size_t)T);
#pragma omp for schedule(static)
        for (int64_t i = 0; i < Nq; ++i) {
            for (int t = 0; t < T; ++t) acc[t] = 0.0;
            for (int64_t j = 0; j < N; ++j) {
                double f = kernel_of_d2(kkind, kprm, sqdist(P + 3 * i, X + 3 * j));
                for (int t = 0; t < T; ++t) acc[t] += f * C[j * T + t];
            }
            for (int t = 0; t < T; ++t) out[i * T + t] = acc[t];
        }
        free(acc);
    }
}

/* ------------------------------------------------------------------ RBF-PU */
/* PU weight functions (Eq. wght_func): kind 0 = Wendland C2 (1-r)^4 (4r+1) on [0,1);
 * kind 1 = the paper's cubic B-spline (Eq. bspline). */
double orc_pu_phi(int kind, double r) {
    if (r >= 1.0) return 0.0;
    if (kind == 0) {
        double a = 1.0 - r;
        return a * a * a * a * (4.0 * r + 1.0);
    }
    if (r < 0.5) return 2.0 / 3.0 + 4.0 * (r - 1.0) * r * r;
    double a = r - 1.0;
    return -4.0 / 3.0 * a * a * a;
}

/* Evaluate the RBF-PU interpolant (Eq. PU_interp) at Nq points. Patches: Mp centres Om,
 * radius R, members given in CSR form (mstart[Mp+1], members[]), patch coefficients
 * coef[mstart[l] + l*M .. ] laid out per patch as (n_l + M) x T row-major at coff[l].
 * For each point, patches with |p - om_l| < R contribute phi(|p-om|/R) s_l(p) / sum phi.
 * Returns the number of points covered by no patch (their outputs are NaN). */
int64_t orc_pu_eval(const double *P, int64_t Nq, const double *X, const double *Om, int64_t Mp,
                    double R, const int64_t *mstart, const int32_t *members,
                    const int64_t *coff, const double *coef, int L, int kkind, double kprm,
                    int wkind, int T, double *out) {
    int M = (L + 1) * (L + 1);
    int64_t unc = 0;
#pragma omp parallel reduction(+ : unc)
    {
        double *acc = (double *)malloc(sizeof(double) * (size_t)T);
        double *s = (double *)malloc(sizeof(double) * (size_t)T);
        double *Y = (double *)malloc(sizeof(double) * (size_t)M);
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < Nq; ++i) {
            const double *p = P + 3 * i;
            double wsum = 0.0;
            for (int t = 0; t < T; ++t) acc[t] = 0.0;
            orc_sh_eval(L, p, Y);
            for (int64_t l = 0; l < Mp; ++l) {
                double dist = sqrt(sqdist(p, Om + 3 * l));
                if (!(dist < R)) continue;
                double wl = orc_pu_phi(wkind, dist / R);
                int64_t nl = mstart[l + 1] - mstart[l];
                const double *c = coef + coff[l];
                for (int t = 0; t < T; ++t) s[t] = 0.0;
                for (int64_t j = 0; j < nl; ++j) {
                    double f = kernel_of_d2(kkind, kprm, sqdist(p, X + 3 * (int64_t)members[mstart[l] + j]));
                    for (int t = 0; t < T; ++t) s[t] += f * c[j * T + t];
                }
                for (int c2 = 0; c2 < M; ++c2)
                    for (int t = 0; t < T; ++t) s[t] += Y[c2] * c[(nl + c2) * T + t];
                for (int t = 0; t < T; ++t) acc[t] += wl * s[t];
                wsum += wl;
            }
            if (wsum > 0.0) {
                for (int t = 0; t < T; ++t) out[i * T + t] = acc[t] / wsum;
            } else {
                for (int t = 0; t < T; ++t) out[i * T + t] = NAN;
                ++unc;
            }
        }
        free(acc); free(s); free(Y);
    }
    return unc;
}

/* Patch coefficients (Eq. rbf_poly_linsys per patch): for every patch, solve
 * [[A_l, P_l], [P_l^T, 0]] c~ = [q(X_l); 0] for all T tracers. coef laid out as in
 * orc_pu_eval. Returns the number of singular patch systems. */
int64_t orc_pu_coefficients(const double *X, int64_t Mp, const int64_t *mstart,
                            const int32_t *members, const int64_t *coff, int L, int kkind,
                            double kprm, const double *q, int T, double *coef) {
    int M = (L + 1) * (L + 1);
    int64_t nsing = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : nsing)
    for (int64_t l = 0; l < Mp; ++l) {
        int nl = (int)(mstart[l + 1] - mstart[l]);
        int m = nl + M;
        const int32_t *I = members + mstart[l];
        double *A = (double *)calloc((size_t)m * m, sizeof(double));
        double *Y = (double *)malloc(sizeof(double) * (size_t)M);
        double *B = coef + coff[l];
        for (int i = 0; i < nl; ++i) {
            const double *xa = X + 3 * (int64_t)I[i];
            for (int j = 0; j < nl; ++j)
                A[(size_t)i * m + j] = kernel_of_d2(kkind, kprm, sqdist(xa, X + 3 * (int64_t)I[j]));
            orc_sh_eval(L, xa, Y);
            for (int c = 0; c < M; ++c) {
                A[(size_t)i * m + nl + c] = Y[c];
                A[(size_t)(nl + c) * m + i] = Y[c];
            }
            for (int t = 0; t < T; ++t) B[(size_t)i * T + t] = q[(int64_t)I[i] * T + t];
        }
        for (int c = 0; c < M; ++c)
            for (int t = 0; t < T; ++t) B[(size_t)(nl + c) * T + t] = 0.0;
        if (orc_gepp_solve(A, m, B, T) != 0) ++nsing;
        free(A); free(Y);
    }
    return nsing;
}
