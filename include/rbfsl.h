/*
 * rbfsl.h -- C ABI of the GB300 library for RBF semi-Lagrangian (SL) transport on the unit
 * sphere (Shankar & Wright, "Mesh-free semi-Lagrangian methods for transport on a sphere
 * using radial basis functions").
 *
 * Two layers:
 *  1. A context that follows the paper's problem statement (Algorithm 1, "Input"): a
 *     velocity field tangent to S^2, an initial field q(x, 0), the node set X, a time step
 *     and a number of steps. rbfsl_step() runs whole SL steps on the device.
 *  2. Stateless per-step operations on caller-owned device buffers (departure points,
 *     k-nearest-neighbour stencils, stencil weights, the gather-dot W.q). The context calls
 *     the same kernels.
 *
 * Conventions shared by every entry point:
 *  - Return value: RBFSL_OK (0) or a negative RBFSL_E* code; no call aborts the process.
 *  - Layouts are row-major C arrays: points are N x 3 (x, y, z) doubles; tracer fields are
 *    N x T (tracer index fastest); stencils are Nq x n int32 node indices (0-based).
 *  - Device pointers must be allocated on the device current for the call (or the context's
 *    device); `stream` is a cudaStream_t (NULL = the legacy default stream). Stateless
 *    operations are asynchronous with respect to the host: they validate their arguments,
 *    enqueue kernels and return. Per-point failures are reported in the optional device
 *    array `status` (0 = ok, else an RBFSL_E* code) once the stream has reached them.
 *  - The library never keeps a caller pointer after a call returns.
 */
#ifndef RBFSL_H
#define RBFSL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ codes */
enum {
    RBFSL_OK = 0,
    RBFSL_EINVAL = -1,     /* a size, kind or pointer argument is invalid */
    RBFSL_ENOTCONF = -2,   /* a required setter has not been called */
    RBFSL_ENOMEM = -3,     /* device allocation failed */
    RBFSL_ESINGULAR = -4,  /* a stencil / patch / global system met a zero pivot */
    RBFSL_EUNCOVERED = -5, /* a point lies in no RBF-PU patch */
    RBFSL_ETIMEDOUT = -6,  /* a bounded device-side wait gave up */
    RBFSL_ECUDA = -7,      /* a CUDA runtime call failed (see rbfsl_last_error) */
    RBFSL_EKNN = -8        /* the neighbour search could not bracket k neighbours */
};

/* Velocity fields (the ODE of Sec. 3.2, Eq. sl_ode, is integrated in Cartesian form).
 * RBFSL_VEL_RIGID:     u = omega (a x x); params = {a_x, a_y, a_z, omega}, |a| = 1
 *                      (solid-body rotation, Sec. 4.1, for any axis).
 * RBFSL_VEL_DEFORM_Y2: u = x cross grad(psi), psi = kappa y^2 cos(pi t / T_f);
 *                      params = {kappa, T_f}. Reverses at t = T_f / 2 and returns every
 *                      parcel at t = T_f (a reversing deformational flow).
 * RBFSL_VEL_NL:        the paper's deformational flow (Sec. 4.2), params = {kappa, T_f}
 *                      (the paper: T_f = 5, kappa = 10 / T_f); with longitude lambda, latitude
 *                      theta and lp = lambda - 2 pi t / T_f,
 *                        u = kappa cos(pi t/T_f) sin^2(lp) sin(2 theta) + (2 pi/T_f) cos(theta),
 *                        v = kappa cos(pi t/T_f) sin(2 lp) cos(theta)
 *                      (zonal, meridional), evaluated as x cross grad(psi) with
 *                      psi = kappa cos(pi t/T_f) (y cos c - x sin c)^2 - (2 pi/T_f) z,
 *                      c = 2 pi t / T_f. Returns every parcel at t = T_f. The mixed-precision
 *                      tracers evaluate this field's stages in FP64. Not accepted by the batched
 *                      path (rbfsl_batch_add). */
enum { RBFSL_VEL_RIGID = 0, RBFSL_VEL_DEFORM_Y2 = 1, RBFSL_VEL_NL = 2 };

/* Interpolation method (Sec. 3.3). */
enum { RBFSL_LOCAL = 0, RBFSL_GLOBAL = 1, RBFSL_PU = 2 };

/* Local stencil choice. RBFSL_DIRECT: the n nearest nodes of each departure point, with a
 * fresh saddle-point solve per point and step. RBFSL_CENTER: the stencil of the departure
 * point's nearest node (that node and its n-1 nearest neighbours, Sec. 2.2 and 3.3). */
enum { RBFSL_DIRECT = 0, RBFSL_CENTER = 1 };

/* Radial kernels (Sec. 2.4): RBFSL_PHS r^p with odd p (param = p); RBFSL_GAUSS
 * exp(-(eps r)^2) and RBFSL_IMQ (1 + (eps r)^2)^(-1/2) (param = eps). */
enum { RBFSL_PHS = 0, RBFSL_GAUSS = 1, RBFSL_IMQ = 2 };

/* Precision. RBFSL_FP64: every step in FP64. RBFSL_MIXED: saddle-point solves in FP64;
 * departure tracing as an FP32 displacement added to the FP64 node; weights stored and
 * the gather-dot evaluated in FP32 in difference form q_c + sum_j w_j (q_j - q_c). */
enum { RBFSL_FP64 = 0, RBFSL_MIXED = 1 };

/* Element types of caller buffers. RBFSL_F32X2: unevaluated FP32 pairs, value = hi + lo with
 * |lo| <= ulp(hi)/2, interleaved (hi, lo) per element, 8 bytes each: the storage of weights
 * and fields in the mixed-precision step (rbfsl_stencil_weights output, rbfsl_gather_dot). */
enum { RBFSL_F64 = 0, RBFSL_F32 = 1, RBFSL_F32X2 = 2 };
enum { RBFSL_HOST = 0, RBFSL_DEVICE = 1 }; /* where a caller buffer lives */

/* Limits of this library. */
#define RBFSL_MAX_SH_DEGREE 8     /* ell <= 8, (ell+1)^2 <= 81 harmonics */
#define RBFSL_MAX_SYSTEM 160      /* n + (ell+1)^2 <= 160 for one saddle-point system */
#define RBFSL_MAX_K 256           /* neighbours per k-NN query */

/* ================================================================== stateless operations */

/* Departure points (Sec. 3.2, Eq. sl_ode): for each node x_j, integrate d xi/dt = u(xi, t)
 * backward from (x_j, t1) to t1 - dt with classical RK4 (h = -dt), projecting every stage
 * point and the result orthogonally onto S^2.
 *   x, xi: device, N x 3 doubles (may not alias). vel_params: HOST array (4 or 2 doubles).
 *   precision RBFSL_FP64 traces in FP64; RBFSL_MIXED computes the node's own velocity, the
 *   time factors and the final add and projection in FP64 and the stages as FP32 increments
 *   from the node (stage offset and velocity change), so FP32 rounding scales with |u| dt.
 * Errors: EINVAL (N < 0, null pointers, unknown kind or precision), ECUDA. */
int rbfsl_trace_rk4(const double *x, int64_t N, int vel_kind, const double *vel_params,
                    double t1, double dt, int precision, double *xi, void *stream);

/* The same departure points with Fehlberg's fifth-order Runge-Kutta formula, the paper's final
 * integrator choice (Sec. 3.2): six stages (nodes 0, 1/4, 3/8, 12/13, 1, 1/2 and the published
 * coupling coefficients), fifth-order weights 16/135, 0, 6656/12825, 28561/56430, -9/50, 2/55;
 * every stage point and the result projected onto S^2. Arguments, precisions and errors as
 * rbfsl_trace_rk4. */
int rbfsl_trace_rk5(const double *x, int64_t N, int vel_kind, const double *vel_params,
                    double t1, double dt, int precision, double *xi, void *stream);

/* Spatial index for k-nearest-neighbour queries over a fixed node set (replaces the
 * kd-tree of Sec. 3.3): a uniform grid over [-1,1]^3 whose cells hold the nodes sorted by
 * cell. The index owns copies of the nodes (device memory, freed by _destroy).
 *   x: device, N x 3 doubles. k_hint: the typical k of later queries (sets the cell size).
 * Creation synchronises `stream`. Errors: EINVAL, ENOMEM, ECUDA. */
typedef struct rbfsl_knn_index rbfsl_knn_index;
int rbfsl_knn_index_create(rbfsl_knn_index **out, const double *x, int64_t N, int k_hint,
                           void *stream);
int rbfsl_knn_index_destroy(rbfsl_knn_index *index);

/* The k nearest nodes of each query point, ascending by the key (d2, node index) with
 * d2 = ((qx-x)^2 + (qy-y)^2) + (qz-z)^2, every operation rounded to nearest in FP64 (no
 * fused multiply-add): the result equals a brute-force search, ties to the smaller index.
 *   q: device, Nq x 3 doubles. idx: device, Nq x k int32. status: device Nq int32 or NULL
 *   (RBFSL_EKNN where the search failed; idx row then -1).
 * Errors: EINVAL (k < 1, k > RBFSL_MAX_K, k > N), ECUDA. */
int rbfsl_knn_query(const rbfsl_knn_index *index, const double *q, int64_t Nq, int k,
                    int32_t *idx, int32_t *status, void *stream);

/* Stencil weights of the augmented local RBF interpolant (Sec. 2.2, Eqs. rbf_poly and
 * rbf_poly_linsys). For point p_i with stencil S = idx[i, 0..n), solve in FP64
 *   [[A, P], [P^T, 0]] w~ = [phi(|p_i - x_Sj|)_j ; Y(p_i)],   w[i, :] = w~[0:n],
 * A_jk = phi(|x_Sj - x_Sk|), P_jc = Y_c(x_Sj), Y = real orthonormal spherical harmonics
 * of degree <= ell. Then the interpolant at p_i is sum_j w_ij f_Sj (the system is
 * symmetric). Solved by a symmetric indefinite L D L^T factorisation with Bunch-Kaufman
 * pivoting (1 x 1 and 2 x 2 pivots; blocked: the trailing update once per panel of four pivot
 * columns), one warp per point for small systems, four warps for larger ones; the result does
 * not depend on that choice.
 *   x: device N x 3; idx: device Nq x n; p: device Nq x 3; w: device Nq x n of w_dtype
 *   (RBFSL_F64, RBFSL_F32 or RBFSL_F32X2: FP64 solve, result rounded or split into an FP32
 *   pair). status: device Nq or NULL
 *   (RBFSL_ESINGULAR for two coincident stencil nodes or a zero or non-finite pivot; w row
 *   NaN).
 * Errors: EINVAL (n < 1, ell > RBFSL_MAX_SH_DEGREE, n + (ell+1)^2 > RBFSL_MAX_SYSTEM,
 *   kernel not RBFSL_PHS with odd p >= 1), ECUDA. */
int rbfsl_stencil_weights(const double *x, int64_t N, const int32_t *idx, int64_t Nq, int n,
                          int ell, int kernel, double kparam, const double *p, void *w,
                          int w_dtype, int32_t *status, void *stream);

/* Gather-dot (Algorithm 1, "interpolate q to the departure points"): for i < Nq, t < T,
 *   q_out[i, t] = sum_j w[i, j] q[idx[i, j], t]           (w_dtype = q_dtype = RBFSL_F64)
 *   q_out[i, t] = q[c, t] + sum_j w[i, j] (q[idx[i,j], t] - q[c, t]),  c = idx[i, 0]
 *                                                          (w_dtype = q_dtype = RBFSL_F32)
 * The difference form equals the first when sum_j w_ij = 1 and keeps FP32 rounding
 * relative to the local variation of q. dtype RBFSL_F32X2: w, q and q_out are FP32 pairs
 * (Nq x n x 2, N x T x 2, Nq x T x 2 floats) and the first sum is formed in pair arithmetic
 * with FP32 operations only (exact high products by FMA, cross terms, two-sum accumulation):
 * relative rounding ~ n 2^-48 of sum_j |w_ij q_jt| instead of FP32's 2^-24.
 * q_out may not alias q. A negative idx entry (a failed stencil) gives a NaN row.
 * Errors: EINVAL (bad dtype, T < 1, n < 1, null pointers, q_out == q), ECUDA. */
int rbfsl_gather_dot(const int32_t *idx, const void *w, int64_t Nq, int n, const void *q,
                     int T, int dtype, void *q_out, void *stream);

/* Global RBF interpolation matrix (Sec. 2.1, Eq. rbf_linsys), factorised once (Sec. 3.3):
 * A_X[i][j] = phi(|x_i - x_j|) with phi the Gaussian exp(-(eps r)^2) (RBFSL_GAUSS) or the
 * inverse multiquadric (1 + (eps r)^2)^(-1/2) (RBFSL_IMQ), then LU with partial pivoting
 * (FP64, row-major). The paper factorises its positive-definite IMQ matrix by Cholesky; LU is
 * used for every kernel because FP64 Cholesky breaks down on numerically semi-definite
 * Gaussian matrices (eps = 6, N = 10,242).
 *   x: device N x 3. LU: device N x N doubles, overwritten with the factors. perm: device N
 *   int32, the row order P of P A = L U. Allocates and frees O(N) device scratch, synchronises
 *   `stream`. Errors: EINVAL, ENOMEM, ESINGULAR (a zero pivot), ECUDA. */
int rbfsl_global_factor(const double *x, int64_t N, int kernel, double eps, double *LU,
                        int32_t *perm, void *stream);

/* Same factorisation as rbfsl_global_factor, for callers that cannot allocate device memory
 * when they factorise (for example a serving process whose allocator owns the device memory
 * budget, or code that must not trigger the device-wide synchronisation an allocation can
 * cause while other streams run). The paper has no counterpart: this is a property of the
 * library, not of the method.
 *   Allocates nothing: the scratch (pivot rows and a status word) is a file-scope device
 *   array of RBFSL_NOALLOC_FACTOR_MAX_N + 1 int32 that every GPU loading the library holds
 *   until exit; N above RBFSL_NOALLOC_FACTOR_MAX_N is rejected with EINVAL.
 *   Runs on the current device. The first call on a device looks up the array's device
 *   address (cudaGetSymbolAddress); make that first call before any stream capture. The
 *   address is kept for the life of the process: do not reset the device (cudaDeviceReset,
 *   or a reset of its primary context) between calls, which would leave it stale.
 *   All calls share the one array: calls whose work overlaps on the GPU (other streams,
 *   other host threads) race and must be serialised by the caller.
 *   Arguments, outputs and errors as rbfsl_global_factor; synchronises `stream`. */
#define RBFSL_NOALLOC_FACTOR_MAX_N 16384
int rbfsl_global_factor_noalloc(const double *x, int64_t N, int kernel, double eps, double *LU,
                                int32_t *perm, void *stream);

/* Cholesky factorisation of the same matrix (Sec. 3.3: the paper factorises its positive-
 * definite IMQ matrix so), A_X = R^T R, blocked on the upper triangle (half the flops of
 * elimination), returned in rbfsl_global_factor's form so that rbfsl_global_solve and
 * rbfsl_global_cardinal take it unchanged: LU holds the unit lower L = R^T diag(R)^-1 below the
 * diagonal and U = diag(R) R on and above it, perm the identity.
 *   Arguments as rbfsl_global_factor. Allocates and frees O(N) device scratch, synchronises
 *   `stream`. Errors: EINVAL, ENOMEM, ECUDA, ESINGULAR at a non-positive (or non-finite) pivot:
 *   the matrix is not numerically positive definite (for example the Gaussian matrix at
 *   eps = 6, N = 10,242) and LU holds no usable factor; the context then uses
 *   rbfsl_global_factor. */
int rbfsl_global_factor_chol(const double *x, int64_t N, int kernel, double eps, double *LU,
                             int32_t *perm, void *stream);

/* Coefficients of the global interpolant for T fields: solve A_X c = q with the factor of
 * rbfsl_global_factor or rbfsl_global_factor_chol (forward and backward substitution, FP64).
 * q, c: device N x T, may not alias. Errors: EINVAL, ECUDA. */
int rbfsl_global_solve(const double *LU, const int32_t *perm, int64_t N, const double *q, int T,
                       double *c, void *stream);

/* Evaluate the global interpolant (Eq. srbfinterp) at Nq points for T fields:
 *   out[i][t] = sum_j phi(|p_i - x_j|) c[j][t].
 * dtype RBFSL_F64: c and out FP64, FP64 arithmetic. RBFSL_F32: c and out FP32, FP32 kernel
 * values and FP32 accumulation (the mixed-precision evaluation).
 * p: device Nq x 3, x: device N x 3. Errors: EINVAL, ECUDA. */
int rbfsl_global_eval(const double *p, int64_t Nq, const double *x, int64_t N, int kernel,
                      double eps, const void *c, int T, int dtype, void *out, void *stream);

/* RBF partition of unity (Sec. 2.3, 3.3). Patches are the spherical caps |x - omega_l| < R
 * around Mp given centres (the paper takes R = 2 sqrt(n / N) for ~n nodes per patch,
 * Eq. rad_patches, and Mp = ceil(a N / n) centres, Eq. num_patches). Creation finds each
 * patch's nodes, assembles its augmented PHS + spherical-harmonic system (Eq.
 * rbf_poly_linsys, degree ell) and factorises it once (LU with partial pivoting, FP64).
 *   x: device N x 3, centers: device Mp x 3 (copied). kernel must be RBFSL_PHS with odd p.
 *   Synchronises `stream`. Errors: EINVAL (a patch with no node, or more than
 *   RBFSL_MAX_SYSTEM - (ell+1)^2 nodes), ESINGULAR, ENOMEM, ECUDA. */
typedef struct rbfsl_pu rbfsl_pu;
enum { RBFSL_PU_WENDLAND = 0, RBFSL_PU_BSPLINE = 1 };
int rbfsl_pu_create(rbfsl_pu **out, const double *x, int64_t N, const double *centers, int64_t Mp,
                    double radius, int ell, int kernel, double kparam, void *stream);
int rbfsl_pu_destroy(rbfsl_pu *pu);

/* One RBF-PU interpolation (Eq. PU_interp) of T fields q (device N x T, FP64) to Nq points p:
 * patch coefficients [c; d] = A~_l^-1 [q(X_l); 0] (FP64), then
 *   out[i] = sum_l phi_l(p_i) s_l(p_i) / sum_l phi_l(p_i)   over patches containing p_i,
 * phi_l(x) = phi(|x - omega_l| / R), phi = Wendland C2 (1-r)^4 (4r+1) (RBFSL_PU_WENDLAND) or
 * the paper's cubic B-spline (Eq. bspline, RBFSL_PU_BSPLINE). dtype RBFSL_F64: FP64
 * evaluation; RBFSL_F32: FP32 evaluation, out FP32; RBFSL_F32X2: each term's factor formed in
 * FP64, coefficients and sums as FP32 pairs (hi, lo) in pair arithmetic, out N x T pairs
 * (~n 2^-48 relative rounding, against the patch sums' cancellation). The handle keeps a coefficient buffer
 * (reallocated when T changes), so calls on one handle must not overlap.
 * status: device Nq or NULL (RBFSL_EUNCOVERED for a point in no patch, RBFSL_EINVAL for a
 * point in more than 32 patches; out row NaN). Errors: EINVAL, ENOMEM, ECUDA. */
int rbfsl_pu_apply(rbfsl_pu *pu, const double *q, int T, const double *p, int64_t Nq,
                   int weight_kind, int dtype, void *out, int32_t *status, void *stream);

/* Global-interpolant evaluation on the tensor cores (tcgen05): the same sum as
 * rbfsl_global_eval, with the kernel values computed in FP32 and both operands split into a
 * TF32 high part and an FP32 remainder; hi*hi + hi*lo + lo*hi accumulate in FP32 in tensor
 * memory (the mixed-precision evaluation). c: device N x T of c_dtype (RBFSL_F64 or RBFSL_F32);
 * out: device Nq x T FP32. workspace: device buffer of at least
 * rbfsl_global_eval_tc_workspace_bytes(Nq, N, T) bytes (0 for bad sizes), 16-byte aligned: the
 * split coefficients in the tensor-core operand layout, the nodes in FP32, the split-K partial
 * tiles and a status word; the caller owns it and must not share it between calls that overlap
 * on the GPU. The node range is split across CTAs so that the grid fills the device; the
 * partial sums are added in a fixed order, so the result is deterministic for a given device.
 * status: device int32 or NULL; set to RBFSL_ETIMEDOUT if a bounded wait inside the kernel gave
 * up (out is then unspecified), otherwise left unchanged. Asynchronous on `stream`.
 * Errors: EINVAL (sizes, kernel, dtype, workspace too small or misaligned), ECUDA. */
/* Global-interpolant evaluation to FP64 accuracy without FP64 products: Phi(p, x) formed in
 * FP64 (the kernel and distance arithmetic of rbfsl_global_eval) and stored as FP32 pairs, the
 * coefficients split into pairs, then out = Phi c by FP32-pair arithmetic (the product of
 * rbfsl_cardinal_apply): ~2^-48 relative per term. c: device N x T FP64; out: device Nq x T
 * FP32 pairs (Nq x T x 2 floats). workspace: device, 256-byte aligned, at least
 * rbfsl_global_eval_pairs_workspace_bytes(Nq, N, T) (Nq x N x 8 bytes for Phi, the split
 * coefficients and the product's split-K partials); owned by the caller, not shared between
 * calls that overlap on the GPU. Asynchronous on `stream`. Errors: EINVAL, ECUDA. */
size_t rbfsl_global_eval_pairs_workspace_bytes(int64_t Nq, int64_t N, int T);
int rbfsl_global_eval_pairs(const double *p, int64_t Nq, const double *x, int64_t N, int kernel,
                            double eps, const double *c, int T, void *out, void *workspace,
                            size_t workspace_bytes, void *stream);

size_t rbfsl_global_eval_tc_workspace_bytes(int64_t Nq, int64_t N, int T);
int rbfsl_global_eval_tc(const double *p, int64_t Nq, const double *x, int64_t N, int kernel,
                         double eps, const void *c, int c_dtype, int T, float *out,
                         void *workspace, size_t workspace_bytes, int32_t *status, void *stream);

/* Cardinal matrix of the global interpolant at Nq fixed points (Sec. 2.1): the interpolant of
 * q at p is phi(p, X) c with A_X c = q (Eqs. srbfinterp, rbf_linsys), so at all the points it
 * is E q with
 *   E = Phi(P, X) A_X^-1,   E[i][j] = value at p_i of the cardinal function of node x_j.
 * Under a steady flow the departure points are the same at every step, and one product
 * q <- E q (rbfsl_cardinal_apply) replaces the per-step solve and evaluation.
 *   LU, perm: the factor of rbfsl_global_factor for the same x, kernel and eps (A_X is
 *   symmetric, so E^T = A_X^-1 Phi(P, X)^T is solved with it in blocks of points).
 *   x: device N x 3; p: device Nq x 3. E: device Nq x N row-major, e_dtype RBFSL_F64 (doubles)
 *   or RBFSL_F32X2 (FP32 pairs hi = fl32(e), lo = fl32(e - hi); Nq x N x 2 floats), computed in
 *   FP64 either way. Allocates and frees 2 N min(Nq, 512) doubles of device scratch and
 *   synchronises `stream`. Errors: EINVAL (sizes, kernel, dtype, null pointers), ENOMEM, ECUDA. */
int rbfsl_global_cardinal(const double *LU, const int32_t *perm, const double *x, int64_t N,
                          int kernel, double eps, const double *p, int64_t Nq, void *E,
                          int e_dtype, void *stream);

/* q_out = E q for a cardinal matrix E (Nq x N) and T fields q (N x T), row-major:
 *   q_out[i][t] = sum_j E[i][j] q[j][t].
 * dtype RBFSL_F64: E, q, q_out doubles, FP64 arithmetic. RBFSL_F32X2: FP32 pairs, each term
 * formed in pair arithmetic with FP32 operations only (relative rounding ~2^-48 per term; the
 * cardinal values are O(1), so there is no cancellation to amplify it).
 * The sum over j is split into ranges so that the grid covers the device; the partial sums go
 * to `workspace` (at least rbfsl_cardinal_apply_workspace_bytes(Nq, N, T) bytes on the calling
 * device, 0 when no split is needed; the caller owns it and must not share it between calls that
 * overlap on the GPU) and are added in a fixed order, so the result is deterministic for a given
 * device. q_out may not alias q. Asynchronous on `stream`.
 * Errors: EINVAL (sizes, dtype, null pointers, workspace too small), ECUDA. */
size_t rbfsl_cardinal_apply_workspace_bytes(int64_t Nq, int64_t N, int T);
int rbfsl_cardinal_apply(const void *E, int64_t Nq, int64_t N, const void *q, int T, int dtype,
                         void *q_out, void *workspace, size_t workspace_bytes, void *stream);

/* ================================================================== context (Algorithm 1) */
typedef struct rbfsl_ctx rbfsl_ctx;

typedef struct rbfsl_stats {
    int64_t steps_done;        /* SL steps completed since the last set_tracers */
    int64_t singular_points;   /* cumulative per-point ESINGULAR flags */
    int64_t knn_failures;      /* cumulative per-point EKNN flags */
    int64_t uncovered_points;  /* cumulative EUNCOVERED flags (RBF-PU) */
    double time;               /* model time of the current field */
    size_t device_bytes;       /* device memory held by the context */
    int64_t device_timeouts;   /* nonzero if a bounded wait in a device kernel gave up */
    int64_t global_cholesky;   /* global method: 1 if A_X was factorised by Cholesky, 0 if by
                                  LU with partial pivoting (Cholesky broke down), -1 before */
} rbfsl_stats;

/* Create a context on `device` whose work is enqueued on `stream` (a cudaStream_t of that
 * device, or NULL for the legacy default stream). Errors: EINVAL, ECUDA. */
int rbfsl_create(rbfsl_ctx **out, int device, void *stream);
int rbfsl_destroy(rbfsl_ctx *ctx);

/* Node set X (Sec. 3.1): N x 3 doubles on the host or the device, copied. Unit vectors
 * are expected (not checked). Invalidates prepared state. */
int rbfsl_set_nodes(rbfsl_ctx *ctx, const double *xyz, int64_t N, int mem);
/* Velocity field u (Sec. 3.2): kind RBFSL_VEL_* with its parameters (host, copied): 4 for
 * RBFSL_VEL_RIGID (unit axis, angular speed), 2 for RBFSL_VEL_DEFORM_Y2 and RBFSL_VEL_NL
 * (kappa, T_f > 0). With the cardinal global form selected it invalidates prepared state (the
 * departure points change). Errors: EINVAL (kind, count, non-unit axis, T_f <= 0). */
int rbfsl_set_velocity(rbfsl_ctx *ctx, int kind, const double *params, int nparams);
int rbfsl_set_method(rbfsl_ctx *ctx, int method, int stencil_mode);
/* Stencil size n (local) -- Sec. 2.2. */
int rbfsl_set_stencil_size(rbfsl_ctx *ctx, int n);
/* Spherical-harmonic degree ell of the augmentation (Sec. 2.4); ell < 0 selects the
 * paper's rule ell = floor((sqrt(n) - 1) / 2). */
int rbfsl_set_sh_degree(rbfsl_ctx *ctx, int ell);
int rbfsl_set_kernel(rbfsl_ctx *ctx, int kind, double param);
/* RBF-PU patches for the RBFSL_PU method: Mp centres (N x 3 doubles, host or device, copied),
 * cap radius (<= 0: 2 sqrt(n / N) with n the stencil size, Eq. rad_patches) and weight
 * function (RBFSL_PU_WENDLAND or RBFSL_PU_BSPLINE). */
int rbfsl_set_pu(rbfsl_ctx *ctx, const double *centers, int64_t Mp, double radius,
                 int weight_kind, int mem);
int rbfsl_set_precision(rbfsl_ctx *ctx, int precision);
int rbfsl_set_dt(rbfsl_ctx *ctx, double dt);
/* Departure-point integrator of the context's steps (Sec. 3.2): RBFSL_RK4 (default) or RBFSL_RK5
 * (Fehlberg's fifth-order formula, as rbfsl_trace_rk5). Takes effect at the next step; the
 * batched and served paths trace with RK4. Errors: EINVAL. */
enum { RBFSL_RK4 = 4, RBFSL_RK5 = 5 };
int rbfsl_set_integrator(rbfsl_ctx *ctx, int order);
/* Form of the RBFSL_GLOBAL step. RBFSL_GLOBAL_SOLVE (default): per step the coefficients
 * A_X^-1 q and the evaluation at the departure points (Sec. 3.3). RBFSL_GLOBAL_CARDINAL: the
 * departure points are traced once and E = Phi(Xi, X) A_X^-1 is formed at preparation
 * (rbfsl_global_cardinal; A_X's factor is freed afterwards), each step is q <- E q
 * (rbfsl_cardinal_apply: FP64, or FP32-pair arithmetic in RBFSL_MIXED). Valid for a steady
 * velocity only (RBFSL_VEL_RIGID; the first step returns EINVAL otherwise). Invalidates
 * prepared state, as do set_dt and set_integrator while the cardinal form is selected (E
 * depends on the departure points). Errors: EINVAL. */
enum { RBFSL_GLOBAL_SOLVE = 0, RBFSL_GLOBAL_CARDINAL = 1 };
int rbfsl_set_global_form(rbfsl_ctx *ctx, int form);
/* Evaluation arithmetic of the RBFSL_GLOBAL_SOLVE step in RBFSL_MIXED (the solve is FP64 in
 * both). RBFSL_GLOBAL_EVAL_TC (default): split-TF32 products on the tensor cores
 * (rbfsl_global_eval_tc; fastest, ~2^-22 relative). RBFSL_GLOBAL_EVAL_PAIRS: kernel values in
 * FP64, the sum Phi(Xi, X) C in FP32 pairs (rbfsl_global_eval_pairs; ~2^-48 relative, an N x N
 * pair workspace). Where the interpolation matrix is ill-conditioned the iteration feeds the
 * evaluation's rounding back through the next solve, so neither matches FP64 there (at Gaussian
 * eps = 9 on 10,242 nodes both diverge while FP64 does not); the cardinal form does.
 * Invalidates prepared state. Errors: EINVAL. */
enum { RBFSL_GLOBAL_EVAL_PAIRS = 0, RBFSL_GLOBAL_EVAL_TC = 1 };
int rbfsl_set_global_eval(rbfsl_ctx *ctx, int kind);
int rbfsl_set_time(rbfsl_ctx *ctx, double t);
/* Initial field q(X, t): N x T, element type dtype (converted to the context precision),
 * on the host (copied synchronously) or the device (copied on the context stream).
 * Resets steps_done. */
int rbfsl_set_tracers(rbfsl_ctx *ctx, const void *q, int64_t N, int T, int dtype, int mem);
/* Run `nsteps` SL steps (Algorithm 1): departure points, interpolation, q <- q_Xi,
 * t <- t + dt. Asynchronous on the context stream; prepares internal state on first use. */
int rbfsl_step(rbfsl_ctx *ctx, int nsteps);
/* Copy the current field (N x T) out as dtype to host (synchronises the stream) or device
 * (enqueued on the stream). */
int rbfsl_get_q(rbfsl_ctx *ctx, void *out, int dtype, int mem);
/* Synchronise the stream and report counters (per-point failures are summed here). */
int rbfsl_get_stats(rbfsl_ctx *ctx, rbfsl_stats *out);
/* Debug views of the last step (device buffers owned by the context, valid until the next
 * call that changes the context): departure points N x 3, stencils N x n, weights N x n
 * (FP64 in RBFSL_FP64 mode, FP32 in RBFSL_MIXED). NULL where the method has none. */
int rbfsl_last_step_buffers(rbfsl_ctx *ctx, const double **xi, const int32_t **idx,
                            const void **w);
/* ================================================================== batched problems */
/* Many independent local RBF-SL problems advanced together (each with its own nodes, stencil
 * size, degree, PHS power, stencil mode, precision, velocity, time step and tracers). One SL
 * step of every active problem is three small kernels and ONE persistent fused kernel (k-NN
 * stencil, FP64 weights, gather-dot per point; stencils and weights stay on chip), captured
 * once as a CUDA graph and replayed per step (when `stream` is not the legacy default stream).
 * A problem's result is bit-identical alone, in any batch, and through the context API with
 * the same settings (the same per-point device code runs in all three). */
typedef struct rbfsl_batch rbfsl_batch;
typedef struct rbfsl_problem {
    int64_t N;                /* nodes */
    const double *nodes;      /* HOST N x 3, copied */
    int n, ell;               /* stencil size, spherical-harmonic degree */
    double phs_power;         /* odd PHS exponent */
    int mode;                 /* RBFSL_DIRECT or RBFSL_CENTER */
    int precision;            /* RBFSL_FP64 or RBFSL_MIXED */
    int vel_kind;             /* RBFSL_VEL_* */
    double vel_params[4];     /* as rbfsl_set_velocity (unused entries 0) */
    double t0, dt;            /* time of q0 and time step */
    int T;                    /* tracers, 1..256 */
    const double *q0;         /* HOST N x T FP64, copied (rounded to FP32 in mixed precision) */
} rbfsl_problem;
int rbfsl_batch_create(rbfsl_batch **out, int device, void *stream);
int rbfsl_batch_destroy(rbfsl_batch *b);
/* Add a problem (allocates its state, builds its grid index and, in RBFSL_CENTER mode, its
 * stencil factors; synchronises the stream). *id identifies it until rbfsl_batch_remove.
 * Errors: EINVAL, ENOMEM, ESINGULAR, ECUDA. */
int rbfsl_batch_add(rbfsl_batch *b, const rbfsl_problem *problem, int *id);
/* Remove a problem and free its device memory (synchronises the stream). */
int rbfsl_batch_remove(rbfsl_batch *b, int id);
/* Advance every problem of the batch by nsteps SL steps (asynchronous on the stream). */
int rbfsl_batch_step(rbfsl_batch *b, int nsteps);
/* Current field of a problem, N x T FP64 to HOST memory (synchronises the stream). */
int rbfsl_batch_get_q(rbfsl_batch *b, int id, double *out);
int rbfsl_batch_problem_stats(rbfsl_batch *b, int id, rbfsl_stats *out);
/* use_graph = 0: launch the step's kernels eagerly instead of replaying a CUDA graph. */
int rbfsl_batch_set_graph(rbfsl_batch *b, int use_graph);
/* Autotuner: for every RBFSL_DIRECT (n, ell) class of the batch, time the persistent kernel
 * with one warp per point and with four warps per point and keep the faster for later steps.
 * Shapes whose block would need more than a quarter of an SM's shared memory (or more than
 * the largest single-point block) are not tried: every block of the persistent kernel gets
 * the largest class's shared memory, so such a shape would slow the other classes down.
 * Fields, times and step counts are unchanged. choices (may be NULL) receives triples
 * (n, ell, points per tile: 4 = one warp per point, 1 = four warps per point). */
int rbfsl_batch_autotune(rbfsl_batch *b, int *choices, int max_choices);

/* ================================================================== serving */
/* A serving loop for transport solves on one GPU. Requests (a full problem plus a step count)
 * are submitted at any time from any thread and copied. A scheduler thread owned by the
 * server repeats ticks: admit queued requests in arrival order while each fits the
 * device-memory budget and a slot is free; advance every running request by one SL step
 * (all local-stencil requests together in one batched persistent launch, every RBF-PU request
 * on its own stream, so their work overlaps on the device); retire the finished ones (field
 * copied out, device memory freed, latency recorded). State stays on the device between steps.
 * A request's result is bit-identical alone and in any mix. */
typedef struct rbfsl_server rbfsl_server;
typedef struct rbfsl_request {
    int method;               /* RBFSL_LOCAL or RBFSL_PU */
    rbfsl_problem problem;    /* for PU: n = nodes per patch, mode ignored */
    int steps;                /* SL steps to run */
    const double *pu_centers; /* PU: HOST Mp x 3, copied */
    int64_t pu_Mp;
    double pu_radius;         /* PU: <= 0 selects 2 sqrt(n / N) */
    int pu_weight;            /* PU: RBFSL_PU_WENDLAND or RBFSL_PU_BSPLINE */
} rbfsl_request;
typedef struct rbfsl_request_stats {
    double submit_s, admit_s, finish_s; /* seconds since the server was created */
    int64_t steps, node_updates;
    size_t device_bytes;                /* the admission estimate charged to the budget */
    int status;                         /* RBFSL_OK or the failure code */
    char message[160];                  /* the failure's message ("" on success) */
    int64_t failed_points;              /* point-steps with a singular stencil, a failed neighbour
                                           search or no covering patch (NaN rows in the result) */
} rbfsl_request_stats;
typedef struct rbfsl_server_info_t {
    int64_t ticks, queued;
    int running;
    size_t budget_bytes, used_bytes, peak_bytes;
    double now_s;
} rbfsl_server_info_t;
/* budget: device bytes the running requests may hold together (admission estimate per request:
 * nodes, departure points, fields, index, stencil or patch factors). max_slots: concurrent
 * requests. Starts the scheduler thread. Errors: EINVAL, ECUDA, ENOMEM. */
int rbfsl_server_create(rbfsl_server **out, int device, size_t hbm_budget_bytes, int max_slots);
/* Stop the scheduler and free everything (running requests are dropped). */
int rbfsl_server_destroy(rbfsl_server *s);
/* Queue a request; ENOMEM if it alone exceeds the budget. Thread-safe. */
int rbfsl_server_submit(rbfsl_server *s, const rbfsl_request *r, uint64_t *ticket);
/* state: 0 queued, 1 running, 2 done, < 0 failed (an RBFSL_E* code). */
int rbfsl_server_poll(rbfsl_server *s, uint64_t ticket, int *state);
/* Collect a finished request: its field (N x T FP64, HOST, may be NULL) and statistics; the
 * ticket is released. EINVAL while it is queued or running; the failure code if it failed. */
int rbfsl_server_result(rbfsl_server *s, uint64_t ticket, double *q_out, rbfsl_request_stats *st);
/* Block until no request is queued or running, or timeout_s passes (ETIMEDOUT). */
int rbfsl_server_wait_idle(rbfsl_server *s, double timeout_s);
int rbfsl_server_info(rbfsl_server *s, rbfsl_server_info_t *out);

/* Measured FP64 FMA throughput of the current device in TFLOP/s (2 flops per FMA): chains of
 * dependent FMAs in every thread of 8 blocks of 256 threads per SM, `iters` FMAs per chain and
 * eight chains per thread, timed with CUDA events after one shorter warm-up launch. The roofline
 * denominator of the FP64 stencil solves. The paper has no counterpart: a measurement utility.
 * Synchronises `stream`. Errors: EINVAL, ECUDA. */
int rbfsl_fp64_fma_rate(int64_t iters, double *tflops, void *stream);

/* Message of the last failed call on this context (thread-local when ctx is NULL). */
const char *rbfsl_last_error(const rbfsl_ctx *ctx);
const char *rbfsl_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RBFSL_H */
