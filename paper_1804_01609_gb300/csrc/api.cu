// Context API: the problem statement of Algorithm 1 (velocity, initial field, node set,
// time step) and the SL time loop on the device. Every step of the loop runs in this
// library's kernels; the host only validates, allocates and enqueues.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace rbfsl {

static thread_local std::string g_err;
void set_error(const std::string &msg) { g_err = msg; }
const char *get_error() { return g_err.c_str(); }

// Accumulate per-point failure flags of one step into device counters.
__global__ void count_status(const int32_t *__restrict__ st, int64_t N,
                             unsigned long long *__restrict__ ctr) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int32_t s = i < N ? st[i] : 0;
    const unsigned sing = __ballot_sync(0xffffffffu, s == RBFSL_ESINGULAR);
    const unsigned knn = __ballot_sync(0xffffffffu, s == RBFSL_EKNN);
    const unsigned unc = __ballot_sync(0xffffffffu, s == RBFSL_EUNCOVERED || s == RBFSL_EINVAL);
    if ((threadIdx.x & 31) == 0) {
        if (sing) atomicAdd(&ctr[0], (unsigned long long)__popc(sing));
        if (knn) atomicAdd(&ctr[1], (unsigned long long)__popc(knn));
        if (unc) atomicAdd(&ctr[2], (unsigned long long)__popc(unc));
    }
}

template <typename A, typename B>
__global__ void convert_kernel(const A *__restrict__ in, B *__restrict__ out, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = (B)in[i];
}

// Mixed-precision field storage (FP32 pairs, see pair_add) from and to plain arrays.
template <typename A>
__global__ void to_pair_kernel(const A *__restrict__ in, float2 *__restrict__ out, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const A v = in[i];
    const float hi = (float)v;
    out[i] = make_float2(hi, (float)(v - (A)hi));
}

template <typename B>
__global__ void from_pair_kernel(const float2 *__restrict__ in, B *__restrict__ out, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float2 v = in[i];
    out[i] = (B)((double)v.x + (double)v.y);
}

}  // namespace rbfsl

using namespace rbfsl;

struct rbfsl_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    // problem statement
    int64_t N = 0;
    double *X = nullptr;
    int vel_kind = -1;
    double vel[4] = {0, 0, 0, 0};
    int method = RBFSL_LOCAL, mode = RBFSL_DIRECT;
    int n = 0, ell = -1, kkind = RBFSL_PHS;
    double kparam = 3.0;
    int precision = RBFSL_FP64;
    double dt = 0.0, t = 0.0;
    int integrator = RBFSL_RK4;
    int global_form = RBFSL_GLOBAL_SOLVE;
    int global_eval = RBFSL_GLOBAL_EVAL_TC;  // mixed precision: evaluation arithmetic
    int T = 0;
    void *q = nullptr, *q_next = nullptr;  // N x T, FP64 or FP32 pairs (mixed), 8 bytes each
    int64_t steps_done = 0;
    // prepared state (local method)
    bool prepared = false;
    rbfsl_knn_index *knn = nullptr;
    double *xi = nullptr;
    int32_t *I = nullptr, *K = nullptr, *Ik = nullptr, *status = nullptr;
    void *W = nullptr;
    unsigned long long *ctr = nullptr;  // [singular, knn failures]
    // prepared state (global method)
    double *LU = nullptr, *C64 = nullptr, *Q64 = nullptr;
    void *tc_ws = nullptr;     // global, mixed: tensor-core evaluation workspace
    size_t tc_ws_bytes = 0;
    int32_t *dev_err = nullptr;  // RBFSL_ETIMEDOUT from a bounded device wait
    int32_t *perm = nullptr, *piv = nullptr;
    int global_cholesky = -1;  // global: 1 Cholesky, 0 LU (Cholesky broke down), -1 not factorised
    void *E = nullptr;         // global, cardinal form: Nq x N, FP64 or FP32 pairs
    void *card_ws = nullptr;   // its split-K partial sums
    size_t card_ws_bytes = 0;
    int prepared_T = 0;
    // RBF-PU
    double *pu_centers = nullptr;
    int64_t pu_Mp = 0;
    double pu_radius = 0.0;
    int pu_wkind = RBFSL_PU_WENDLAND;
    rbfsl_pu *pu = nullptr;
    size_t bytes = 0;
};

namespace {

int fail(rbfsl_ctx *c, int code, const std::string &msg) {
    if (c) c->err = msg;
    set_error(msg);
    return code;
}

int ctx_cuda(rbfsl_ctx *c, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return RBFSL_OK;
    cudaGetLastError();  // clear the runtime's record so later launches are not blamed
    return fail(c, e == cudaErrorMemoryAllocation ? RBFSL_ENOMEM : RBFSL_ECUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define CTX_TRY(c, expr)                                         \
    do {                                                         \
        int _rc = ctx_cuda((c), (expr), #expr);                  \
        if (_rc != RBFSL_OK) return _rc;                         \
    } while (0)

#define CTX_RC(c, expr)                                          \
    do {                                                         \
        int _rc = (expr);                                        \
        if (_rc != RBFSL_OK) return fail((c), _rc, get_error()); \
    } while (0)

template <typename P>
int dalloc(rbfsl_ctx *c, P **p, size_t bytes) {
    cudaError_t e = cudaMalloc((void **)p, bytes ? bytes : 1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(c, RBFSL_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    c->bytes += bytes;
    return RBFSL_OK;
}

void release_prepared(rbfsl_ctx *c) {
    if (c->knn) rbfsl_knn_index_destroy(c->knn);
    c->knn = nullptr;
    cudaFree(c->xi); cudaFree(c->I); cudaFree(c->K); cudaFree(c->Ik); cudaFree(c->status);
    cudaFree(c->W); cudaFree(c->ctr);
    c->xi = nullptr; c->I = c->K = c->Ik = c->status = nullptr; c->W = nullptr; c->ctr = nullptr;
    cudaFree(c->LU); cudaFree(c->C64); cudaFree(c->Q64); cudaFree(c->perm); cudaFree(c->piv);
    cudaFree(c->tc_ws); cudaFree(c->dev_err);
    c->tc_ws = nullptr; c->tc_ws_bytes = 0; c->dev_err = nullptr;
    cudaFree(c->E); cudaFree(c->card_ws);
    c->E = nullptr; c->card_ws = nullptr; c->card_ws_bytes = 0;
    c->global_cholesky = -1;
    if (c->pu) rbfsl_pu_destroy(c->pu);
    c->pu = nullptr;
    c->LU = c->C64 = c->Q64 = nullptr; c->perm = c->piv = nullptr;
    c->prepared = false;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

int effective_ell(const rbfsl_ctx *c) {
    if (c->ell >= 0) return c->ell;
    return (int)std::floor(0.5 * (std::sqrt((double)c->n) - 1.0));
}

// Global method (Sec. 3.3): A_X assembled and factorised once; per step a solve and an
// evaluation at the departure points.
int prepare_global_cardinal(rbfsl_ctx *c);

// A_X factorised by Cholesky as the paper does (Sec. 3.3); where that breaks down (a matrix
// that is positive definite but not numerically so, e.g. Gaussian eps = 6 at N = 10,242) by LU
// with partial pivoting. Both leave the factor in the form the solve takes.
int factor_global(rbfsl_ctx *c) {
    int rc = global_factor_chol_full(c->X, c->N, c->kkind, c->kparam, c->LU, c->perm, c->stream);
    if (rc == RBFSL_OK) {
        c->global_cholesky = 1;
        return RBFSL_OK;
    }
    if (rc != RBFSL_ESINGULAR) return fail(c, rc, get_error());
    CTX_RC(c, global_factor_full(c->X, c->N, c->kkind, c->kparam, c->LU, c->perm, c->piv, c->status, c->stream));
    c->global_cholesky = 0;
    return RBFSL_OK;
}

int prepare_global(rbfsl_ctx *c) {
    if (c->kkind != RBFSL_GAUSS && c->kkind != RBFSL_IMQ)
        return fail(c, RBFSL_EINVAL, "the global method needs RBFSL_GAUSS or RBFSL_IMQ");
    if (c->global_form == RBFSL_GLOBAL_CARDINAL) return prepare_global_cardinal(c);
    const int64_t N = c->N, T = c->T;
    int rc;
    if ((rc = dalloc(c, &c->xi, N * 3 * sizeof(double)))) return rc;
    if ((rc = dalloc(c, &c->LU, N * N * sizeof(double)))) return rc;
    if ((rc = dalloc(c, &c->perm, N * sizeof(int32_t)))) return rc;
    if ((rc = dalloc(c, &c->piv, N * sizeof(int32_t)))) return rc;
    if ((rc = dalloc(c, &c->status, sizeof(int32_t)))) return rc;
    if ((rc = dalloc(c, &c->C64, N * T * sizeof(double)))) return rc;
    if ((rc = dalloc(c, &c->ctr, 3 * sizeof(unsigned long long)))) return rc;
    CTX_TRY(c, cudaMemsetAsync(c->ctr, 0, 3 * sizeof(unsigned long long), c->stream));
    if ((rc = dalloc(c, &c->dev_err, sizeof(int32_t)))) return rc;
    CTX_TRY(c, cudaMemsetAsync(c->dev_err, 0, sizeof(int32_t), c->stream));
    if (c->precision == RBFSL_MIXED) {
        if ((rc = dalloc(c, &c->Q64, N * T * sizeof(double)))) return rc;
        c->tc_ws_bytes = c->global_eval == RBFSL_GLOBAL_EVAL_TC ? global_eval_tc_workspace(N, N, (int)T)
                                                                 : global_eval_pairs_workspace(N, N, (int)T);
        if ((rc = dalloc(c, &c->tc_ws, c->tc_ws_bytes))) return rc;
    }
    if ((rc = factor_global(c))) return rc;
    c->prepared_T = c->T;
    c->prepared = true;
    return RBFSL_OK;
}

// Cardinal form (steady flow): departure points traced once, E = Phi(Xi, X) A_X^-1 formed from
// the factor, which is freed; each step is q <- E q.
int prepare_global_cardinal(rbfsl_ctx *c) {
    if (c->vel_kind != RBFSL_VEL_RIGID)
        return fail(c, RBFSL_EINVAL, "the cardinal form needs a steady velocity field (RBFSL_VEL_RIGID)");
    const int64_t N = c->N;
    int rc;
    if ((rc = dalloc(c, &c->xi, N * 3 * sizeof(double)))) return rc;
    if ((rc = dalloc(c, &c->LU, N * N * sizeof(double)))) return rc;
    if ((rc = dalloc(c, &c->perm, N * sizeof(int32_t)))) return rc;
    if ((rc = dalloc(c, &c->piv, N * sizeof(int32_t)))) return rc;
    if ((rc = dalloc(c, &c->status, sizeof(int32_t)))) return rc;
    if ((rc = dalloc(c, &c->ctr, 3 * sizeof(unsigned long long)))) return rc;
    CTX_TRY(c, cudaMemsetAsync(c->ctr, 0, 3 * sizeof(unsigned long long), c->stream));
    if ((rc = dalloc(c, &c->E, N * N * 8))) return rc;
    c->card_ws_bytes = cardinal_apply_workspace(N, N, c->T);
    if (c->card_ws_bytes && (rc = dalloc(c, &c->card_ws, c->card_ws_bytes))) return rc;
    CTX_RC(c, launch_trace_order(c->X, N, c->vel_kind, c->vel, c->t + c->dt, c->dt, RBFSL_FP64, c->integrator,
                                 c->xi, c->stream));
    if ((rc = factor_global(c))) return rc;
    CTX_RC(c, global_cardinal_build(c->LU, c->perm, c->X, N, c->kkind, c->kparam, c->xi, N, c->E,
                                    c->precision == RBFSL_FP64 ? RBFSL_F64 : RBFSL_F32X2, c->stream));
    cudaFree(c->LU);
    c->LU = nullptr;
    c->bytes -= N * N * sizeof(double);
    c->prepared_T = c->T;
    c->prepared = true;
    return RBFSL_OK;
}

int one_step_global(rbfsl_ctx *c) {
    const int64_t N = c->N, NT = N * (int64_t)c->T;
    if (c->global_form == RBFSL_GLOBAL_CARDINAL) {
        CTX_RC(c, launch_cardinal_apply(c->E, N, N, c->q, c->T, c->precision == RBFSL_FP64 ? RBFSL_F64 : RBFSL_F32X2,
                                        c->q_next, c->card_ws, c->card_ws_bytes, c->stream));
        std::swap(c->q, c->q_next);
        c->t += c->dt;
        ++c->steps_done;
        return RBFSL_OK;
    }
    const double t1 = c->t + c->dt;
    const unsigned blocks = (unsigned)((NT + 255) / 256);
    CTX_RC(c, launch_trace_order(c->X, N, c->vel_kind, c->vel, t1, c->dt, c->precision, c->integrator, c->xi, c->stream));
    if (c->precision == RBFSL_FP64) {
        CTX_RC(c, global_solve(c->LU, c->perm, N, (const double *)c->q, c->T, c->C64, c->stream));
        CTX_RC(c, launch_global_eval(c->xi, N, c->X, N, c->kkind, c->kparam, c->C64, c->T, RBFSL_F64,
                                     c->q_next, RBFSL_F64, c->stream));
    } else if (c->global_eval == RBFSL_GLOBAL_EVAL_PAIRS) {
        // FP64 solve of the field (FP32 pairs widened); kernel values in FP64, the sum in
        // FP32-pair arithmetic, straight into the pair field
        from_pair_kernel<double><<<blocks, 256, 0, c->stream>>>((const float2 *)c->q, c->Q64, NT);
        CTX_RC(c, global_solve(c->LU, c->perm, N, c->Q64, c->T, c->C64, c->stream));
        CTX_RC(c, launch_global_eval_pairs(c->xi, N, c->X, N, c->kkind, c->kparam, c->C64, c->T,
                                           (float2 *)c->q_next, c->tc_ws, c->tc_ws_bytes, c->stream));
    } else {
        // FP64 solve of the field (FP32 pairs widened); evaluation on the tensor cores (split
        // TF32, FP32 accumulation) into the freed FP64 right-hand side buffer, stored as pairs
        from_pair_kernel<double><<<blocks, 256, 0, c->stream>>>((const float2 *)c->q, c->Q64, NT);
        CTX_RC(c, global_solve(c->LU, c->perm, N, c->Q64, c->T, c->C64, c->stream));
        float *q32 = reinterpret_cast<float *>(c->Q64);
        CTX_RC(c, launch_global_eval_tc(c->xi, N, c->X, N, c->kkind, c->kparam, c->C64, RBFSL_F64, c->T, q32,
                                        c->tc_ws, c->dev_err, c->stream));
        to_pair_kernel<float><<<blocks, 256, 0, c->stream>>>(q32, (float2 *)c->q_next, NT);
        CTX_RC(c, launch_status("global step (mixed)"));
    }
    std::swap(c->q, c->q_next);
    c->t = t1;
    ++c->steps_done;
    return RBFSL_OK;
}

// RBF-PU (Sec. 3.3): patches and their LU factors once; per step the patch coefficients and
// the blended evaluation at the departure points.
int prepare_pu(rbfsl_ctx *c) {
    if (!c->pu_centers) return fail(c, RBFSL_ENOTCONF, "set_pu has not been called");
    if (c->kkind != RBFSL_PHS) return fail(c, RBFSL_EINVAL, "the RBF-PU method needs the PHS kernel");
    const int64_t N = c->N, T = c->T;
    double R = c->pu_radius;
    if (!(R > 0)) {
        if (c->n < 1) return fail(c, RBFSL_ENOTCONF, "RBF-PU radius needs a stencil size (nodes per patch)");
        R = 2.0 * std::sqrt((double)c->n / (double)N);
    }
    const int ell = c->ell >= 0 ? c->ell : 3;
    int rc;
    if ((rc = dalloc(c, &c->xi, N * 3 * sizeof(double)))) return rc;
    if ((rc = dalloc(c, &c->status, N * sizeof(int32_t)))) return rc;
    if ((rc = dalloc(c, &c->ctr, 3 * sizeof(unsigned long long)))) return rc;
    CTX_TRY(c, cudaMemsetAsync(c->ctr, 0, 3 * sizeof(unsigned long long), c->stream));
    if (c->precision == RBFSL_MIXED) {
        if ((rc = dalloc(c, &c->Q64, N * T * sizeof(double)))) return rc;
    }
    CTX_RC(c, rbfsl_pu_create(&c->pu, c->X, N, c->pu_centers, c->pu_Mp, R, ell, c->kkind, c->kparam, c->stream));
    c->bytes += c->pu->bytes;
    c->prepared_T = c->T;
    c->prepared = true;
    return RBFSL_OK;
}

int one_step_pu(rbfsl_ctx *c) {
    const int64_t N = c->N, NT = N * (int64_t)c->T;
    const double t1 = c->t + c->dt;
    CTX_RC(c, launch_trace_order(c->X, N, c->vel_kind, c->vel, t1, c->dt, c->precision, c->integrator, c->xi, c->stream));
    const double *q64 = (const double *)c->q;
    const unsigned blocks = (unsigned)((NT + 255) / 256);
    if (c->precision == RBFSL_MIXED) {
        from_pair_kernel<double><<<blocks, 256, 0, c->stream>>>((const float2 *)c->q, c->Q64, NT);
        q64 = c->Q64;
    }
    // mixed: FP64 coefficient solves, the blend in FP32-pair arithmetic straight into the pair field
    CTX_RC(c, rbfsl_pu_apply(c->pu, q64, c->T, c->xi, N, c->pu_wkind,
                             c->precision == RBFSL_FP64 ? RBFSL_F64 : RBFSL_F32X2, c->q_next, c->status,
                             c->stream));
    count_status<<<(unsigned)((N + 255) / 256), 256, 0, c->stream>>>(c->status, N, c->ctr);
    std::swap(c->q, c->q_next);
    c->t = t1;
    ++c->steps_done;
    return RBFSL_OK;
}

int prepare(rbfsl_ctx *c) {
    if (c->prepared) return RBFSL_OK;
    if (!c->X) return fail(c, RBFSL_ENOTCONF, "set_nodes has not been called");
    if (c->vel_kind < 0) return fail(c, RBFSL_ENOTCONF, "set_velocity has not been called");
    if (!(c->dt > 0)) return fail(c, RBFSL_ENOTCONF, "set_dt has not been called");
    if (!c->q) return fail(c, RBFSL_ENOTCONF, "set_tracers has not been called");
    if (c->method == RBFSL_GLOBAL) return prepare_global(c);
    if (c->method == RBFSL_PU) return prepare_pu(c);
    if (c->n < 1 || c->n > c->N) return fail(c, RBFSL_ENOTCONF, "stencil size not set or > N");
    const int ell = effective_ell(c);
    if (ell > RBFSL_MAX_SH_DEGREE || c->n + (ell + 1) * (ell + 1) > RBFSL_MAX_SYSTEM)
        return fail(c, RBFSL_EINVAL, "n + (ell+1)^2 exceeds RBFSL_MAX_SYSTEM");
    const int pw = (int)c->kparam;
    if (c->kkind != RBFSL_PHS || pw < 1 || !(pw & 1))
        return fail(c, RBFSL_EINVAL, "local stencils need the PHS kernel with odd power");
    const int64_t N = c->N, n = c->n;
    int rc;
    if ((rc = dalloc(c, &c->xi, N * 3 * sizeof(double)))) return rc;
    if ((rc = dalloc(c, &c->I, N * n * sizeof(int32_t)))) return rc;
    if ((rc = dalloc(c, &c->status, N * sizeof(int32_t)))) return rc;
    if ((rc = dalloc(c, &c->W, N * n * 8))) return rc;  // FP64, or FP32 pairs (mixed)
    if ((rc = dalloc(c, &c->ctr, 3 * sizeof(unsigned long long)))) return rc;
    CTX_TRY(c, cudaMemsetAsync(c->ctr, 0, 3 * sizeof(unsigned long long), c->stream));
    CTX_RC(c, rbfsl_knn_index_create(&c->knn, c->X, N, (int)n, c->stream));
    c->bytes += c->knn->bytes;
    if (c->mode == RBFSL_CENTER) {
        // stencil of node k: x_k and its n-1 nearest neighbours (Sec. 2.2), its saddle-point
        // matrix factorised once (LU with partial pivoting, FP64; Sec. 3.3)
        const int64_t m = n + (ell + 1) * (ell + 1);
        if ((rc = dalloc(c, &c->K, N * sizeof(int32_t)))) return rc;
        if ((rc = dalloc(c, &c->Ik, N * n * sizeof(int32_t)))) return rc;
        if ((rc = dalloc(c, &c->LU, N * m * m * sizeof(double)))) return rc;
        if ((rc = dalloc(c, &c->perm, N * m * sizeof(int32_t)))) return rc;
        CTX_RC(c, launch_knn(c->knn, c->X, N, (int)n, c->Ik, c->status, c->stream));
        std::vector<int64_t> ms(N + 1), lo(N);
        for (int64_t k = 0; k <= N; ++k) ms[k] = k * n;
        for (int64_t k = 0; k < N; ++k) lo[k] = k * m * m;
        int64_t *d_ms = nullptr, *d_lo = nullptr;
        int32_t *d_bad = nullptr;
        CTX_TRY(c, cudaMalloc(&d_ms, (N + 1) * sizeof(int64_t)));
        CTX_TRY(c, cudaMalloc(&d_lo, N * sizeof(int64_t)));
        CTX_TRY(c, cudaMalloc(&d_bad, sizeof(int32_t)));
        CTX_TRY(c, cudaMemcpy(d_ms, ms.data(), (N + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
        CTX_TRY(c, cudaMemcpy(d_lo, lo.data(), N * sizeof(int64_t), cudaMemcpyHostToDevice));
        CTX_TRY(c, cudaMemsetAsync(d_bad, 0, sizeof(int32_t), c->stream));
        rc = launch_stencil_factor(c->X, d_ms, c->Ik, d_lo, N, (int)n, (ell + 1) * (ell + 1), ell, pw,
                                   c->LU, c->perm, d_bad, c->stream, 1);
        int32_t bad = 0;
        if (rc == RBFSL_OK) {
            cudaError_t e = cudaMemcpyAsync(&bad, d_bad, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) rc = ctx_cuda(c, e, "centre factorisation");
        }
        cudaFree(d_ms); cudaFree(d_lo); cudaFree(d_bad);
        if (rc != RBFSL_OK) return fail(c, rc, get_error());
        if (bad) return fail(c, RBFSL_ESINGULAR, std::to_string(bad) + " singular centre stencils");
    }
    c->prepared = true;
    return RBFSL_OK;
}

int one_step(rbfsl_ctx *c) {
    if (c->method == RBFSL_GLOBAL) return one_step_global(c);
    if (c->method == RBFSL_PU) return one_step_pu(c);
    const int64_t N = c->N;
    const int n = c->n, ell = effective_ell(c), pw = (int)c->kparam;
    const double t1 = c->t + c->dt;
    const int wdt = c->precision == RBFSL_FP64 ? RBFSL_F64 : RBFSL_F32X2;
    CTX_RC(c, launch_trace_order(c->X, N, c->vel_kind, c->vel, t1, c->dt, c->precision, c->integrator, c->xi, c->stream));
    if (c->mode == RBFSL_DIRECT) {
        CTX_RC(c, launch_knn(c->knn, c->xi, N, n, c->I, c->status, c->stream));
        CTX_RC(c, launch_weights(c->X, c->I, N, n, ell, pw, c->xi, c->W, wdt, c->status, c->stream));
    } else {
        CTX_RC(c, launch_knn(c->knn, c->xi, N, 1, c->K, c->status, c->stream));
        CTX_RC(c, launch_center_weights(c->X, c->K, c->Ik, c->LU, c->perm, N, n, ell, pw, c->xi, c->I, c->W,
                                        wdt, c->status, c->stream));
    }
    count_status<<<(unsigned)((N + 255) / 256), 256, 0, c->stream>>>(c->status, N, c->ctr);
    CTX_RC(c, launch_gather(c->I, c->W, N, n, c->q, c->T, wdt, c->q_next, c->stream));
    std::swap(c->q, c->q_next);
    c->t = t1;
    ++c->steps_done;
    return RBFSL_OK;
}

}  // namespace

extern "C" {

const char *rbfsl_version(void) { return "rbfsl-gb300 0.1 (sm_103a)"; }

const char *rbfsl_last_error(const rbfsl_ctx *c) { return c ? c->err.c_str() : get_error(); }

int rbfsl_create(rbfsl_ctx **out, int device, void *stream) {
    RBFSL_CHECK_ARG(out != nullptr, "create: out is null");
    int ndev = 0;
    RBFSL_CUDA_TRY(cudaGetDeviceCount(&ndev));
    RBFSL_CHECK_ARG(device >= 0 && device < ndev, "create: no such device");
    auto *c = new rbfsl_ctx();
    c->device = device;
    c->stream = (cudaStream_t)stream;
    DeviceGuard g(device);
    int rc = sh_tables_init();
    if (rc != RBFSL_OK) {
        delete c;
        return rc;
    }
    *out = c;
    return RBFSL_OK;
}

int rbfsl_destroy(rbfsl_ctx *c) {
    if (!c) return RBFSL_OK;
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    release_prepared(c);
    cudaFree(c->X); cudaFree(c->q); cudaFree(c->q_next); cudaFree(c->pu_centers);
    delete c;
    return RBFSL_OK;
}

int rbfsl_set_nodes(rbfsl_ctx *c, const double *xyz, int64_t N, int mem) {
    if (!c) return fail(nullptr, RBFSL_EINVAL, "null context");
    if (!xyz || N < 1 || N >= ((int64_t)1 << 31) || (mem != RBFSL_HOST && mem != RBFSL_DEVICE))
        return fail(c, RBFSL_EINVAL, "set_nodes: bad arguments");
    DeviceGuard g(c->device);
    CTX_TRY(c, cudaStreamSynchronize(c->stream));
    release_prepared(c);
    cudaFree(c->X); c->X = nullptr;
    cudaFree(c->q); cudaFree(c->q_next); c->q = c->q_next = nullptr;
    c->bytes = 0;
    c->N = N;
    int rc = dalloc(c, &c->X, N * 3 * sizeof(double));
    if (rc) return rc;
    CTX_TRY(c, cudaMemcpyAsync(c->X, xyz, N * 3 * sizeof(double),
                               mem == RBFSL_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                               c->stream));
    CTX_TRY(c, cudaStreamSynchronize(c->stream));
    return RBFSL_OK;
}

static void drop_cardinal(rbfsl_ctx *c);

int rbfsl_set_velocity(rbfsl_ctx *c, int kind, const double *params, int nparams) {
    if (!c) return fail(nullptr, RBFSL_EINVAL, "null context");
    if (!params) return fail(c, RBFSL_EINVAL, "set_velocity: params is null");
    if (kind == RBFSL_VEL_RIGID) {
        if (nparams != 4) return fail(c, RBFSL_EINVAL, "rigid rotation takes 4 parameters");
        const double a = std::sqrt(params[0] * params[0] + params[1] * params[1] + params[2] * params[2]);
        if (!(std::fabs(a - 1.0) < 1e-12)) return fail(c, RBFSL_EINVAL, "rotation axis is not a unit vector");
    } else if (kind == RBFSL_VEL_DEFORM_Y2 || kind == RBFSL_VEL_NL) {
        if (nparams != 2 || !(params[1] > 0)) return fail(c, RBFSL_EINVAL, "deformation takes {kappa, T_f > 0}");
    } else {
        return fail(c, RBFSL_EINVAL, "unknown velocity kind");
    }
    drop_cardinal(c);
    c->vel_kind = kind;
    for (int i = 0; i < 4; ++i) c->vel[i] = i < nparams ? params[i] : 0.0;
    return RBFSL_OK;
}

int rbfsl_set_method(rbfsl_ctx *c, int method, int stencil_mode) {
    if (!c) return fail(nullptr, RBFSL_EINVAL, "null context");
    if (method < RBFSL_LOCAL || method > RBFSL_PU) return fail(c, RBFSL_EINVAL, "unknown method");
    if (stencil_mode != RBFSL_DIRECT && stencil_mode != RBFSL_CENTER)
        return fail(c, RBFSL_EINVAL, "unknown stencil mode");
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    release_prepared(c);
    c->method = method;
    c->mode = stencil_mode;
    return RBFSL_OK;
}

int rbfsl_set_stencil_size(rbfsl_ctx *c, int n) {
    if (!c) return fail(nullptr, RBFSL_EINVAL, "null context");
    if (n < 1) return fail(c, RBFSL_EINVAL, "stencil size must be >= 1");
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    release_prepared(c);
    c->n = n;
    return RBFSL_OK;
}

int rbfsl_set_sh_degree(rbfsl_ctx *c, int ell) {
    if (!c) return fail(nullptr, RBFSL_EINVAL, "null context");
    if (ell > RBFSL_MAX_SH_DEGREE) return fail(c, RBFSL_EINVAL, "ell > RBFSL_MAX_SH_DEGREE");
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    release_prepared(c);
    c->ell = ell;
    return RBFSL_OK;
}

int rbfsl_set_kernel(rbfsl_ctx *c, int kind, double param) {
    if (!c) return fail(nullptr, RBFSL_EINVAL, "null context");
    if (kind < RBFSL_PHS || kind > RBFSL_IMQ || !(param > 0)) return fail(c, RBFSL_EINVAL, "bad kernel");
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    release_prepared(c);
    c->kkind = kind;
    c->kparam = param;
    return RBFSL_OK;
}

int rbfsl_set_pu(rbfsl_ctx *c, const double *centers, int64_t Mp, double radius, int weight_kind, int mem) {
    if (!c) return fail(nullptr, RBFSL_EINVAL, "null context");
    if (!centers || Mp < 1 || (mem != RBFSL_HOST && mem != RBFSL_DEVICE) ||
        (weight_kind != RBFSL_PU_WENDLAND && weight_kind != RBFSL_PU_BSPLINE) || radius > 2.0)
        return fail(c, RBFSL_EINVAL, "set_pu: bad arguments");
    DeviceGuard g(c->device);
    CTX_TRY(c, cudaStreamSynchronize(c->stream));
    release_prepared(c);
    cudaFree(c->pu_centers);
    c->pu_centers = nullptr;
    CTX_TRY(c, cudaMalloc(&c->pu_centers, Mp * 3 * sizeof(double)));
    CTX_TRY(c, cudaMemcpy(c->pu_centers, centers, Mp * 3 * sizeof(double),
                          mem == RBFSL_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice));
    c->pu_Mp = Mp;
    c->pu_radius = radius;
    c->pu_wkind = weight_kind;
    return RBFSL_OK;
}

int rbfsl_set_precision(rbfsl_ctx *c, int precision) {
    if (!c) return fail(nullptr, RBFSL_EINVAL, "null context");
    if (precision != RBFSL_FP64 && precision != RBFSL_MIXED) return fail(c, RBFSL_EINVAL, "unknown precision");
    if (precision == c->precision) return RBFSL_OK;
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    release_prepared(c);
    cudaFree(c->q); cudaFree(c->q_next);
    c->q = c->q_next = nullptr;  // the field must be set again in the new precision
    c->T = 0;
    c->precision = precision;
    return RBFSL_OK;
}

// The cardinal matrix depends on the departure points: changing them re-prepares.
static void drop_cardinal(rbfsl_ctx *c) {
    if (c->method != RBFSL_GLOBAL || c->global_form != RBFSL_GLOBAL_CARDINAL || !c->prepared) return;
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    release_prepared(c);
}

int rbfsl_set_integrator(rbfsl_ctx *c, int order) {
    if (!c) return fail(nullptr, RBFSL_EINVAL, "null context");
    if (order != RBFSL_RK4 && order != RBFSL_RK5) return fail(c, RBFSL_EINVAL, "integrator must be RBFSL_RK4 or RBFSL_RK5");
    if (order != c->integrator) drop_cardinal(c);
    c->integrator = order;
    return RBFSL_OK;
}

int rbfsl_set_global_form(rbfsl_ctx *c, int form) {
    if (!c) return fail(nullptr, RBFSL_EINVAL, "null context");
    if (form != RBFSL_GLOBAL_SOLVE && form != RBFSL_GLOBAL_CARDINAL)
        return fail(c, RBFSL_EINVAL, "global form must be RBFSL_GLOBAL_SOLVE or RBFSL_GLOBAL_CARDINAL");
    if (form != c->global_form && c->method == RBFSL_GLOBAL) {
        DeviceGuard g(c->device);
        cudaStreamSynchronize(c->stream);
        release_prepared(c);
    }
    c->global_form = form;
    return RBFSL_OK;
}

int rbfsl_set_global_eval(rbfsl_ctx *c, int kind) {
    if (!c) return fail(nullptr, RBFSL_EINVAL, "null context");
    if (kind != RBFSL_GLOBAL_EVAL_PAIRS && kind != RBFSL_GLOBAL_EVAL_TC)
        return fail(c, RBFSL_EINVAL, "global evaluation must be RBFSL_GLOBAL_EVAL_PAIRS or RBFSL_GLOBAL_EVAL_TC");
    if (kind != c->global_eval && c->method == RBFSL_GLOBAL) {
        DeviceGuard g(c->device);
        cudaStreamSynchronize(c->stream);
        release_prepared(c);
    }
    c->global_eval = kind;
    return RBFSL_OK;
}

int rbfsl_set_dt(rbfsl_ctx *c, double dt) {
    if (!c) return fail(nullptr, RBFSL_EINVAL, "null context");
    if (!(dt > 0) || !std::isfinite(dt)) return fail(c, RBFSL_EINVAL, "dt must be positive");
    if (dt != c->dt) drop_cardinal(c);
    c->dt = dt;
    return RBFSL_OK;
}

int rbfsl_set_time(rbfsl_ctx *c, double t) {
    if (!c) return fail(nullptr, RBFSL_EINVAL, "null context");
    if (!std::isfinite(t)) return fail(c, RBFSL_EINVAL, "time must be finite");
    c->t = t;
    return RBFSL_OK;
}

int rbfsl_set_tracers(rbfsl_ctx *c, const void *q, int64_t N, int T, int dtype, int mem) {
    if (!c) return fail(nullptr, RBFSL_EINVAL, "null context");
    if (!c->X) return fail(c, RBFSL_ENOTCONF, "set_nodes must come before set_tracers");
    if (!q || N != c->N || T < 1 || (dtype != RBFSL_F64 && dtype != RBFSL_F32) ||
        (mem != RBFSL_HOST && mem != RBFSL_DEVICE))
        return fail(c, RBFSL_EINVAL, "set_tracers: bad arguments");
    DeviceGuard g(c->device);
    const int64_t cnt = N * (int64_t)T;
    if (T != c->T || !c->q) {
        CTX_TRY(c, cudaStreamSynchronize(c->stream));
        if (c->method != RBFSL_LOCAL) release_prepared(c);  // per-field buffers depend on T
        cudaFree(c->q); cudaFree(c->q_next);
        c->q = c->q_next = nullptr;
        int rc;
        // 8 bytes per element whatever the precision: either buffer can stage the other
        // element type during the conversions of set_tracers / get_q.
        if ((rc = dalloc(c, &c->q, cnt * 8))) return rc;
        if ((rc = dalloc(c, &c->q_next, cnt * 8))) return rc;
        c->T = T;
    }
    const int in_es = dtype == RBFSL_F64 ? 8 : 4;
    const unsigned blocks = (unsigned)((cnt + 255) / 256);
    const cudaMemcpyKind kind = mem == RBFSL_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (c->precision == RBFSL_FP64 && dtype == RBFSL_F64) {
        CTX_TRY(c, cudaMemcpyAsync(c->q, q, cnt * 8, kind, c->stream));
    } else {
        // stage the caller's type in q_next, convert into q (FP64, or FP32 pairs when mixed)
        CTX_TRY(c, cudaMemcpyAsync(c->q_next, q, cnt * in_es, kind, c->stream));
        if (c->precision == RBFSL_FP64)
            convert_kernel<float, double><<<blocks, 256, 0, c->stream>>>((const float *)c->q_next, (double *)c->q, cnt);
        else if (dtype == RBFSL_F64)
            to_pair_kernel<double><<<blocks, 256, 0, c->stream>>>((const double *)c->q_next, (float2 *)c->q, cnt);
        else
            to_pair_kernel<float><<<blocks, 256, 0, c->stream>>>((const float *)c->q_next, (float2 *)c->q, cnt);
        CTX_RC(c, launch_status("set_tracers convert"));
    }
    if (mem == RBFSL_HOST) CTX_TRY(c, cudaStreamSynchronize(c->stream));
    c->steps_done = 0;
    return RBFSL_OK;
}

int rbfsl_step(rbfsl_ctx *c, int nsteps) {
    if (!c) return fail(nullptr, RBFSL_EINVAL, "null context");
    if (nsteps < 0) return fail(c, RBFSL_EINVAL, "nsteps < 0");
    DeviceGuard g(c->device);
    int rc = prepare(c);
    if (rc) return rc;
    for (int s = 0; s < nsteps; ++s)
        if ((rc = one_step(c))) return rc;
    return RBFSL_OK;
}

int rbfsl_get_q(rbfsl_ctx *c, void *out, int dtype, int mem) {
    if (!c) return fail(nullptr, RBFSL_EINVAL, "null context");
    if (!c->q) return fail(c, RBFSL_ENOTCONF, "no tracers");
    if (!out || (dtype != RBFSL_F64 && dtype != RBFSL_F32) || (mem != RBFSL_HOST && mem != RBFSL_DEVICE))
        return fail(c, RBFSL_EINVAL, "get_q: bad arguments");
    DeviceGuard g(c->device);
    const int out_es = dtype == RBFSL_F64 ? 8 : 4;
    const int64_t cnt = c->N * (int64_t)c->T;
    const cudaMemcpyKind kind = mem == RBFSL_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (c->precision == RBFSL_FP64 && dtype == RBFSL_F64) {
        CTX_TRY(c, cudaMemcpyAsync(out, c->q, cnt * 8, kind, c->stream));
    } else {
        const unsigned blocks = (unsigned)((cnt + 255) / 256);
        if (c->precision == RBFSL_FP64)
            convert_kernel<double, float><<<blocks, 256, 0, c->stream>>>((const double *)c->q, (float *)c->q_next, cnt);
        else if (dtype == RBFSL_F64)
            from_pair_kernel<double><<<blocks, 256, 0, c->stream>>>((const float2 *)c->q, (double *)c->q_next, cnt);
        else
            from_pair_kernel<float><<<blocks, 256, 0, c->stream>>>((const float2 *)c->q, (float *)c->q_next, cnt);
        CTX_RC(c, launch_status("get_q convert"));
        CTX_TRY(c, cudaMemcpyAsync(out, c->q_next, cnt * out_es, kind, c->stream));
    }
    if (mem == RBFSL_HOST) CTX_TRY(c, cudaStreamSynchronize(c->stream));
    return RBFSL_OK;
}

int rbfsl_get_stats(rbfsl_ctx *c, rbfsl_stats *out) {
    if (!c || !out) return fail(c, RBFSL_EINVAL, "get_stats: null argument");
    DeviceGuard g(c->device);
    CTX_TRY(c, cudaStreamSynchronize(c->stream));
    std::memset(out, 0, sizeof(*out));
    if (c->ctr) {
        unsigned long long h[3] = {0, 0, 0};
        CTX_TRY(c, cudaMemcpy(h, c->ctr, sizeof(h), cudaMemcpyDeviceToHost));
        out->singular_points = (int64_t)h[0];
        out->knn_failures = (int64_t)h[1];
        out->uncovered_points = (int64_t)h[2];
    }
    if (c->dev_err) {
        int32_t e = 0;
        CTX_TRY(c, cudaMemcpy(&e, c->dev_err, sizeof(e), cudaMemcpyDeviceToHost));
        out->device_timeouts = e != 0;
    }
    out->steps_done = c->steps_done;
    out->time = c->t;
    out->device_bytes = c->bytes;
    out->global_cholesky = c->global_cholesky;
    return RBFSL_OK;
}

int rbfsl_last_step_buffers(rbfsl_ctx *c, const double **xi, const int32_t **idx, const void **w) {
    if (!c) return fail(nullptr, RBFSL_EINVAL, "null context");
    if (xi) *xi = c->xi;
    if (idx) *idx = c->I;
    if (w) *w = c->W;
    return RBFSL_OK;
}

}  // extern "C"
