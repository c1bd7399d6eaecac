// Stencil weights of the augmented local RBF interpolant (Sec. 2.2, Eqs. rbf_poly and
// rbf_poly_linsys), FP64 throughout.
//
// Each point's group of warps assembles the lower triangle of the symmetric (n + M) x (n + M)
// saddle-point system in shared memory (M = (ell+1)^2):
//     [ A    P ] w~ = [ phi(|p - x_j|) ]      A_jk = |x_j - x_k|^pw   (PHS, zero diagonal)
//     [ P^T  0 ]      [ Y(p)           ]      P_jc = Y_c(x_j)
// and solves it by a blocked Bunch-Kaufman L D L^T factorisation (weights_point_ldl: panels of
// four pivot columns updated on the fly, one trailing update per panel): ~m^3 / 3 flops per
// point, half of Gaussian elimination's, bound by GB300's FP64 rate. Small systems take one warp
// per point (four points per block); larger ones four warps per point, several points per SM so
// that one point's pivot steps overlap the others' trailing updates.
#include "common.cuh"
#include "kernels.cuh"
#include "device_ops.cuh"

namespace rbfsl {

__constant__ ShTables c_sh;

namespace {
bool g_sh_ready[64] = {false};
}

int sh_tables_init() {
    int dev = 0;
    RBFSL_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 64 && g_sh_ready[dev]) return RBFSL_OK;
    ShTables t{};
    const double pi = 3.14159265358979323846;
    for (int m = 0; m <= kMaxL; ++m) {
        double q = 1.0;
        for (int i = 1; i <= m; ++i) q *= (double)(2 * i - 1);
        t.qmm[m] = q;
        for (int l = m; l <= kMaxL; ++l) {
            const int id = l * l + l + m;
            double ratio = 1.0;  // (l-m)! / (l+m)!
            for (int i = l - m + 1; i <= l + m; ++i) ratio /= (double)i;
            t.K[id] = std::sqrt((m == 0 ? 1.0 : 2.0) * (2.0 * l + 1.0) / (4.0 * pi) * ratio);
            if (l == m + 1) {
                t.a[id] = 2.0 * m + 1.0;
                t.b[id] = 0.0;
            } else if (l >= m + 2) {
                t.a[id] = (2.0 * l - 1.0) / (double)(l - m);
                t.b[id] = (double)(l + m - 1) / (double)(l - m);
            }
        }
    }
    RBFSL_CUDA_TRY(cudaMemcpyToSymbol(c_sh, &t, sizeof(t)));
    if (dev < 64) g_sh_ready[dev] = true;
    return RBFSL_OK;
}

struct WeightsArgs {
    const double *X;
    const int32_t *idx;
    int64_t Nq;
    int n, ell, half, m;
    int region_doubles;  // shared-memory doubles per point
    const double *P;
    int32_t *status;
};

// NW warps per point (1 or 4). With NW = 1 a block holds blockDim/32 independent points and
// the group barrier is __syncwarp; with NW > 1 a block is one point and uses __syncthreads.
// At most 72 registers (seven 128-thread blocks per SM, no spills): where shared memory allows
// more than four points per SM (m = 71: 25 KB each) the register file would otherwise cap the
// blocks at five (11.3 against 10.1 ms at N = 40,962); at m = 109 shared memory caps them at four
// either way.
template <int NW, typename WT>
__global__ void __launch_bounds__(NW == 1 ? 128 : NW * 32, 7) weights_kernel(WeightsArgs a, WT *__restrict__ W) {
    extern __shared__ double smem[];
    constexpr int GT = NW * kWarp;
    const int g = threadIdx.x / GT, t = threadIdx.x % GT;
    const int spb = blockDim.x / GT;
    const int64_t i = (int64_t)blockIdx.x * spb + g;
    if (i >= a.Nq) return;  // NW == 1 only (with NW > 1 the grid has exactly Nq blocks)
    double *R = smem + (size_t)g * a.region_doubles;
    double *w = nullptr;
    const int rc = weights_point_ldl<NW>(R, a.X, a.idx + i * a.n, a.n, a.m, a.ell, a.half,
                                         a.P[3 * i], a.P[3 * i + 1], a.P[3 * i + 2], t, w);
    if (t >= kWarp) return;
    const int n = a.n, lane = t;
    for (int j = lane; j < n; j += kWarp) W[i * n + j] = wcast<WT>(rc == RBFSL_OK ? w[j] : (double)NAN);
    if (a.status && lane == 0) a.status[i] = rc;
}

template <int NW, typename WT>
int launch_weights_nw(const WeightsArgs &a, int spb, void *w, cudaStream_t s) {
    const int smem = spb * a.region_doubles * 8;
    RBFSL_CUDA_TRY(cudaFuncSetAttribute(weights_kernel<NW, WT>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    // all of the unified L1 / shared storage as shared memory: as many points per SM as fit
    RBFSL_CUDA_TRY(cudaFuncSetAttribute(weights_kernel<NW, WT>,
                                        cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    const unsigned blocks = (unsigned)((a.Nq + spb - 1) / spb);
    weights_kernel<NW, WT><<<blocks, spb * NW * kWarp, smem, s>>>(a, (WT *)w);
    return launch_status("stencil_weights");
}

template <int NW>
int launch_weights_typed(const WeightsArgs &a, int spb, void *w, int w_dtype, cudaStream_t s) {
    if (w_dtype == RBFSL_F64) return launch_weights_nw<NW, double>(a, spb, w, s);
    if (w_dtype == RBFSL_F32X2) return launch_weights_nw<NW, float2>(a, spb, w, s);
    return launch_weights_nw<NW, float>(a, spb, w, s);
}

int launch_weights(const double *x, const int32_t *idx, int64_t Nq, int n, int ell, int power,
                   const double *p, void *w, int w_dtype, int32_t *status, cudaStream_t s) {
    if (Nq == 0) return RBFSL_OK;
    int rc = sh_tables_init();
    if (rc != RBFSL_OK) return rc;
    WeightsArgs a{};
    a.X = x; a.idx = idx; a.Nq = Nq; a.n = n; a.ell = ell; a.half = (power - 1) / 2;
    a.P = p; a.status = status;
    a.m = n + (ell + 1) * (ell + 1);
    a.region_doubles = ldl_doubles(n, a.m);
    const int bytes = a.region_doubles * 8;
    if (bytes > kWeightsSmallBytes) {
        // larger systems (m >~ 45): four warps per point (one per SM sub-partition), one point
        // per block, as many blocks per SM as shared memory allows (four at m = 109)
        return launch_weights_typed<4>(a, 1, w, w_dtype, s);
    }
    return launch_weights_typed<1>(a, 4, w, w_dtype, s);  // four independent points (warps) per block
}

// Centre-stencil weights, one warp per point (see center_point): bound by HBM bandwidth
// (8 m^2 bytes of factor per point) and the FP64 rate (2 m^2 flops per point).
template <typename WT>
__global__ void __launch_bounds__(128) center_weights_kernel(
    const double *__restrict__ X, const int32_t *__restrict__ Kc, const int32_t *__restrict__ Ik,
    const double *__restrict__ LU, const int32_t *__restrict__ perm, int64_t Nq, int n, int ell,
    int half, const double *__restrict__ P, int32_t *__restrict__ I, WT *__restrict__ W,
    int32_t *__restrict__ status) {
    extern __shared__ double sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int M = (ell + 1) * (ell + 1), m = n + M;
    const int64_t i = (int64_t)blockIdx.x * 4 + warp;
    if (i >= Nq) return;
    double *b = sm + (size_t)warp * 2 * m, *y = b + m;
    const int64_t k = Kc[i];
    if (k < 0) {
        for (int j = lane; j < n; j += 32) { W[i * n + j] = wcast<WT>((double)NAN); I[i * n + j] = -1; }
        if (status && lane == 0) status[i] = RBFSL_EKNN;
        return;
    }
    for (int j = lane; j < n; j += 32) I[i * n + j] = Ik[k * n + j];
    center_point(X, Ik + k * n, LU + (size_t)k * m * m, perm + (size_t)k * m, n, m, ell, half,
                 P[3 * i], P[3 * i + 1], P[3 * i + 2], b, y, lane);
    for (int j = lane; j < n; j += 32) W[i * n + j] = wcast<WT>(y[j]);
    if (status && lane == 0) status[i] = RBFSL_OK;
}

int launch_center_weights(const double *X, const int32_t *K, const int32_t *Ik, const double *LU,
                          const int32_t *perm, int64_t Nq, int n, int ell, int power,
                          const double *p, int32_t *I, void *w, int w_dtype, int32_t *status,
                          cudaStream_t s) {
    if (Nq == 0) return RBFSL_OK;
    int rc = sh_tables_init();
    if (rc) return rc;
    const int m = n + (ell + 1) * (ell + 1);
    const size_t smem = 4 * 2 * m * sizeof(double);
    const unsigned blocks = (unsigned)((Nq + 3) / 4);
    if (w_dtype == RBFSL_F64)
        center_weights_kernel<double><<<blocks, 128, smem, s>>>(X, K, Ik, LU, perm, Nq, n, ell, (power - 1) / 2,
                                                                p, I, (double *)w, status);
    else if (w_dtype == RBFSL_F32X2)
        center_weights_kernel<float2><<<blocks, 128, smem, s>>>(X, K, Ik, LU, perm, Nq, n, ell, (power - 1) / 2,
                                                                p, I, (float2 *)w, status);
    else
        center_weights_kernel<float><<<blocks, 128, smem, s>>>(X, K, Ik, LU, perm, Nq, n, ell, (power - 1) / 2,
                                                               p, I, (float *)w, status);
    return launch_status("center_weights");
}

}  // namespace rbfsl

extern "C" int rbfsl_stencil_weights(const double *x, int64_t N, const int32_t *idx, int64_t Nq,
                                     int n, int ell, int kernel, double kparam, const double *p,
                                     void *w, int w_dtype, int32_t *status, void *stream) {
    using namespace rbfsl;
    RBFSL_CHECK_ARG(Nq >= 0 && N >= 1, "stencil_weights: bad sizes");
    RBFSL_CHECK_ARG(n >= 1 && n <= N, "stencil_weights: n out of range");
    RBFSL_CHECK_ARG(ell >= 0 && ell <= RBFSL_MAX_SH_DEGREE, "stencil_weights: ell out of range");
    RBFSL_CHECK_ARG(n + (ell + 1) * (ell + 1) <= RBFSL_MAX_SYSTEM,
                    "stencil_weights: n + (ell+1)^2 exceeds RBFSL_MAX_SYSTEM");
    const int pw = (int)kparam;
    RBFSL_CHECK_ARG(kernel == RBFSL_PHS && (double)pw == kparam && pw >= 1 && (pw & 1),
                    "stencil_weights: only the PHS kernel r^p with odd p is supported");
    RBFSL_CHECK_ARG(w_dtype == RBFSL_F64 || w_dtype == RBFSL_F32 || w_dtype == RBFSL_F32X2,
                    "stencil_weights: bad w_dtype");
    RBFSL_CHECK_ARG(Nq == 0 || (x && idx && p && w), "stencil_weights: null pointer");
    return launch_weights(x, idx, Nq, n, ell, pw, p, w, w_dtype, status, (cudaStream_t)stream);
}
