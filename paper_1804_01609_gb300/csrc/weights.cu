// Stencil weights of the augmented local RBF interpolant (Sec. 2.2, Eqs. rbf_poly and
// rbf_poly_linsys), one warp per evaluation point, FP64 throughout.
//
// The warp assembles the (n + M) x (n + M + 1) augmented saddle-point system in shared
// memory (M = (ell+1)^2):
//     [ A    P  | phi(|p - x_j|) ]      A_jk = |x_j - x_k|^pw   (PHS, zero diagonal)
//     [ P^T  0  | Y(p)           ]      P_jc = Y_c(x_j)
// and eliminates it with partial pivoting (largest magnitude, smaller row on a tie; the
// pivot search is a warp-shuffle arg-max). Lanes own columns during the rank-1 updates, so
// the pivot row lives in registers and each update is one shared-memory load, one DFMA and
// one store. GB300's FP64 rate is the roofline of this kernel: ~(2/3) m^3 flops per point.
#include <cstdlib>

#include "common.cuh"
#include "kernels.cuh"

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
    int n, ell, half, m, ld;
    int stencil_doubles;  // shared-memory doubles per point
    const double *P;
    int32_t *status;
};

// Shared-memory layout of one point: A (m x ld, the augmented [A~ | b] system), the stencil
// coordinates (3 x n), the inverse pivots (m), one flag word.
__host__ __device__ inline int stencil_doubles(int n, int m, int ld) { return m * ld + 3 * n + m + 1; }

// Trailing update of one elimination step for the rows r0, r0 + NW, r0 + 2 NW, ... < m:
// A[r][j] -= A[r][k] * A[k][j] for the NCH column chunks j = k+1+lane+32c <= m. NCH is a
// compile-time count so that no FP64 instruction is issued for a chunk with no live column
// (a predicated-off DFMA still takes an FP64 issue slot). Rows go two at a time, and the next
// pair's operands are loaded before the current pair is stored, so shared-memory latency
// overlaps the DFMAs.
template <int NW, int NCH>
__device__ __forceinline__ void trailing_update(double *__restrict__ A, int ld, int m, int k,
                                                int r, int lane) {
    double pk[NCH];
    int jc[NCH];
    bool on[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        jc[c] = k + 1 + lane + c * kWarp;
        on[c] = jc[c] <= m;
        pk[c] = on[c] ? A[k * ld + jc[c]] : 0.0;
    }
    if (r + NW < m) {
        double l0 = A[r * ld + k], l1 = A[(r + NW) * ld + k];
        double v0[NCH], v1[NCH];
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            v0[c] = on[c] ? A[r * ld + jc[c]] : 0.0;
            v1[c] = on[c] ? A[(r + NW) * ld + jc[c]] : 0.0;
        }
        for (;;) {
            const int rn = r + 2 * NW;
            const bool more = rn + NW < m;
            double nl0 = 0.0, nl1 = 0.0, nv0[NCH], nv1[NCH];
            if (more) {
                nl0 = A[rn * ld + k];
                nl1 = A[(rn + NW) * ld + k];
            }
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                nv0[c] = (more && on[c]) ? A[rn * ld + jc[c]] : 0.0;
                nv1[c] = (more && on[c]) ? A[(rn + NW) * ld + jc[c]] : 0.0;
            }
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                if (c < NCH - 1 || on[c]) {
                    A[r * ld + jc[c]] = fma(-l0, pk[c], v0[c]);
                    A[(r + NW) * ld + jc[c]] = fma(-l1, pk[c], v1[c]);
                }
            }
            r = rn;
            if (!more) break;
            l0 = nl0;
            l1 = nl1;
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                v0[c] = nv0[c];
                v1[c] = nv1[c];
            }
        }
    }
    if (r < m) {
        const double l0 = A[r * ld + k];
#pragma unroll
        for (int c = 0; c < NCH; ++c)
            if (c < NCH - 1 || on[c]) A[r * ld + jc[c]] = fma(-l0, pk[c], A[r * ld + jc[c]]);
    }
}

// NW warps per point (1 or 4). With NW = 1 a block holds blockDim/32 independent points and
// the group barrier is __syncwarp; with NW = 4 a block is one point and uses __syncthreads.
template <int NW, typename WT>
__global__ void __launch_bounds__(NW == 8 ? 256 : 128) weights_kernel(WeightsArgs a, WT *__restrict__ W) {
    extern __shared__ double smem[];
    constexpr int GT = NW * kWarp;
    const int g = threadIdx.x / GT, t = threadIdx.x % GT;
    const int warp = t >> 5, lane = t & 31;
    const int spb = blockDim.x / GT;
    const int64_t i = (int64_t)blockIdx.x * spb + g;
    if (i >= a.Nq) return;  // NW == 1 only (with NW > 1 the grid has exactly Nq blocks)
    const int n = a.n, m = a.m, ld = a.ld, M = m - n;
    double *A = smem + (size_t)g * a.stencil_doubles;
    double *cx = A + (size_t)m * ld, *cy = cx + n, *cz = cy + n, *invp = cz + n;
    int *flag = reinterpret_cast<int *>(invp + m);
    auto gsync = [] {
        if (NW == 1) __syncwarp(); else __syncthreads();
    };

    if (t == 0) *flag = 0;
    gsync();
    for (int j = t; j < n; j += GT) {
        const int64_t s = a.idx[i * n + j];
        if (s < 0) { *flag = 1; continue; }  // a failed neighbour search leaves -1
        cx[j] = a.X[3 * s];
        cy[j] = a.X[3 * s + 1];
        cz[j] = a.X[3 * s + 2];
    }
    gsync();
    if (*flag) {
        for (int j = t; j < n; j += GT) W[i * n + j] = (WT)NAN;
        if (a.status && t == 0) a.status[i] = RBFSL_EKNN;
        return;
    }
    const double px = a.P[3 * i], py = a.P[3 * i + 1], pz = a.P[3 * i + 2];

    // ---- assembly. RBF block: the n(n-1)/2 pairs j < k are folded into rows of n-1 pairs
    // (row f and row n-1-f together) so that every thread has work.
    const int P2 = n * (n - 1) / 2;
    for (int p = t; p < P2; p += GT) {
        const int f = p / (n - 1), e = p - f * (n - 1);
        int r, c;
        if (e < n - 1 - f) { r = f; c = f + 1 + e; } else { r = n - 1 - f; c = e + 1; }
        const double dx = cx[r] - cx[c], dy = cy[r] - cy[c], dz = cz[r] - cz[c];
        const double v = phs_from_d2(dx * dx + dy * dy + dz * dz, a.half);
        A[r * ld + c] = v;
        A[c * ld + r] = v;
    }
    for (int j = t; j < n; j += GT) {
        A[j * ld + j] = 0.0;
        sh_eval(a.ell, cx[j], cy[j], cz[j], [&](int c, double v) {
            A[j * ld + n + c] = v;
            A[(n + c) * ld + j] = v;
        });
        const double dx = px - cx[j], dy = py - cy[j], dz = pz - cz[j];
        A[j * ld + m] = phs_from_d2(dx * dx + dy * dy + dz * dz, a.half);
    }
    for (int e = t; e < M * M; e += GT) A[(n + e / M) * ld + n + e % M] = 0.0;
    if (t == 0) sh_eval(a.ell, px, py, pz, [&](int c, double v) { A[(n + c) * ld + m] = v; });
    gsync();

    // ---- Gaussian elimination with partial pivoting on [A~ | b]
    for (int k = 0; k < m; ++k) {
        if (warp == 0) {
            // pivot: largest |a_rk| (integer compare of the magnitude bits), smaller row on a tie
            long long best = -1;
            int bidx = m;
            for (int r = k + lane; r < m; r += kWarp) {
                const long long v = __double_as_longlong(A[r * ld + k]) & 0x7fffffffffffffffLL;
                if (v > best) { best = v; bidx = r; }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const long long ob = __shfl_xor_sync(0xffffffffu, best, off);
                const int oi = __shfl_xor_sync(0xffffffffu, bidx, off);
                if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
            }
            if (best <= 0 || best >= 0x7ff0000000000000LL) {  // zero, inf or NaN pivot
                if (lane == 0) *flag = 2;
            } else {
                if (bidx != k) {
                    for (int c = k + lane; c <= m; c += kWarp) {
                        const double tmp = A[k * ld + c];
                        A[k * ld + c] = A[bidx * ld + c];
                        A[bidx * ld + c] = tmp;
                    }
                    __syncwarp();
                }
                const double inv = 1.0 / A[k * ld + k];
                if (lane == 0) invp[k] = inv;
                for (int r = k + 1 + lane; r < m; r += kWarp) A[r * ld + k] *= inv;
            }
        }
        gsync();
        if (*flag) break;
        // trailing update: rows k+1.. cyclic over the NW warps, lanes over the m - k columns
        // k+1..m in chunks of 32 (pivot row in registers)
        switch ((m - k + kWarp - 1) / kWarp) {
            case 1: trailing_update<NW, 1>(A, ld, m, k, k + 1 + warp, lane); break;
            case 2: trailing_update<NW, 2>(A, ld, m, k, k + 1 + warp, lane); break;
            case 3: trailing_update<NW, 3>(A, ld, m, k, k + 1 + warp, lane); break;
            case 4: trailing_update<NW, 4>(A, ld, m, k, k + 1 + warp, lane); break;
            default: trailing_update<NW, 5>(A, ld, m, k, k + 1 + warp, lane); break;
        }
        gsync();
    }
    if (warp != 0) return;
    if (*flag) {
        for (int j = lane; j < n; j += kWarp) W[i * n + j] = (WT)NAN;
        if (a.status && lane == 0) a.status[i] = RBFSL_ESINGULAR;
        return;
    }
    // ---- back substitution on the rhs column (warp 0), with the stored inverse pivots
    for (int r = m - 1; r >= 0; --r) {
        const double xr = A[r * ld + m] * invp[r];
        __syncwarp();
        if (lane == 0) A[r * ld + m] = xr;
        for (int s = lane; s < r; s += kWarp) A[s * ld + m] = fma(-A[s * ld + r], xr, A[s * ld + m]);
        __syncwarp();
    }
    for (int j = lane; j < n; j += kWarp) W[i * n + j] = (WT)A[j * ld + m];
    if (a.status && lane == 0) a.status[i] = RBFSL_OK;
}

template <int NW, typename WT>
int launch_weights_nw(const WeightsArgs &a, int spb, void *w, cudaStream_t s) {
    const int smem = spb * a.stencil_doubles * 8;
    RBFSL_CUDA_TRY(cudaFuncSetAttribute(weights_kernel<NW, WT>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    const unsigned blocks = (unsigned)((a.Nq + spb - 1) / spb);
    weights_kernel<NW, WT><<<blocks, spb * NW * kWarp, smem, s>>>(a, (WT *)w);
    return launch_status("stencil_weights");
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
    a.ld = (a.m + 1) | 1;  // odd stride: column accesses hit distinct banks
    a.stencil_doubles = stencil_doubles(n, a.m, a.ld);
    const int bytes = a.stencil_doubles * 8;
    if (bytes > 40 * 1024) {
        // large systems (m >~ 70): several warps per point so that every SM sub-partition's
        // FP64 unit is fed although only one or two points fit in shared memory.
        // RBFSL_WEIGHTS_WARPS=8 selects eight warps per point (default four).
        static const int nw = [] {
            const char *e = getenv("RBFSL_WEIGHTS_WARPS");
            return (e && atoi(e) == 8) ? 8 : 4;
        }();
        if (nw == 8)
            return w_dtype == RBFSL_F64 ? launch_weights_nw<8, double>(a, 1, w, s)
                                        : launch_weights_nw<8, float>(a, 1, w, s);
        return w_dtype == RBFSL_F64 ? launch_weights_nw<4, double>(a, 1, w, s)
                                    : launch_weights_nw<4, float>(a, 1, w, s);
    }
    const int spb = 4;  // four independent points (warps) per block
    return w_dtype == RBFSL_F64 ? launch_weights_nw<1, double>(a, spb, w, s)
                                : launch_weights_nw<1, float>(a, spb, w, s);
}

// Centre-stencil weights (Sec. 3.3): the departure point p_i uses the stencil of its nearest
// node K_i, whose saddle-point matrix was factorised once (row-major LU of the m x m system,
// row order perm). Per point: b = [phi(|p - x_Sj|); Y(p)], then L U w~ = P b with row-wise
// dot products (lanes over a contiguous factor row, warp-shuffle sums); w = w~[0:n]. One warp
// per point; the factor rows are streamed once, so the kernel is bound by HBM bandwidth
// (8 m^2 bytes per point) and the FP64 rate (2 m^2 flops per point).
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
        for (int j = lane; j < n; j += 32) { W[i * n + j] = (WT)NAN; I[i * n + j] = -1; }
        if (status && lane == 0) status[i] = RBFSL_EKNN;
        return;
    }
    const double px = P[3 * i], py = P[3 * i + 1], pz = P[3 * i + 2];
    for (int j = lane; j < n; j += 32) {
        const int64_t s = Ik[k * n + j];
        I[i * n + j] = (int32_t)s;
        const double dx = px - X[3 * s], dy = py - X[3 * s + 1], dz = pz - X[3 * s + 2];
        b[j] = phs_from_d2(dx * dx + dy * dy + dz * dz, half);
    }
    if (lane == 0) sh_eval(ell, px, py, pz, [&](int c, double v) { b[n + c] = v; });
    __syncwarp();
    const double *F = LU + (size_t)k * m * m;
    const int32_t *pr = perm + (size_t)k * m;
    for (int r = lane; r < m; r += 32) y[r] = b[pr[r]];
    __syncwarp();
    // forward: y_r -= sum_{c<r} L_rc y_c (unit lower)
    for (int r = 1; r < m; ++r) {
        double s = 0.0;
        for (int c = lane; c < r; c += 32) s = fma(F[(size_t)r * m + c], y[c], s);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) y[r] -= s;
        __syncwarp();
    }
    // backward: y_r = (y_r - sum_{c>r} U_rc y_c) / U_rr
    for (int r = m - 1; r >= 0; --r) {
        double s = 0.0;
        for (int c = r + 1 + lane; c < m; c += 32) s = fma(F[(size_t)r * m + c], y[c], s);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) y[r] = (y[r] - s) / F[(size_t)r * m + r];
        __syncwarp();
    }
    for (int j = lane; j < n; j += 32) W[i * n + j] = (WT)y[j];
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
    RBFSL_CHECK_ARG(w_dtype == RBFSL_F64 || w_dtype == RBFSL_F32, "stencil_weights: bad w_dtype");
    RBFSL_CHECK_ARG(Nq == 0 || (x && idx && p && w), "stencil_weights: null pointer");
    return launch_weights(x, idx, Nq, n, ell, pw, p, w, w_dtype, status, (cudaStream_t)stream);
}
