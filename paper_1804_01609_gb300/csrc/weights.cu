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
    int warp_doubles;
    const double *P;
    int32_t *status;
};

template <typename WT>
__global__ void __launch_bounds__(128) weights_direct_kernel(WeightsArgs a, WT *__restrict__ W) {
    extern __shared__ double smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * wpb + warp;
    if (i >= a.Nq) return;
    const int n = a.n, m = a.m, ld = a.ld, M = m - n;
    double *A = smem + (size_t)warp * a.warp_doubles;
    double *cx = A + (size_t)m * ld, *cy = cx + n, *cz = cy + n;

    // ---- stencil coordinates and the evaluation point (a failed neighbour search leaves -1)
    bool bad = false;
    for (int j = lane; j < n; j += kWarp) {
        const int64_t s = a.idx[i * n + j];
        if (s < 0) { bad = true; continue; }
        cx[j] = a.X[3 * s];
        cy[j] = a.X[3 * s + 1];
        cz[j] = a.X[3 * s + 2];
    }
    if (__any_sync(0xffffffffu, bad)) {
        for (int j = lane; j < n; j += kWarp) W[i * n + j] = (WT)NAN;
        if (a.status && lane == 0) a.status[i] = RBFSL_EKNN;
        return;
    }
    const double px = a.P[3 * i], py = a.P[3 * i + 1], pz = a.P[3 * i + 2];
    __syncwarp();

    // ---- assembly: RBF block (symmetric, zero diagonal), harmonics block, zero block, rhs
    for (int r = 0; r < n; ++r) {
        const double xr = cx[r], yr = cy[r], zr = cz[r];
        if (lane == 0) A[r * ld + r] = 0.0;
        for (int c = r + 1 + lane; c < n; c += kWarp) {
            const double dx = xr - cx[c], dy = yr - cy[c], dz = zr - cz[c];
            const double v = phs_from_d2(dx * dx + dy * dy + dz * dz, a.half);
            A[r * ld + c] = v;
            A[c * ld + r] = v;
        }
    }
    for (int j = lane; j < n; j += kWarp) {
        sh_eval(a.ell, cx[j], cy[j], cz[j], [&](int c, double v) {
            A[j * ld + n + c] = v;
            A[(n + c) * ld + j] = v;
        });
        const double dx = px - cx[j], dy = py - cy[j], dz = pz - cz[j];
        A[j * ld + m] = phs_from_d2(dx * dx + dy * dy + dz * dz, a.half);
    }
    for (int e = lane; e < M * M; e += kWarp) A[(n + e / M) * ld + n + e % M] = 0.0;
    if (lane == 0) sh_eval(a.ell, px, py, pz, [&](int c, double v) { A[(n + c) * ld + m] = v; });
    __syncwarp();

    // ---- Gaussian elimination with partial pivoting on [A~ | b]
    bool singular = false;
    for (int k = 0; k < m; ++k) {
        double best = -1.0;
        int bidx = m;
        for (int r = k + lane; r < m; r += kWarp) {
            const double v = fabs(A[r * ld + k]);
            if (v > best) { best = v; bidx = r; }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, off);
            const int oi = __shfl_xor_sync(0xffffffffu, bidx, off);
            if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
        }
        if (!(best > 0.0) || !isfinite(best)) { singular = true; break; }
        if (bidx != k) {
            for (int c = k + lane; c <= m; c += kWarp) {
                const double t = A[k * ld + c];
                A[k * ld + c] = A[bidx * ld + c];
                A[bidx * ld + c] = t;
            }
            __syncwarp();
        }
        const double inv = 1.0 / A[k * ld + k];
        for (int r = k + 1 + lane; r < m; r += kWarp) A[r * ld + k] *= inv;
        __syncwarp();
        // columns k+1..m (m - k of them) in chunks of 32; the pivot row in registers
        const int ncols = m - k;
        double pk[5];
        int jc[5];
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            jc[c] = k + 1 + lane + c * kWarp;
            pk[c] = (c * kWarp < ncols && jc[c] <= m) ? A[k * ld + jc[c]] : 0.0;
        }
        const int nch = (ncols + kWarp - 1) / kWarp;
        int r = k + 1;
        for (; r + 1 < m; r += 2) {
            const double l0 = A[r * ld + k], l1 = A[(r + 1) * ld + k];
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                if (c < nch && jc[c] <= m) {
                    const double v0 = A[r * ld + jc[c]], v1 = A[(r + 1) * ld + jc[c]];
                    A[r * ld + jc[c]] = fma(-l0, pk[c], v0);
                    A[(r + 1) * ld + jc[c]] = fma(-l1, pk[c], v1);
                }
            }
        }
        if (r < m) {
            const double l0 = A[r * ld + k];
#pragma unroll
            for (int c = 0; c < 5; ++c)
                if (c < nch && jc[c] <= m) A[r * ld + jc[c]] = fma(-l0, pk[c], A[r * ld + jc[c]]);
        }
        __syncwarp();
    }

    if (singular) {
        for (int j = lane; j < n; j += kWarp) W[i * n + j] = (WT)NAN;
        if (a.status && lane == 0) a.status[i] = RBFSL_ESINGULAR;
        return;
    }
    // ---- back substitution on the rhs column
    for (int r = m - 1; r >= 0; --r) {
        const double xr = A[r * ld + m] / A[r * ld + r];
        __syncwarp();
        if (lane == 0) A[r * ld + m] = xr;
        for (int s = lane; s < r; s += kWarp) A[s * ld + m] = fma(-A[s * ld + r], xr, A[s * ld + m]);
        __syncwarp();
    }
    for (int j = lane; j < n; j += kWarp) W[i * n + j] = (WT)A[j * ld + m];
    if (a.status && lane == 0) a.status[i] = RBFSL_OK;
}

// Four warps per point, for systems too large to give every SM sub-partition its own warp
// with one warp per point (m > ~70: one m x (m+1) FP64 matrix is ~40-100 KB). Each SM
// sub-partition has its own FP64 unit, so the elimination is spread over 4 warps: warp 0
// picks the pivot, swaps and scales the column; then all warps update the trailing rows
// (row-cyclic over warps, lanes over columns, pivot row in registers).
constexpr int kCtaWarps = 4;

template <typename WT>
__global__ void __launch_bounds__(kCtaWarps * 32) weights_cta_kernel(WeightsArgs a, WT *__restrict__ W) {
    extern __shared__ double smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t i = blockIdx.x;
    const int n = a.n, m = a.m, ld = a.ld, M = m - n;
    double *A = smem;
    double *cx = A + (size_t)m * ld, *cy = cx + n, *cz = cy + n;
    __shared__ int s_flag;

    if (tid == 0) s_flag = 0;
    __syncthreads();
    for (int j = tid; j < n; j += kCtaWarps * kWarp) {
        const int64_t s = a.idx[i * n + j];
        if (s < 0) { s_flag = 1; continue; }
        cx[j] = a.X[3 * s];
        cy[j] = a.X[3 * s + 1];
        cz[j] = a.X[3 * s + 2];
    }
    __syncthreads();
    if (s_flag) {
        for (int j = tid; j < n; j += kCtaWarps * kWarp) W[i * n + j] = (WT)NAN;
        if (a.status && tid == 0) a.status[i] = RBFSL_EKNN;
        return;
    }
    const double px = a.P[3 * i], py = a.P[3 * i + 1], pz = a.P[3 * i + 2];

    // ---- assembly
    for (int r = warp; r < n; r += kCtaWarps) {
        const double xr = cx[r], yr = cy[r], zr = cz[r];
        if (lane == 0) A[r * ld + r] = 0.0;
        for (int c = r + 1 + lane; c < n; c += kWarp) {
            const double dx = xr - cx[c], dy = yr - cy[c], dz = zr - cz[c];
            const double v = phs_from_d2(dx * dx + dy * dy + dz * dz, a.half);
            A[r * ld + c] = v;
            A[c * ld + r] = v;
        }
    }
    for (int j = tid; j < n; j += kCtaWarps * kWarp) {
        sh_eval(a.ell, cx[j], cy[j], cz[j], [&](int c, double v) {
            A[j * ld + n + c] = v;
            A[(n + c) * ld + j] = v;
        });
        const double dx = px - cx[j], dy = py - cy[j], dz = pz - cz[j];
        A[j * ld + m] = phs_from_d2(dx * dx + dy * dy + dz * dz, a.half);
    }
    for (int e = tid; e < M * M; e += kCtaWarps * kWarp) A[(n + e / M) * ld + n + e % M] = 0.0;
    if (tid == 0) sh_eval(a.ell, px, py, pz, [&](int c, double v) { A[(n + c) * ld + m] = v; });
    __syncthreads();

    // ---- Gaussian elimination with partial pivoting on [A~ | b]
    for (int k = 0; k < m; ++k) {
        if (warp == 0) {
            double best = -1.0;
            int bidx = m;
            for (int r = k + lane; r < m; r += kWarp) {
                const double v = fabs(A[r * ld + k]);
                if (v > best) { best = v; bidx = r; }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, off);
                const int oi = __shfl_xor_sync(0xffffffffu, bidx, off);
                if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
            }
            if (!(best > 0.0) || !isfinite(best)) {
                if (lane == 0) s_flag = 2;
            } else {
                if (bidx != k) {
                    for (int c = k + lane; c <= m; c += kWarp) {
                        const double t = A[k * ld + c];
                        A[k * ld + c] = A[bidx * ld + c];
                        A[bidx * ld + c] = t;
                    }
                    __syncwarp();
                }
                const double inv = 1.0 / A[k * ld + k];
                for (int r = k + 1 + lane; r < m; r += kWarp) A[r * ld + k] *= inv;
            }
        }
        __syncthreads();
        if (s_flag) break;
        const int ncols = m - k;
        double pk[5];
        int jc[5];
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            jc[c] = k + 1 + lane + c * kWarp;
            pk[c] = (c * kWarp < ncols && jc[c] <= m) ? A[k * ld + jc[c]] : 0.0;
        }
        const int nch = (ncols + kWarp - 1) / kWarp;
        int r = k + 1 + warp;
        for (; r + kCtaWarps < m; r += 2 * kCtaWarps) {
            const int r1 = r + kCtaWarps;
            const double l0 = A[r * ld + k], l1 = A[r1 * ld + k];
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                if (c < nch && jc[c] <= m) {
                    const double v0 = A[r * ld + jc[c]], v1 = A[r1 * ld + jc[c]];
                    A[r * ld + jc[c]] = fma(-l0, pk[c], v0);
                    A[r1 * ld + jc[c]] = fma(-l1, pk[c], v1);
                }
            }
        }
        if (r < m) {
            const double l0 = A[r * ld + k];
#pragma unroll
            for (int c = 0; c < 5; ++c)
                if (c < nch && jc[c] <= m) A[r * ld + jc[c]] = fma(-l0, pk[c], A[r * ld + jc[c]]);
        }
        __syncthreads();
    }
    if (warp != 0) return;
    if (s_flag) {
        for (int j = lane; j < n; j += kWarp) W[i * n + j] = (WT)NAN;
        if (a.status && lane == 0) a.status[i] = RBFSL_ESINGULAR;
        return;
    }
    // ---- back substitution on the rhs column (warp 0)
    for (int r = m - 1; r >= 0; --r) {
        const double xr = A[r * ld + m] / A[r * ld + r];
        __syncwarp();
        if (lane == 0) A[r * ld + m] = xr;
        for (int s = lane; s < r; s += kWarp) A[s * ld + m] = fma(-A[s * ld + r], xr, A[s * ld + m]);
        __syncwarp();
    }
    for (int j = lane; j < n; j += kWarp) W[i * n + j] = (WT)A[j * ld + m];
    if (a.status && lane == 0) a.status[i] = RBFSL_OK;
}

int weights_layout(int n, int ell, int *m, int *ld, int *warp_doubles, int *wpb) {
    *m = n + (ell + 1) * (ell + 1);
    *ld = (*m + 1) | 1;  // odd stride: column accesses hit distinct banks
    *warp_doubles = *m * *ld + 3 * n;
    const int per_warp = *warp_doubles * 8;
    *wpb = 100 * 1024 / per_warp;
    *wpb = *wpb < 1 ? 1 : (*wpb > 4 ? 4 : *wpb);
    return per_warp * *wpb;
}

int launch_weights(const double *x, const int32_t *idx, int64_t Nq, int n, int ell, int power,
                   const double *p, void *w, int w_dtype, int32_t *status, cudaStream_t s) {
    if (Nq == 0) return RBFSL_OK;
    int rc = sh_tables_init();
    if (rc != RBFSL_OK) return rc;
    WeightsArgs a{};
    a.X = x; a.idx = idx; a.Nq = Nq; a.n = n; a.ell = ell; a.half = (power - 1) / 2;
    a.P = p; a.status = status;
    int wpb = 1;
    const int smem = weights_layout(n, ell, &a.m, &a.ld, &a.warp_doubles, &wpb);
    const int per_stencil = a.warp_doubles * 8;
    if (per_stencil > 40 * 1024) {
        // large systems: one CTA of four warps per point
        if (w_dtype == RBFSL_F64) {
            RBFSL_CUDA_TRY(cudaFuncSetAttribute(weights_cta_kernel<double>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, per_stencil));
            weights_cta_kernel<double><<<(unsigned)Nq, kCtaWarps * kWarp, per_stencil, s>>>(a, (double *)w);
        } else {
            RBFSL_CUDA_TRY(cudaFuncSetAttribute(weights_cta_kernel<float>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, per_stencil));
            weights_cta_kernel<float><<<(unsigned)Nq, kCtaWarps * kWarp, per_stencil, s>>>(a, (float *)w);
        }
        return launch_status("stencil_weights");
    }
    const unsigned blocks = (unsigned)((Nq + wpb - 1) / wpb);
    if (w_dtype == RBFSL_F64) {
        RBFSL_CUDA_TRY(cudaFuncSetAttribute(weights_direct_kernel<double>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        weights_direct_kernel<double><<<blocks, wpb * kWarp, smem, s>>>(a, (double *)w);
    } else {
        RBFSL_CUDA_TRY(cudaFuncSetAttribute(weights_direct_kernel<float>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        weights_direct_kernel<float><<<blocks, wpb * kWarp, smem, s>>>(a, (float *)w);
    }
    return launch_status("stencil_weights");
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
