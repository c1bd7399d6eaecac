// Global RBF interpolation (Sec. 2.1, Eqs. srbfinterp and rbf_linsys; Sec. 3.3): the dense
// N x N interpolation matrix A_X is factorised once (Cholesky as in the paper, or LU with
// partial pivoting where Cholesky breaks down; FP64), then every step solves A_X C = Q for all
// tracers and evaluates the interpolant at the departure points.
//
// Storage is row-major FP64. LU is blocked right-looking: per panel of 64 columns, a
// column-by-column pivot/scale/update, the row swaps applied to the rest of the matrix, a
// unit-lower triangular solve for the panel's block row, and an FP64 tiled GEMM for the
// trailing matrix. Cholesky is blocked on the upper triangle and handed on in LU form. The
// per-step solve works on 64-row blocks of the triangular factors. All of it is bound by
// GB300's FP64 rate.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace rbfsl {

constexpr int kNb = 64;  // panel / block size

__device__ __forceinline__ double radial(int kind, double eps2, double d2) {
    return kind == RBFSL_GAUSS ? exp(-eps2 * d2) : rsqrt(1.0 + eps2 * d2);
}

__global__ void global_assemble(const double *__restrict__ X, int64_t N, int kind, double eps2,
                                double *__restrict__ A) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N * N) return;
    const int64_t i = e / N, j = e - i * N;
    const double dx = X[3 * i] - X[3 * j], dy = X[3 * i + 1] - X[3 * j + 1], dz = X[3 * i + 2] - X[3 * j + 2];
    A[e] = radial(kind, eps2, dx * dx + dy * dy + dz * dz);
}

// Pivot of column j (rows j..N-1), swap rows j and p inside the panel [j0, j0 + nb), scale the
// column below the diagonal. One block. status[0] is set on a zero / non-finite pivot.
__global__ void __launch_bounds__(1024) lu_pivot_scale(double *__restrict__ A, int64_t N, int64_t j,
                                                       int64_t j0, int nb, int32_t *__restrict__ piv,
                                                       int32_t *__restrict__ status) {
    __shared__ long long s_best[32];
    __shared__ int s_idx[32];
    __shared__ int s_p;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    long long best = -1;
    int bidx = (int)N;
    for (int64_t i = j + t; i < N; i += blockDim.x) {
        const long long v = __double_as_longlong(A[i * N + j]) & 0x7fffffffffffffffLL;
        if (v > best) { best = v; bidx = (int)i; }
    }
    for (int off = 16; off > 0; off >>= 1) {
        const long long ob = __shfl_xor_sync(0xffffffffu, best, off);
        const int oi = __shfl_xor_sync(0xffffffffu, bidx, off);
        if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
    }
    if (lane == 0) { s_best[warp] = best; s_idx[warp] = bidx; }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        best = lane < nw ? s_best[lane] : -1;
        bidx = lane < nw ? s_idx[lane] : (int)N;
        for (int off = 16; off > 0; off >>= 1) {
            const long long ob = __shfl_xor_sync(0xffffffffu, best, off);
            const int oi = __shfl_xor_sync(0xffffffffu, bidx, off);
            if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
        }
        if (lane == 0) {
            const bool bad = best <= 0 || best >= 0x7ff0000000000000LL;
            if (bad) { status[0] = RBFSL_ESINGULAR; bidx = (int)j; }
            s_p = bidx;
            piv[j] = bidx;
        }
    }
    __syncthreads();
    const int64_t p = s_p;
    if (p != j) {
        for (int64_t c = j0 + t; c < j0 + nb; c += blockDim.x) {
            const double tmp = A[j * N + c];
            A[j * N + c] = A[p * N + c];
            A[p * N + c] = tmp;
        }
    }
    __syncthreads();
    const double d = A[j * N + j];
    if (d == 0.0) return;
    const double inv = 1.0 / d;
    for (int64_t i = j + 1 + t; i < N; i += blockDim.x) A[i * N + j] *= inv;
}

// Rank-1 update of the panel's remaining columns: A[i][c] -= A[i][j] A[j][c] for i > j,
// j < c < j0 + nb. One warp per row, lanes over the panel columns.
__global__ void lu_panel_update(double *__restrict__ A, int64_t N, int64_t j, int64_t j0, int nb) {
    const int64_t i = j + 1 + ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= N) return;
    const double l = A[i * N + j];
    for (int64_t c = j + 1 + lane; c < j0 + nb; c += 32) A[i * N + c] = fma(-l, A[j * N + c], A[i * N + c]);
}

// Apply the panel's swaps piv[j0 .. j0+nb) to the columns outside the panel.
__global__ void lu_laswp(double *__restrict__ A, int64_t N, int64_t j0, int nb,
                         const int32_t *__restrict__ piv) {
    const int64_t c0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t width = N - nb;
    if (c0 >= width) return;
    const int64_t c = c0 < j0 ? c0 : c0 + nb;
    for (int64_t j = j0; j < j0 + nb && j < N; ++j) {
        const int64_t p = piv[j];
        if (p != j) {
            const double tmp = A[j * N + c];
            A[j * N + c] = A[p * N + c];
            A[p * N + c] = tmp;
        }
    }
}

// U12 = L11^-1 A12 for the block row j0..j0+nb, columns >= j0 + nb (unit lower L11).
__global__ void lu_trsm_row(double *__restrict__ A, int64_t N, int64_t j0, int nb) {
    __shared__ double L[kNb][kNb + 1];
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x)
        L[e / nb][e % nb] = A[(j0 + e / nb) * N + j0 + e % nb];
    __syncthreads();
    const int64_t c = j0 + nb + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= N) return;
    double col[kNb];
#pragma unroll
    for (int r = 0; r < kNb; ++r) col[r] = r < nb ? A[(j0 + r) * N + c] : 0.0;
#pragma unroll
    for (int r = 1; r < kNb; ++r) {
        double s = col[r];
#pragma unroll
        for (int q = 0; q < r; ++q) s = fma(-L[r][q], col[q], s);
        col[r] = s;
    }
#pragma unroll
    for (int r = 1; r < kNb; ++r)
        if (r < nb) A[(j0 + r) * N + c] = col[r];
}

// C[M x Nc] -= A[M x K] B[K x Nc], K <= 64, row-major with leading dimensions lda/ldb/ldc.
// BM x BN output tiles, (BM/4)(BN/4) threads with 4 x 4 outputs each; K is staged through
// shared memory in chunks of 32 (A transposed so that the inner-loop reads are conflict free).
// kTransA: A is given transposed (Am[k * lda + row]); kUpper: only tiles that reach the
// diagonal or above it are updated (the symmetric trailing update of the Cholesky factor).
template <int BM, int BN, bool kTransA = false, bool kUpper = false>
__global__ void __launch_bounds__((BM / 4) * (BN / 4)) gemm_sub_f64(
    const double *__restrict__ Am, int64_t lda, const double *__restrict__ Bm, int64_t ldb,
    double *__restrict__ Cm, int64_t ldc, int64_t M, int64_t Nc, int K) {
    constexpr int KC = 32, NT = (BM / 4) * (BN / 4);
    __shared__ double As[KC][BM + 1];  // As[k][row]
    __shared__ double Bs[KC][BN + 1];  // Bs[k][col]
    const int64_t row0 = blockIdx.y * (int64_t)BM, col0 = blockIdx.x * (int64_t)BN;
    if (kUpper && col0 + BN <= row0) return;  // every element of the tile below the diagonal
    const int t = threadIdx.x;
    const int tr = (t / (BN / 4)) * 4, tc = (t % (BN / 4)) * 4;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += KC) {
        __syncthreads();
        for (int e = t; e < BM * KC; e += NT) {
            if (kTransA) {
                const int k = e / BM, r = e % BM;
                As[k][r] = (row0 + r < M && k0 + k < K) ? Am[(k0 + k) * lda + row0 + r] : 0.0;
            } else {
                const int r = e / KC, k = e % KC;
                As[k][r] = (row0 + r < M && k0 + k < K) ? Am[(row0 + r) * lda + k0 + k] : 0.0;
            }
        }
        for (int e = t; e < KC * BN; e += NT) {
            const int kk = e / BN, c = e % BN;
            Bs[kk][c] = (k0 + kk < K && col0 + c < Nc) ? Bm[(k0 + kk) * ldb + col0 + c] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < KC; ++k) {
            double a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) { a[u] = As[k][tr + u]; b[u] = Bs[k][tc + u]; }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int64_t r = row0 + tr + u;
        if (r >= M) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int64_t c = col0 + tc + v;
            if (c < Nc) Cm[r * ldc + c] -= acc[u][v];
        }
    }
}

int launch_gemm_sub(const double *A, int64_t lda, const double *B, int64_t ldb, double *C,
                    int64_t ldc, int64_t M, int64_t Nc, int K, cudaStream_t s) {
    if (M <= 0 || Nc <= 0 || K <= 0) return RBFSL_OK;
    if (Nc >= 1024) {  // trailing updates of the factorisation: large square tiles
        dim3 grid((unsigned)((Nc + 63) / 64), (unsigned)((M + 63) / 64));
        gemm_sub_f64<64, 64><<<grid, 256, 0, s>>>(A, lda, B, ldb, C, ldc, M, Nc, K);
    } else {  // few right-hand sides (the per-step solve): small tiles for enough blocks
        dim3 grid((unsigned)((Nc + 31) / 32), (unsigned)((M + 31) / 32));
        gemm_sub_f64<32, 32><<<grid, 64, 0, s>>>(A, lda, B, ldb, C, ldc, M, Nc, K);
    }
    return launch_status("gemm_sub_f64");
}

// The solve's trailing update C[M x T] -= A[M x K] B[K x T] (K <= 64, row-major), one warp per
// row of C: lanes over columns (two per lane per 64-column pass), the row's K factor entries held
// by the lanes and broadcast by shuffles, B read through L1. Small-grid GEMM tiles would give a
// block step only about one warp per SM sub-partition; rows per warp keep the rounds balanced.
// Same accumulation order per element as gemm_sub_f64 (k ascending, then subtracted).
__global__ void __launch_bounds__(256) gemm_rows_sub(const double *__restrict__ Am, int64_t lda,
                                                     const double *__restrict__ Bm, int64_t ldb,
                                                     double *__restrict__ Cm, int64_t ldc, int64_t M, int T, int K) {
    const int lane = threadIdx.x & 31;
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= M) return;
    const double a_lo = lane < K ? Am[row * lda + lane] : 0.0;
    const double a_hi = lane + kWarp < K ? Am[row * lda + lane + kWarp] : 0.0;
    for (int c0 = 0; c0 < T; c0 += 2 * kWarp) {
        const int c1 = c0 + lane, c2 = c0 + kWarp + lane;
        double acc1 = 0.0, acc2 = 0.0;
        for (int k = 0; k < K; ++k) {
            const double a = __shfl_sync(0xffffffffu, k < kWarp ? a_lo : a_hi, k & (kWarp - 1));
            if (c1 < T) acc1 = fma(a, Bm[k * ldb + c1], acc1);
            if (c2 < T) acc2 = fma(a, Bm[k * ldb + c2], acc2);
        }
        if (c1 < T) Cm[row * ldc + c1] -= acc1;
        if (c2 < T) Cm[row * ldc + c2] -= acc2;
    }
}

int launch_gemm_rows_sub(const double *A, int64_t lda, const double *B, int64_t ldb, double *C, int64_t ldc,
                         int64_t M, int T, int K, cudaStream_t s) {
    if (M <= 0 || T <= 0 || K <= 0) return RBFSL_OK;
    gemm_rows_sub<<<(unsigned)((M * kWarp + 255) / 256), 256, 0, s>>>(A, lda, B, ldb, C, ldc, M, T, K);
    return launch_status("gemm_rows_sub");
}

int global_factor(double *A, int64_t N, int32_t *piv, int32_t *status, cudaStream_t s) {
    for (int64_t j0 = 0; j0 < N; j0 += kNb) {
        const int nb = (int)std::min<int64_t>(kNb, N - j0);
        for (int64_t j = j0; j < j0 + nb; ++j) {
            lu_pivot_scale<<<1, 1024, 0, s>>>(A, N, j, j0, nb, piv, status);
            if (j + 1 < j0 + nb && j + 1 < N) {
                const int64_t rows = N - j - 1;
                lu_panel_update<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, s>>>(A, N, j, j0, nb);
            }
        }
        if (N > nb) lu_laswp<<<(unsigned)((N - nb + 255) / 256), 256, 0, s>>>(A, N, j0, nb, piv);
        const int64_t rest = N - j0 - nb;
        if (rest > 0) {
            lu_trsm_row<<<(unsigned)((rest + 127) / 128), 128, 0, s>>>(A, N, j0, nb);
            int rc = launch_gemm_sub(A + (j0 + nb) * N + j0, N, A + j0 * N + j0 + nb, N,
                                     A + (j0 + nb) * N + j0 + nb, N, rest, rest, nb, s);
            if (rc) return rc;
        }
        int rc = launch_status("global_factor");
        if (rc) return rc;
    }
    return RBFSL_OK;
}

// ---- Cholesky factorisation A_X = R^T R (Sec. 3.3: the paper's choice for its positive-definite
// IMQ matrix), blocked right-looking on the upper triangle: the 64 x 64 diagonal block in one
// CTA, the block row by triangular solves with R11^T, the trailing upper triangle by
// R12^T R12 (tiles below the diagonal skipped: half of elimination's flops). status[0] is set
// at a non-positive or non-finite pivot (breakdown; the caller falls back to LU).
__global__ void __launch_bounds__(1024) chol_diag(double *__restrict__ A, int64_t N, int64_t j0, int nb,
                                                  int32_t *__restrict__ status) {
    __shared__ double D[kNb][kNb + 1];
    __shared__ int bad;
    const int t = threadIdx.x;
    if (t == 0) bad = 0;
    for (int e = t; e < nb * nb; e += blockDim.x) D[e / nb][e % nb] = A[(j0 + e / nb) * N + j0 + e % nb];
    __syncthreads();
    for (int k = 0; k < nb; ++k) {
        if (t == 0) {
            const double d = D[k][k];
            if (!(d > 0.0) || !isfinite(d)) bad = 1;
            D[k][k] = sqrt(d);
        }
        __syncthreads();
        const double r = D[k][k];
        for (int c = k + 1 + t; c < nb; c += blockDim.x) D[k][c] /= r;
        __syncthreads();
        const int w = nb - k - 1;  // upper part of the remaining block: rows i, columns c >= i
        for (int e = t; e < w * w; e += blockDim.x) {
            const int i = k + 1 + e / w, c = k + 1 + e % w;
            if (c >= i) D[i][c] = fma(-D[k][i], D[k][c], D[i][c]);
        }
        __syncthreads();
    }
    for (int e = t; e < nb * nb; e += blockDim.x) {
        const int i = e / nb, c = e % nb;
        if (c >= i) A[(j0 + i) * N + j0 + c] = D[i][c];
    }
    if (t == 0 && bad) status[0] = RBFSL_ESINGULAR;
}

// R12 = R11^-T A12 for the block row j0..j0+nb, columns >= j0 + nb: thread per column.
__global__ void chol_trsm_row(double *__restrict__ A, int64_t N, int64_t j0, int nb) {
    __shared__ double R[kNb][kNb + 1];
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x)
        R[e / nb][e % nb] = A[(j0 + e / nb) * N + j0 + e % nb];
    __syncthreads();
    const int64_t c = j0 + nb + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= N) return;
    double col[kNb];
#pragma unroll
    for (int r = 0; r < kNb; ++r) col[r] = r < nb ? A[(j0 + r) * N + c] : 0.0;
#pragma unroll
    for (int r = 0; r < kNb; ++r) {
        if (r >= nb) break;
        double s = col[r];
#pragma unroll
        for (int q = 0; q < r; ++q) s = fma(-R[q][r], col[q], s);
        col[r] = s / R[r][r];
    }
#pragma unroll
    for (int r = 0; r < kNb; ++r)
        if (r < nb) A[(j0 + r) * N + c] = col[r];
}

// The factor in the elimination's form: L = R^T diag(R)^-1 below the diagonal (unit), U =
// diag(R) R on and above it, so that the per-step solve takes it unchanged (identity row order).
__global__ void chol_to_lu_lower(double *__restrict__ A, int64_t N, double *__restrict__ dg) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N * N) return;
    const int64_t r = e / N, c = e - r * N;
    if (r == c) dg[r] = A[e];
    else if (r > c) A[e] = A[c * N + r] / A[c * N + c];
}
__global__ void chol_to_lu_upper(double *__restrict__ A, int64_t N, const double *__restrict__ dg) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N * N) return;
    const int64_t r = e / N, c = e - r * N;
    if (c >= r) A[e] = dg[r] * A[e];
}

int global_factor_chol(double *A, int64_t N, double *dg, int32_t *status, cudaStream_t s) {
    for (int64_t j0 = 0; j0 < N; j0 += kNb) {
        const int nb = (int)std::min<int64_t>(kNb, N - j0);
        chol_diag<<<1, 1024, 0, s>>>(A, N, j0, nb, status);
        const int64_t rest = N - j0 - nb;
        if (rest > 0) {
            chol_trsm_row<<<(unsigned)((rest + 127) / 128), 128, 0, s>>>(A, N, j0, nb);
            const double *R12 = A + j0 * N + j0 + nb;
            double *A22 = A + (j0 + nb) * N + j0 + nb;
            dim3 grid((unsigned)((rest + 63) / 64), (unsigned)((rest + 63) / 64));
            gemm_sub_f64<64, 64, true, true><<<grid, 256, 0, s>>>(R12, N, R12, N, A22, N, rest, rest, nb);
        }
        int rc = launch_status("global_factor_chol");
        if (rc) return rc;
    }
    const int64_t NN = N * N;
    chol_to_lu_lower<<<(unsigned)((NN + 255) / 256), 256, 0, s>>>(A, N, dg);
    chol_to_lu_upper<<<(unsigned)((NN + 255) / 256), 256, 0, s>>>(A, N, dg);
    return launch_status("global_factor_chol");
}

// ---- per-step solve C = A_X^-1 Q with the factor (row-major, T columns)
__global__ void gather_rows(const double *__restrict__ Q, const int32_t *__restrict__ perm,
                            int64_t N, int T, double *__restrict__ Y) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N * T) return;
    const int64_t i = e / T;
    Y[e] = Q[(int64_t)perm[i] * T + (e - i * T)];
}

// In-place solve of the diagonal block (rows r0..r0+nb) of the factor: unit lower (forward) or
// upper with stored diagonal (backward), column-oriented substitution, one warp per right-hand
// side, kTrsmCols warps (right-hand sides) per block. A 64 x 64 triangular solve with T
// right-hand sides is T * 64^2 / 2 FP64 FMAs, too many for one SM's FP64 rate, so the columns go
// to different SMs. The block's warps stage the diagonal block in shared memory together (eight
// loads in flight per thread), then lane l of each warp holds rows l and l + 32 in registers and
// each step broadcasts the finished value by a shuffle.
constexpr int kTrsmCols = 4;

__global__ void __launch_bounds__(kTrsmCols * 32) trsm_diag_col(const double *__restrict__ LU, int64_t N, int64_t r0,
                                                                int nb, double *__restrict__ Y, int T, int upper) {
    __shared__ double D[kNb][kNb + 1];
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * kTrsmCols + (threadIdx.x >> 5);
    const int nn = nb * nb;
    for (int e0 = threadIdx.x; e0 < nn; e0 += 8 * kTrsmCols * kWarp) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * kTrsmCols * kWarp;
            v[u] = e < nn ? LU[(r0 + e / nb) * N + r0 + e % nb] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * kTrsmCols * kWarp;
            if (e < nn) D[e / nb][e % nb] = v[u];
        }
    }
    __syncthreads();
    if (c >= T) return;
    double y0 = lane < nb ? Y[(r0 + lane) * T + c] : 0.0;
    double y1 = lane + kWarp < nb ? Y[(r0 + lane + kWarp) * T + c] : 0.0;
    const int s0 = lane, s1 = lane + kWarp;
    if (!upper) {
        for (int r = 0; r < nb - 1; ++r) {
            const double yr = __shfl_sync(0xffffffffu, r < kWarp ? y0 : y1, r & (kWarp - 1));
            if (r < kWarp && s0 > r && s0 < nb) y0 = fma(-D[s0][r], yr, y0);  // rows < 32 done after r = 31
            if (s1 > r && s1 < nb) y1 = fma(-D[s1][r], yr, y1);
        }
    } else {
        // reciprocal pivots, all at once, so that a step's multiply replaces a division
        const double i0 = lane < nb ? 1.0 / D[lane][lane] : 0.0;
        const double i1 = lane + kWarp < nb ? 1.0 / D[lane + kWarp][lane + kWarp] : 0.0;
        for (int r = nb - 1; r >= 0; --r) {
            if (r < kWarp) {
                if (lane == r) y0 *= i0;
            } else if (lane == r - kWarp) {
                y1 *= i1;
            }
            const double yr = __shfl_sync(0xffffffffu, r < kWarp ? y0 : y1, r & (kWarp - 1));
            if (s0 < r) y0 = fma(-D[s0][r], yr, y0);
            if (r > kWarp && s1 < r) y1 = fma(-D[s1][r], yr, y1);  // rows >= 32 done below r = 33
        }
    }
    if (lane < nb) Y[(r0 + lane) * T + c] = y0;
    if (lane + kWarp < nb) Y[(r0 + lane + kWarp) * T + c] = y1;
}

int global_solve(const double *LU, const int32_t *perm, int64_t N, const double *Q, int T,
                 double *C, cudaStream_t s) {
    const int64_t NT = N * T;
    gather_rows<<<(unsigned)((NT + 255) / 256), 256, 0, s>>>(Q, perm, N, T, C);
    // forward: L y = P q
    for (int64_t r0 = 0; r0 < N; r0 += kNb) {
        const int nb = (int)std::min<int64_t>(kNb, N - r0);
        trsm_diag_col<<<(unsigned)((T + kTrsmCols - 1) / kTrsmCols), kTrsmCols * 32, 0, s>>>(LU, N, r0, nb, C, T, 0);
        int rc = launch_gemm_rows_sub(LU + (r0 + nb) * N + r0, N, C + r0 * T, T, C + (r0 + nb) * T, T,
                                      N - r0 - nb, T, nb, s);
        if (rc) return rc;
    }
    // backward: U c = y
    const int64_t last = ((N - 1) / kNb) * kNb;
    for (int64_t r0 = last; r0 >= 0; r0 -= kNb) {
        const int nb = (int)std::min<int64_t>(kNb, N - r0);
        trsm_diag_col<<<(unsigned)((T + kTrsmCols - 1) / kTrsmCols), kTrsmCols * 32, 0, s>>>(LU, N, r0, nb, C, T, 1);
        int rc = launch_gemm_rows_sub(LU + r0, N, C + r0 * T, T, C, T, r0, T, nb, s);
        if (rc) return rc;
    }
    return launch_status("global_solve");
}

// ---- evaluation of the interpolant at Nq points: out[i][t] = sum_j phi(|p_i - x_j|) C[j][t]
// Tiles of TP points x 64 tracers per block (TP = 8 in FP64, 32 in FP32); the kernel values of
// a 32-node chunk are computed once into shared memory and reused by all 64 tracers.
template <typename R, typename O, int TP>
__global__ void __launch_bounds__(TP * 8) global_eval_kernel(const double *__restrict__ P, int64_t Nq,
                                                          const double *__restrict__ X, int64_t N,
                                                          int kind, double eps2,
                                                          const R *__restrict__ C, int T,
                                                          O *__restrict__ out) {
    constexpr int TT = 64, TK = 32, NT = TP * 8;  // NT threads: 2 points x 4 tracers each
    __shared__ R Ph[TP][TK + 1];
    __shared__ R Cs[TK][TT];
    __shared__ double ps[TP][3];
    const int t = threadIdx.x;
    const int64_t p0 = blockIdx.x * (int64_t)TP;
    const int t0 = blockIdx.y * TT;
    if (t < TP * 3) {
        const int64_t pi = p0 + t / 3;
        ps[t / 3][t % 3] = pi < Nq ? P[3 * pi + t % 3] : 0.0;
    }
    // thread owns points (t/16)*2 .. +2 and tracers (t%16)*4 .. +4
    const int pr = (t / 16) * 2, tc = (t % 16) * 4;
    R acc[2][4] = {};
    for (int64_t k0 = 0; k0 < N; k0 += TK) {
        __syncthreads();
        for (int e = t; e < TP * TK; e += NT) {
            const int a = e / TK, b = e % TK;
            const int64_t j = k0 + b;
            R v = R(0);
            if (j < N) {
                if (sizeof(R) == 8) {
                    const double dx = ps[a][0] - X[3 * j], dy = ps[a][1] - X[3 * j + 1], dz = ps[a][2] - X[3 * j + 2];
                    v = (R)radial(kind, eps2, dx * dx + dy * dy + dz * dz);
                } else {
                    const float dx = (float)ps[a][0] - (float)X[3 * j], dy = (float)ps[a][1] - (float)X[3 * j + 1],
                                dz = (float)ps[a][2] - (float)X[3 * j + 2];
                    const float d2 = dx * dx + dy * dy + dz * dz;
                    v = (R)(kind == RBFSL_GAUSS ? __expf(-(float)eps2 * d2) : rsqrtf(1.0f + (float)eps2 * d2));
                }
            }
            Ph[a][b] = v;
        }
        for (int e = t; e < TK * TT; e += NT) {
            const int b = e / TT, c = e % TT;
            const int64_t j = k0 + b;
            Cs[b][c] = (j < N && t0 + c < T) ? C[j * T + t0 + c] : R(0);
        }
        __syncthreads();
#pragma unroll 8
        for (int b = 0; b < TK; ++b) {
            const R f0 = Ph[pr][b], f1 = Ph[pr + 1][b];
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const R cv = Cs[b][tc + v];
                acc[0][v] = fma(f0, cv, acc[0][v]);
                acc[1][v] = fma(f1, cv, acc[1][v]);
            }
        }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int64_t pi = p0 + pr + u;
        if (pi >= Nq) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v)
            if (t0 + tc + v < T) out[pi * T + t0 + tc + v] = (O)acc[u][v];
    }
}

int launch_global_eval(const double *P, int64_t Nq, const double *X, int64_t N, int kind,
                       double eps, const void *C, int T, int dtype, void *out, int out_dtype,
                       cudaStream_t s) {
    if (Nq == 0) return RBFSL_OK;
    dim3 grid((unsigned)((Nq + 31) / 32), (unsigned)((T + 63) / 64));
    const double e2 = eps * eps;
    if (dtype == RBFSL_F64) {
        // 8 points per block (64 threads): four times the blocks of 32, so that the FP64-bound
        // grid spreads evenly over the SMs (N = 10,242: 1,281 blocks instead of 321; 22.4 ->
        // 18.0 ms at T = 64)
        dim3 g8((unsigned)((Nq + 7) / 8), grid.y);
        global_eval_kernel<double, double, 8><<<g8, 64, 0, s>>>(P, Nq, X, N, kind, e2, (const double *)C, T, (double *)out);
    } else if (out_dtype == RBFSL_F32) {
        global_eval_kernel<float, float, 32><<<grid, 256, 0, s>>>(P, Nq, X, N, kind, e2, (const float *)C, T, (float *)out);
    } else {
        global_eval_kernel<float, double, 32><<<grid, 256, 0, s>>>(P, Nq, X, N, kind, e2, (const float *)C, T, (double *)out);
    }
    return launch_status("global_eval");
}

int launch_global_assemble(const double *X, int64_t N, int kind, double eps, double *A, cudaStream_t s) {
    const int64_t NN = N * N;
    global_assemble<<<(unsigned)((NN + 255) / 256), 256, 0, s>>>(X, N, kind, eps * eps, A);
    return launch_status("global_assemble");
}

}  // namespace rbfsl

// ---- C ABI
namespace rbfsl {
// Assemble and factorise; piv (N) and status (1) are device scratch; perm receives the final
// row order. Synchronises the stream.
int global_factor_full(const double *x, int64_t N, int kernel, double eps, double *LU, int32_t *perm,
                       int32_t *piv, int32_t *status, cudaStream_t s) {
    int rc = RBFSL_OK;
    if (cudaMemsetAsync(status, 0, sizeof(int32_t), s) != cudaSuccess) {
        cudaGetLastError();
        set_error("global_factor: memset failed");
        return RBFSL_ECUDA;
    }
    rc = launch_global_assemble(x, N, kernel, eps, LU, s);
    if (rc == RBFSL_OK) rc = global_factor(LU, N, piv, status, s);
    if (rc != RBFSL_OK) return rc;
    std::vector<int32_t> hp(N);
    int32_t hs = 0;
    if (cudaMemcpyAsync(hp.data(), piv, N * sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&hs, status, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        set_error(std::string("global_factor: ") + cudaGetErrorString(cudaGetLastError()));
        return RBFSL_ECUDA;
    }
    // final row order: apply the swaps to the identity
    std::vector<int32_t> order(N);
    for (int64_t i = 0; i < N; ++i) order[i] = (int32_t)i;
    for (int64_t j = 0; j < N; ++j) std::swap(order[j], order[hp[j]]);
    if (cudaMemcpy(perm, order.data(), N * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        set_error("global_factor: copy of the permutation failed");
        return RBFSL_ECUDA;
    }
    if (hs != 0) {
        set_error("global_factor: zero pivot (the interpolation matrix is singular)");
        return RBFSL_ESINGULAR;
    }
    return RBFSL_OK;
}
}  // namespace rbfsl

extern "C" int rbfsl_global_factor(const double *x, int64_t N, int kernel, double eps, double *LU,
                                   int32_t *perm, void *stream) {
    using namespace rbfsl;
    RBFSL_CHECK_ARG(N >= 1 && N <= 200000, "global_factor: N out of range");
    RBFSL_CHECK_ARG(x && LU && perm, "global_factor: null pointer");
    RBFSL_CHECK_ARG((kernel == RBFSL_GAUSS || kernel == RBFSL_IMQ) && eps > 0,
                    "global_factor: kernel must be RBFSL_GAUSS or RBFSL_IMQ with eps > 0");
    int32_t *piv = nullptr, *status = nullptr;
    if (cudaMalloc(&piv, N * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&status, sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(piv);
        set_error("global_factor: out of device memory");
        return RBFSL_ENOMEM;
    }
    const int rc = global_factor_full(x, N, kernel, eps, LU, perm, piv, status, (cudaStream_t)stream);
    cudaFree(piv);
    cudaFree(status);
    return rc;
}

namespace rbfsl {
// Assemble and factorise by Cholesky into the elimination's form (perm = identity). Returns
// RBFSL_ESINGULAR at a breakdown (LU then holds no usable factor). Synchronises the stream.
int global_factor_chol_full(const double *x, int64_t N, int kernel, double eps, double *LU, int32_t *perm,
                            cudaStream_t s) {
    double *dg = nullptr;
    int32_t *status = nullptr;
    if (cudaMalloc(&dg, N * sizeof(double)) != cudaSuccess || cudaMalloc(&status, sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(dg);
        set_error("global_factor_chol: out of device memory");
        return RBFSL_ENOMEM;
    }
    int rc = RBFSL_OK;
    int32_t hs = 0;
    std::vector<int32_t> id(N);
    for (int64_t i = 0; i < N; ++i) id[i] = (int32_t)i;
    if (cudaMemsetAsync(status, 0, sizeof(int32_t), s) != cudaSuccess) rc = RBFSL_ECUDA;
    if (rc == RBFSL_OK) rc = launch_global_assemble(x, N, kernel, eps, LU, s);
    if (rc == RBFSL_OK) rc = global_factor_chol(LU, N, dg, status, s);
    if (rc == RBFSL_OK &&
        (cudaMemcpyAsync(&hs, status, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
         cudaMemcpyAsync(perm, id.data(), N * sizeof(int32_t), cudaMemcpyHostToDevice, s) != cudaSuccess ||
         cudaStreamSynchronize(s) != cudaSuccess)) {
        set_error(std::string("global_factor_chol: ") + cudaGetErrorString(cudaGetLastError()));
        rc = RBFSL_ECUDA;
    }
    cudaFree(dg);
    cudaFree(status);
    if (rc == RBFSL_OK && hs != 0) {
        set_error("global_factor_chol: non-positive pivot (the matrix is not numerically positive definite)");
        rc = RBFSL_ESINGULAR;
    }
    return rc;
}
}  // namespace rbfsl

extern "C" int rbfsl_global_factor_chol(const double *x, int64_t N, int kernel, double eps, double *LU,
                                        int32_t *perm, void *stream) {
    using namespace rbfsl;
    RBFSL_CHECK_ARG(N >= 1 && N <= 200000, "global_factor_chol: N out of range");
    RBFSL_CHECK_ARG(x && LU && perm, "global_factor_chol: null pointer");
    RBFSL_CHECK_ARG((kernel == RBFSL_GAUSS || kernel == RBFSL_IMQ) && eps > 0,
                    "global_factor_chol: kernel must be RBFSL_GAUSS or RBFSL_IMQ with eps > 0");
    return global_factor_chol_full(x, N, kernel, eps, LU, perm, (cudaStream_t)stream);
}

extern "C" int rbfsl_global_solve(const double *LU, const int32_t *perm, int64_t N, const double *q,
                                  int T, double *c, void *stream) {
    using namespace rbfsl;
    RBFSL_CHECK_ARG(N >= 1 && T >= 1, "global_solve: bad sizes");
    RBFSL_CHECK_ARG(LU && perm && q && c && q != c, "global_solve: null or aliased pointer");
    return global_solve(LU, perm, N, q, T, c, (cudaStream_t)stream);
}

extern "C" int rbfsl_global_eval(const double *p, int64_t Nq, const double *x, int64_t N, int kernel,
                                 double eps, const void *c, int T, int dtype, void *out, void *stream) {
    using namespace rbfsl;
    RBFSL_CHECK_ARG(Nq >= 0 && N >= 1 && T >= 1, "global_eval: bad sizes");
    RBFSL_CHECK_ARG(Nq == 0 || (p && x && c && out), "global_eval: null pointer");
    RBFSL_CHECK_ARG((kernel == RBFSL_GAUSS || kernel == RBFSL_IMQ) && eps > 0, "global_eval: bad kernel");
    RBFSL_CHECK_ARG(dtype == RBFSL_F64 || dtype == RBFSL_F32, "global_eval: bad dtype");
    return launch_global_eval(p, Nq, x, N, kernel, eps, c, T, dtype, out, dtype, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------------------
// FP64-accurate evaluation without FP64 products: the kernel matrix Phi(P, X) formed in FP64
// (the same radial function and distance operations as the FP64 evaluation) and stored as FP32
// pairs, the coefficients split into pairs, then Phi C by the FP32-pair product of the cardinal
// form (rbfsl_cardinal_apply): ~2^-48 relative per term against the split-TF32 evaluation's
// ~2^-22, at a fraction of the FP64 products' cost.
namespace rbfsl {

__global__ void phi_pairs_kernel(const double *__restrict__ P, int64_t Nq, const double *__restrict__ X, int64_t N,
                                 int kind, double eps2, float2 *__restrict__ E) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= Nq * N) return;
    const int64_t i = e / N, j = e - i * N;
    const double dx = P[3 * i] - X[3 * j], dy = P[3 * i + 1] - X[3 * j + 1], dz = P[3 * i + 2] - X[3 * j + 2];
    E[e] = pair_from(radial(kind, eps2, dx * dx + dy * dy + dz * dz));
}

__global__ void f64_to_pairs(const double *__restrict__ in, float2 *__restrict__ out, int64_t n) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n) out[e] = pair_from(in[e]);
}

size_t global_eval_pairs_workspace(int64_t Nq, int64_t N, int T) {
    const size_t phi = ((size_t)Nq * N * sizeof(float2) + 255) & ~(size_t)255;
    const size_t cp = ((size_t)N * T * sizeof(float2) + 255) & ~(size_t)255;
    return phi + cp + cardinal_apply_workspace(Nq, N, T);
}

int launch_global_eval_pairs(const double *P, int64_t Nq, const double *X, int64_t N, int kind, double eps,
                             const double *C, int T, float2 *out, void *ws, size_t ws_bytes, cudaStream_t s) {
    if (Nq == 0) return RBFSL_OK;
    const size_t need = global_eval_pairs_workspace(Nq, N, T);
    if (!ws || ws_bytes < need) {
        set_error("global_eval_pairs: workspace too small");
        return RBFSL_EINVAL;
    }
    float2 *E = (float2 *)ws;
    const size_t phi = ((size_t)Nq * N * sizeof(float2) + 255) & ~(size_t)255;
    float2 *Cp = (float2 *)((char *)ws + phi);
    const size_t cp = ((size_t)N * T * sizeof(float2) + 255) & ~(size_t)255;
    void *aws = (char *)ws + phi + cp;
    const int64_t ne = Nq * N, nc = N * (int64_t)T;
    phi_pairs_kernel<<<(unsigned)((ne + 255) / 256), 256, 0, s>>>(P, Nq, X, N, kind, eps * eps, E);
    f64_to_pairs<<<(unsigned)((nc + 255) / 256), 256, 0, s>>>(C, Cp, nc);
    int rc = launch_status("global_eval_pairs");
    if (rc) return rc;
    return launch_cardinal_apply(E, Nq, N, Cp, T, RBFSL_F32X2, out, aws, ws_bytes - phi - cp, s);
}

}  // namespace rbfsl

extern "C" size_t rbfsl_global_eval_pairs_workspace_bytes(int64_t Nq, int64_t N, int T) {
    if (Nq < 0 || N < 1 || T < 1) return 0;
    return rbfsl::global_eval_pairs_workspace(Nq, N, T);
}

extern "C" int rbfsl_global_eval_pairs(const double *p, int64_t Nq, const double *x, int64_t N, int kernel,
                                       double eps, const double *c, int T, void *out, void *workspace,
                                       size_t workspace_bytes, void *stream) {
    using namespace rbfsl;
    RBFSL_CHECK_ARG(Nq >= 0 && N >= 1 && T >= 1, "global_eval_pairs: bad sizes");
    RBFSL_CHECK_ARG(Nq == 0 || (p && x && c && out && workspace), "global_eval_pairs: null pointer");
    RBFSL_CHECK_ARG((kernel == RBFSL_GAUSS || kernel == RBFSL_IMQ) && eps > 0, "global_eval_pairs: bad kernel");
    RBFSL_CHECK_ARG(((uintptr_t)workspace & 255) == 0, "global_eval_pairs: workspace must be 256-byte aligned");
    return launch_global_eval_pairs(p, Nq, x, N, kernel, eps, c, T, (float2 *)out, workspace, workspace_bytes,
                                    (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------------------
// Allocation-free variant of rbfsl_global_factor (no counterpart in the paper).
//
// Some callers cannot call cudaMalloc at the point where they factorise: a serving process
// whose allocator owns the device memory budget, or host code that must not trigger the
// device-wide synchronisation an allocation can cause while other streams are running.
// This variant keeps its scratch -- the pivot row of every elimination step and one status
// word -- in the file-scope device array below, sized for N <= RBFSL_NOALLOC_FACTOR_MAX_N.
// Every GPU that loads the library holds that array (64 KB) until the process exits.
namespace rbfsl {

constexpr int64_t kNoAllocMaxN = RBFSL_NOALLOC_FACTOR_MAX_N;

// [0, N): pivot rows of the elimination; [kNoAllocMaxN]: status word (0 or ESINGULAR).
static __device__ __align__(256) int32_t g_factor_scratch[kNoAllocMaxN + 1];

// Device address of g_factor_scratch for each device, looked up on the first call made on
// that device (the name of a __device__ array in host code is not a device address) and kept
// for the life of the process. Atomic so that host threads making their first calls at the same
// time do not race on the entry (they may both look it up; they store the same address).
static std::atomic<int32_t *> g_factor_scratch_ptr[64];

// Final row order from the recorded swaps (one thread: N <= kNoAllocMaxN).
__global__ void noalloc_row_order(const int32_t *__restrict__ piv, int64_t N, int32_t *__restrict__ perm) {
    for (int64_t i = 0; i < N; ++i) perm[i] = (int32_t)i;
    for (int64_t j = 0; j < N; ++j) {
        const int32_t p = piv[j];
        const int32_t t = perm[j];
        perm[j] = perm[p];
        perm[p] = t;
    }
}

}  // namespace rbfsl

extern "C" int rbfsl_global_factor_noalloc(const double *x, int64_t N, int kernel, double eps,
                                           double *LU, int32_t *perm, void *stream) {
    using namespace rbfsl;
    RBFSL_CHECK_ARG(N >= 1, "global_factor_noalloc: N < 1");
    RBFSL_CHECK_ARG(N <= kNoAllocMaxN,
                    "global_factor_noalloc: N exceeds RBFSL_NOALLOC_FACTOR_MAX_N (16384); "
                    "use rbfsl_global_factor");
    RBFSL_CHECK_ARG(x && LU && perm, "global_factor_noalloc: null pointer");
    RBFSL_CHECK_ARG((kernel == RBFSL_GAUSS || kernel == RBFSL_IMQ) && eps > 0,
                    "global_factor_noalloc: kernel must be RBFSL_GAUSS or RBFSL_IMQ with eps > 0");
    int dev = 0;
    RBFSL_CUDA_TRY(cudaGetDevice(&dev));
    RBFSL_CHECK_ARG(dev >= 0 && dev < 64, "global_factor_noalloc: device index >= 64");
    int32_t *piv = g_factor_scratch_ptr[dev].load(std::memory_order_acquire);
    if (!piv) {
        RBFSL_CUDA_TRY(cudaGetSymbolAddress((void **)&piv, g_factor_scratch));
        g_factor_scratch_ptr[dev].store(piv, std::memory_order_release);
    }
    int32_t *status = piv + kNoAllocMaxN;
    cudaStream_t s = (cudaStream_t)stream;
    // the array keeps the previous call's contents: the status word must start at zero
    RBFSL_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int32_t), s));
    int rc = launch_global_assemble(x, N, kernel, eps, LU, s);
    if (rc == RBFSL_OK) rc = global_factor(LU, N, piv, status, s);
    if (rc != RBFSL_OK) return rc;
    noalloc_row_order<<<1, 1, 0, s>>>(piv, N, perm);
    if ((rc = launch_status("global_factor_noalloc"))) return rc;
    int32_t hs = 0;
    RBFSL_CUDA_TRY(cudaMemcpyAsync(&hs, status, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    RBFSL_CUDA_TRY(cudaStreamSynchronize(s));
    if (hs != 0) {
        set_error("global_factor_noalloc: zero pivot (the interpolation matrix is singular)");
        return RBFSL_ESINGULAR;
    }
    return RBFSL_OK;
}
