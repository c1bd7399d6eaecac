// RBF partition of unity (Sec. 2.3, Eqs. wght_func, bspline, pu_func, PU_interp; Sec. 3.3).
//
// Set-up: patches are the spherical caps |x - omega_l| < R around given centres; members are
// found by a radius query on the node grid and sorted by node index; each patch's augmented
// saddle-point matrix (Eq. rbf_poly_linsys, n_l nodes + (ell+1)^2 harmonics) is factorised
// once by LU with partial pivoting in FP64 and stored with its row order.
// Per step: (1) the patch coefficients [c; d] = A~_l^-1 [q(X_l); 0] for all tracers, one block
// per patch (forward and back substitution with the stored factors); (2) for each evaluation
// point, the patches that contain it (radius query on the centre grid), their interpolants
// s_l (Eq. rbf_poly) blended with the weights phi(|p - omega_l| / R) / sum phi (Eq. pu_func).
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"


namespace rbfsl {

constexpr int kPuMaxMembers = RBFSL_MAX_SYSTEM - 16;  // ell = 3 leaves 144 nodes per patch
constexpr int kPuMaxCand = 256;                         // members gathered per patch
constexpr int kPuMaxPatches = 32;                       // patches containing one point

__device__ __forceinline__ double pu_phi(int kind, double r) {
    if (r >= 1.0) return 0.0;
    if (kind == 0) {  // Wendland C2
        const double a = 1.0 - r;
        return a * a * a * a * (4.0 * r + 1.0);
    }
    if (r < 0.5) return 2.0 / 3.0 + 4.0 * (r - 1.0) * r * r;  // cubic B-spline, Eq. bspline
    const double a = r - 1.0;
    return -4.0 / 3.0 * a * a * a;
}

// Patch membership: count (members == nullptr) or gather + sort (members != nullptr).
__global__ void __launch_bounds__(128) pu_members_kernel(KnnGrid g, const double *__restrict__ Om,
                                                         int64_t Mp, double R,
                                                         int32_t *__restrict__ counts,
                                                         const int64_t *__restrict__ mstart,
                                                         int32_t *__restrict__ members) {
    __shared__ int buf[4][kPuMaxCand];
    __shared__ int cnt[4];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t l = (int64_t)blockIdx.x * 4 + warp;
    if (l >= Mp) return;
    const double ox = Om[3 * l], oy = Om[3 * l + 1], oz = Om[3 * l + 2];
    if (lane == 0) cnt[warp] = 0;
    __syncwarp();
    grid_ball_foreach(g, ox, oy, oz, R * (1.0 + 1e-9) + 1e-15, lane, [&](int p) {
        const double d2 = sqdist_rn(ox, oy, oz, g.sx[p], g.sy[p], g.sz[p]);
        if (sqrt(d2) < R) {
            const int slot = atomicAdd(&cnt[warp], 1);
            if (slot < kPuMaxCand) buf[warp][slot] = g.sid[p];
        }
    });
    __syncwarp();
    const int n = cnt[warp];
    if (!members) {
        if (lane == 0) counts[l] = n;
        return;
    }
    // sort the member indices ascending (bitonic, padded to a power of two)
    const int nn = min(n, kPuMaxCand);
    int P = 1;
    while (P < nn) P <<= 1;
    for (int i = nn + lane; i < P; i += 32) buf[warp][i] = 0x7fffffff;
    __syncwarp();
    for (int len = 2; len <= P; len <<= 1)
        for (int st = len >> 1; st > 0; st >>= 1) {
            for (int i = lane; i < P; i += 32) {
                const int j = i ^ st;
                if (j > i) {
                    const int a = buf[warp][i], b = buf[warp][j];
                    if ((a > b) == ((i & len) == 0)) { buf[warp][i] = b; buf[warp][j] = a; }
                }
            }
            __syncwarp();
        }
    const int64_t base = mstart[l];
    for (int i = lane; i < nn; i += 32) members[base + i] = buf[warp][i];
}

// Factorise patch l's saddle-point matrix (one block of 128 threads per patch).
__global__ void __launch_bounds__(128) pu_factor_kernel(const double *__restrict__ X,
                                                        const int64_t *__restrict__ mstart,
                                                        const int32_t *__restrict__ members,
                                                        const int64_t *__restrict__ lu_off, int M,
                                                        int ell, int half, double *__restrict__ LU,
                                                        int32_t *__restrict__ perm,
                                                        int32_t *__restrict__ status, int colmajor) {
    extern __shared__ double sm[];
    __shared__ int s_p, s_bad;
    __shared__ int order[RBFSL_MAX_SYSTEM];
    const int64_t l = blockIdx.x;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int n = (int)(mstart[l + 1] - mstart[l]), m = n + M, ld = m | 1;
    const int32_t *I = members + mstart[l];
    double *A = sm, *cx = A + (size_t)m * ld, *cy = cx + n, *cz = cy + n;
    for (int j = t; j < n; j += 128) {
        const int64_t s = I[j];
        cx[j] = X[3 * s]; cy[j] = X[3 * s + 1]; cz[j] = X[3 * s + 2];
    }
    if (t == 0) s_bad = 0;
    for (int i = t; i < m; i += 128) order[i] = i;
    __syncthreads();
    const int P2 = n * (n - 1) / 2;
    for (int p = t; p < P2; p += 128) {
        const int f = p / (n - 1), e = p - f * (n - 1);
        int r, c;
        if (e < n - 1 - f) { r = f; c = f + 1 + e; } else { r = n - 1 - f; c = e + 1; }
        const double dx = cx[r] - cx[c], dy = cy[r] - cy[c], dz = cz[r] - cz[c];
        const double v = phs_from_d2(dx * dx + dy * dy + dz * dz, half);
        A[r * ld + c] = v;
        A[c * ld + r] = v;
    }
    for (int j = t; j < n; j += 128) {
        A[j * ld + j] = 0.0;
        sh_eval(ell, cx[j], cy[j], cz[j], [&](int c, double v) {
            A[j * ld + n + c] = v;
            A[(n + c) * ld + j] = v;
        });
    }
    for (int e = t; e < M * M; e += 128) A[(n + e / M) * ld + n + e % M] = 0.0;
    __syncthreads();
    for (int k = 0; k < m; ++k) {
        if (warp == 0) {
            long long best = -1;
            int bidx = m;
            for (int r = k + lane; r < m; r += 32) {
                const long long v = __double_as_longlong(A[r * ld + k]) & 0x7fffffffffffffffLL;
                if (v > best) { best = v; bidx = r; }
            }
            for (int off = 16; off > 0; off >>= 1) {
                const long long ob = __shfl_xor_sync(0xffffffffu, best, off);
                const int oi = __shfl_xor_sync(0xffffffffu, bidx, off);
                if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
            }
            if (lane == 0) {
                if (best <= 0 || best >= 0x7ff0000000000000LL) { s_bad = 1; bidx = k; }
                s_p = bidx;
                if (bidx != k) { const int o = order[k]; order[k] = order[bidx]; order[bidx] = o; }
            }
        }
        __syncthreads();
        if (s_bad) break;
        const int p = s_p;
        if (p != k)
            for (int c = t; c < m; c += 128) {
                const double tmp = A[k * ld + c]; A[k * ld + c] = A[p * ld + c]; A[p * ld + c] = tmp;
            }
        __syncthreads();
        const double inv = 1.0 / A[k * ld + k];
        for (int r = k + 1 + t; r < m; r += 128) A[r * ld + k] *= inv;
        __syncthreads();
        const int rows = m - k - 1, cols = m - k - 1;
        for (int e = t; e < rows * cols; e += 128) {
            const int r = k + 1 + e / cols, c = k + 1 + e % cols;
            A[r * ld + c] = fma(-A[r * ld + k], A[k * ld + c], A[r * ld + c]);
        }
        __syncthreads();
    }
    if (s_bad) {
        if (t == 0) atomicAdd(status, 1);
        return;
    }
    double *out = LU + lu_off[l];
    if (!colmajor) {
        for (int e = t; e < m * m; e += 128) out[e] = A[(e / m) * ld + e % m];
    } else {  // column-major, upper columns scaled by the reciprocal diagonal, which is stored on
              // the diagonal (centre stencils: the backward substitution multiplies once per row)
        for (int e = t; e < m * m; e += 128) {
            const int c = e / m, r = e % m;
            const double inv = 1.0 / A[c * ld + c];
            out[e] = r == c ? inv : (r < c ? A[r * ld + c] * inv : A[r * ld + c]);
        }
    }
    int32_t *pr = perm + mstart[l] + l * M;
    for (int i = t; i < m; i += 128) pr[i] = order[i];
}

// Patch coefficients for all tracers (one block per patch): Y = P [q(X_l); 0], L U c = Y.
__global__ void __launch_bounds__(128) pu_coef_kernel(const int64_t *__restrict__ mstart,
                                                      const int32_t *__restrict__ members,
                                                      const int64_t *__restrict__ lu_off, int M,
                                                      const double *__restrict__ LU,
                                                      const int32_t *__restrict__ perm,
                                                      const double *__restrict__ q, int T,
                                                      double *__restrict__ coef) {
    extern __shared__ double Y[];
    const int64_t l = blockIdx.x;
    const int t = threadIdx.x;
    const int n = (int)(mstart[l + 1] - mstart[l]), m = n + M;
    const int32_t *I = members + mstart[l];
    const int32_t *pr = perm + mstart[l] + l * M;
    const double *F = LU + lu_off[l];
    for (int e = t; e < m * T; e += 128) {
        const int i = e / T, c = e % T;
        const int src = pr[i];
        Y[e] = src < n ? q[(int64_t)I[src] * T + c] : 0.0;
    }
    __syncthreads();
    for (int r = 0; r < m - 1; ++r) {  // unit lower
        for (int e = t; e < (m - 1 - r) * T; e += 128) {
            const int s = r + 1 + e / T, c = e % T;
            Y[s * T + c] = fma(-F[s * m + r], Y[r * T + c], Y[s * T + c]);
        }
        __syncthreads();
    }
    for (int r = m - 1; r >= 0; --r) {  // upper
        if (t < T) Y[r * T + t] /= F[r * m + r];
        __syncthreads();
        for (int e = t; e < r * T; e += 128) {
            const int s = e / T, c = e % T;
            Y[s * T + c] = fma(-F[s * m + r], Y[r * T + c], Y[s * T + c]);
        }
        __syncthreads();
    }
    double *out = coef + (mstart[l] + l * M) * T;
    for (int e = t; e < m * T; e += 128) out[e] = Y[e];
}

// Per-point patch search of the blend (one warp): the patches whose caps contain p, ordered by
// patch index (the blend's summation order), their distances |p - omega_l|, the harmonics Y(p)
// and the sum of the PU weight function. Returns the patch count, or -1 after writing NaN to the
// point's outputs (via `fail`) and its status: EINVAL when more than kPuMaxPatches patches
// overlap, EUNCOVERED when none contains p.
struct PuPointShared {
    int pl[4][kPuMaxPatches];
    double pd[4][kPuMaxPatches];
    int sl[4][kPuMaxPatches];
    double sd[4][kPuMaxPatches];
    int cnt[4];
    double Ys[4][(RBFSL_MAX_SH_DEGREE + 1) * (RBFSL_MAX_SH_DEGREE + 1)];
};

template <typename Fail>
__device__ __forceinline__ int pu_point_patches(const KnnGrid &cg, double Rr, int wkind, int ell, double px,
                                                double py, double pz, int warp, int lane, PuPointShared &sh,
                                                double &wsum, int32_t *status, int64_t i, Fail fail) {
    if (lane == 0) sh.cnt[warp] = 0;
    __syncwarp();
    grid_ball_foreach(cg, px, py, pz, Rr * (1.0 + 1e-9) + 1e-15, lane, [&](int p) {
        const double d = sqrt(sqdist_rn(px, py, pz, cg.sx[p], cg.sy[p], cg.sz[p]));
        if (d < Rr) {
            const int slot = atomicAdd(&sh.cnt[warp], 1);
            if (slot < kPuMaxPatches) { sh.pl[warp][slot] = cg.sid[p]; sh.pd[warp][slot] = d; }
        }
    });
    __syncwarp();
    if (sh.cnt[warp] > kPuMaxPatches) {  // more overlapping patches than the kernel gathers
        fail();
        if (status && lane == 0) status[i] = RBFSL_EINVAL;
        return -1;
    }
    const int np = sh.cnt[warp];
    if (lane < np) {
        int rank = 0;
        for (int j = 0; j < np; ++j) rank += sh.pl[warp][j] < sh.pl[warp][lane];
        sh.sl[warp][rank] = sh.pl[warp][lane];
        sh.sd[warp][rank] = sh.pd[warp][lane];
    }
    if (lane == 0) sh_eval(ell, px, py, pz, [&](int c, double v) { sh.Ys[warp][c] = v; });
    __syncwarp();
    wsum = 0.0;
    for (int a = 0; a < np; ++a) wsum += pu_phi(wkind, sh.sd[warp][a] / Rr);
    if (np == 0 || !(wsum > 0.0)) {
        fail();
        if (status && lane == 0) status[i] = RBFSL_EUNCOVERED;
        return -1;
    }
    return np;
}

// Blend the patch interpolants at Nq points; one warp per point, tracers in chunks of 16.
// R = double: FP64 throughout; R = float: FP32 kernel values and sums.
template <typename R>
__global__ void __launch_bounds__(128) pu_eval_kernel(KnnGrid cg, double Rr, int wkind,
                                                      const double *__restrict__ X,
                                                      const int64_t *__restrict__ mstart,
                                                      const int32_t *__restrict__ members, int M,
                                                      int ell, int half, const R *__restrict__ coef,
                                                      int T, const double *__restrict__ P,
                                                      int64_t Nq, R *__restrict__ out,
                                                      int32_t *__restrict__ status) {
    constexpr int TC = 16;
    __shared__ PuPointShared sh;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 4 + warp;
    if (i >= Nq) return;
    const double px = P[3 * i], py = P[3 * i + 1], pz = P[3 * i + 2];
    double wsum;
    const int np = pu_point_patches(cg, Rr, wkind, ell, px, py, pz, warp, lane, sh, wsum, status, i, [&] {
        for (int c = lane; c < T; c += 32) out[i * T + c] = (R)NAN;
    });
    if (np < 0) return;
    const R winv = (R)(1.0 / wsum);
    for (int t0 = 0; t0 < T; t0 += TC) {
        const int tc = min(TC, T - t0);
        R acc[TC];
#pragma unroll
        for (int c = 0; c < TC; ++c) acc[c] = R(0);
        for (int a = 0; a < np; ++a) {
            const int64_t l = sh.sl[warp][a];
            const R wl = (R)pu_phi(wkind, sh.sd[warp][a] / Rr) * winv;
            const int n = (int)(mstart[l + 1] - mstart[l]);
            const int32_t *I = members + mstart[l];
            const R *C = coef + (mstart[l] + l * M) * T + t0;
            for (int j = lane; j < n; j += 32) {
                const int64_t s = I[j];
                R f;
                if (sizeof(R) == 8) {
                    const double dx = px - X[3 * s], dy = py - X[3 * s + 1], dz = pz - X[3 * s + 2];
                    f = (R)phs_from_d2(dx * dx + dy * dy + dz * dz, half);
                } else {
                    const float dx = (float)(px - X[3 * s]), dy = (float)(py - X[3 * s + 1]),
                                dz = (float)(pz - X[3 * s + 2]);
                    const float d2 = dx * dx + dy * dy + dz * dz;
                    float v = sqrtf(d2);
                    for (int h = 0; h < half; ++h) v *= d2;
                    f = (R)v;
                }
                f *= wl;
#pragma unroll
                for (int c = 0; c < TC; ++c)
                    if (c < tc) acc[c] = fma(f, C[(int64_t)j * T + c], acc[c]);
            }
            for (int k = lane; k < M; k += 32) {
                const R yv = (R)sh.Ys[warp][k] * wl;
#pragma unroll
                for (int c = 0; c < TC; ++c)
                    if (c < tc) acc[c] = fma(yv, C[(int64_t)(n + k) * T + c], acc[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < TC; ++c) {
            R v = acc[c];
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (lane == 0 && c < tc) out[i * T + t0 + c] = v;
        }
    }
    if (status && lane == 0) status[i] = RBFSL_OK;
}

// The blend for the mixed step: each term's factor (kernel value or harmonic times the
// normalised PU weight) is formed in FP64 as in the FP64 kernel and split into an FP32 pair;
// coefficients are FP32 pairs; the sums are pair arithmetic with FP32 operations (pair_fma,
// then a two-sum reduction over the lanes). The patch sums cancel strongly (sum |c phi| reaches
// ~3e3 |s|), which plain FP32 sums turn into ~1e-4 relative errors; pairs keep ~n 2^-48.
__global__ void __launch_bounds__(128) pu_eval_pair_kernel(KnnGrid cg, double Rr, int wkind,
                                                           const double *__restrict__ X,
                                                           const int64_t *__restrict__ mstart,
                                                           const int32_t *__restrict__ members, int M,
                                                           int ell, int half, const float2 *__restrict__ coef,
                                                           int T, const double *__restrict__ P, int64_t Nq,
                                                           float2 *__restrict__ out, int32_t *__restrict__ status) {
    constexpr int TC = 16;
    __shared__ PuPointShared sh;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 4 + warp;
    if (i >= Nq) return;
    const double px = P[3 * i], py = P[3 * i + 1], pz = P[3 * i + 2];
    double wsum;
    const int np = pu_point_patches(cg, Rr, wkind, ell, px, py, pz, warp, lane, sh, wsum, status, i, [&] {
        for (int c = lane; c < T; c += 32) out[i * T + c] = make_float2(NAN, NAN);
    });
    if (np < 0) return;
    const double winv = 1.0 / wsum;
    for (int t0 = 0; t0 < T; t0 += TC) {
        const int tc = min(TC, T - t0);
        float ah[TC], al[TC];
#pragma unroll
        for (int c = 0; c < TC; ++c) ah[c] = al[c] = 0.f;
        for (int a = 0; a < np; ++a) {
            const int64_t l = sh.sl[warp][a];
            const double wl = pu_phi(wkind, sh.sd[warp][a] / Rr) * winv;
            const int n = (int)(mstart[l + 1] - mstart[l]);
            const int32_t *I = members + mstart[l];
            const float2 *C = coef + (mstart[l] + l * M) * T + t0;
            for (int j = lane; j < n; j += 32) {
                const int64_t s = I[j];
                const double dx = px - X[3 * s], dy = py - X[3 * s + 1], dz = pz - X[3 * s + 2];
                const float2 f = pair_from(phs_from_d2(dx * dx + dy * dy + dz * dz, half) * wl);
#pragma unroll
                for (int c = 0; c < TC; ++c)
                    if (c < tc) pair_fma(f, C[(int64_t)j * T + c], ah[c], al[c]);
            }
            for (int k = lane; k < M; k += 32) {
                const float2 yv = pair_from(sh.Ys[warp][k] * wl);
#pragma unroll
                for (int c = 0; c < TC; ++c)
                    if (c < tc) pair_fma(yv, C[(int64_t)(n + k) * T + c], ah[c], al[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < TC; ++c) {
            float h = ah[c], lo = al[c];
            for (int off = 16; off > 0; off >>= 1) {  // pair sums across the lanes (two-sum)
                const float oh = __shfl_xor_sync(0xffffffffu, h, off), ol = __shfl_xor_sync(0xffffffffu, lo, off);
                const float s2 = h + oh, bp = s2 - h;
                const float e = (h - (s2 - bp)) + (oh - bp);
                lo = lo + (ol + e);
                h = s2;
            }
            if (lane == 0 && c < tc) out[i * T + t0 + c] = pair_norm(h, lo);
        }
    }
    if (status && lane == 0) status[i] = RBFSL_OK;
}

// Factorise Mp stencil / patch systems given in CSR form (used by RBF-PU and by the local
// method's centre stencils). Dynamic shared memory sized for the largest system.
int launch_stencil_factor(const double *X, const int64_t *mstart, const int32_t *members,
                          const int64_t *lu_off, int64_t count, int max_n, int M, int ell,
                          int power, double *LU, int32_t *perm, int32_t *status, cudaStream_t s,
                          int colmajor) {
    int rc = sh_tables_init();
    if (rc) return rc;
    const int mmax = max_n + M;
    const int smem = ((mmax * (mmax | 1)) + 3 * max_n) * (int)sizeof(double);
    RBFSL_CUDA_TRY(cudaFuncSetAttribute(pu_factor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    pu_factor_kernel<<<(unsigned)count, 128, smem, s>>>(X, mstart, members, lu_off, M, ell, (power - 1) / 2,
                                                        LU, perm, status, colmajor);
    return launch_status("stencil_factor");
}

__global__ void pu_to_pairs(const double *__restrict__ in, float2 *__restrict__ out, int64_t n) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n) out[e] = pair_from(in[e]);
}

template <typename A, typename B>
__global__ void pu_convert(const A *__restrict__ in, B *__restrict__ out, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = (B)in[i];
}

void pu_free(rbfsl_pu *u) {
    if (u->nodes_ix) rbfsl_knn_index_destroy(u->nodes_ix);
    if (u->centers_ix) rbfsl_knn_index_destroy(u->centers_ix);
    cudaFree(u->X); cudaFree(u->centers); cudaFree(u->mstart); cudaFree(u->members);
    cudaFree(u->lu_off); cudaFree(u->LU); cudaFree(u->perm); cudaFree(u->coef);
    cudaFree(u->coef32); cudaFree(u->status);
}

int pu_build(rbfsl_pu *u, const double *x, int64_t N, const double *centers, int64_t Mp, double R,
             int ell, int power, cudaStream_t s) {
    int rc = sh_tables_init();
    if (rc) return rc;
    u->N = N; u->Mp = Mp; u->R = R; u->ell = ell; u->power = power;
    u->M = (ell + 1) * (ell + 1);
    auto alloc = [&](void **p, size_t b) {
        if (cudaMalloc(p, b ? b : 1) != cudaSuccess) {
            cudaGetLastError();
            set_error("pu_build: out of device memory");
            return RBFSL_ENOMEM;
        }
        u->bytes += b;
        return RBFSL_OK;
    };
    if ((rc = alloc((void **)&u->X, N * 3 * sizeof(double)))) return rc;
    if ((rc = alloc((void **)&u->centers, Mp * 3 * sizeof(double)))) return rc;
    if ((rc = alloc((void **)&u->mstart, (Mp + 1) * sizeof(int64_t)))) return rc;
    if ((rc = alloc((void **)&u->lu_off, Mp * sizeof(int64_t)))) return rc;
    if ((rc = alloc((void **)&u->status, sizeof(int32_t)))) return rc;
    RBFSL_CUDA_TRY(cudaMemcpyAsync(u->X, x, N * 3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    RBFSL_CUDA_TRY(cudaMemcpyAsync(u->centers, centers, Mp * 3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    // node grid for membership, centre grid for the evaluation
    const double n_est = N * R * R / 4.0;
    if ((rc = rbfsl_knn_index_create(&u->nodes_ix, u->X, N, std::max(1, (int)n_est), s))) return rc;
    const double a_est = Mp * R * R / 4.0;
    if ((rc = rbfsl_knn_index_create(&u->centers_ix, u->centers, Mp, std::max(1, (int)a_est), s))) return rc;
    u->bytes += u->nodes_ix->bytes + u->centers_ix->bytes;
    // membership counts, host prefix sums
    int32_t *counts = nullptr;
    if ((rc = alloc((void **)&counts, Mp * sizeof(int32_t)))) return rc;
    const unsigned blocks = (unsigned)((Mp + 3) / 4);
    pu_members_kernel<<<blocks, 128, 0, s>>>(grid_view(u->nodes_ix), u->centers, Mp, R, counts, nullptr, nullptr);
    std::vector<int32_t> hc(Mp);
    cudaError_t e = cudaMemcpyAsync(hc.data(), counts, Mp * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(counts);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("pu_build: ") + cudaGetErrorString(e));
        return RBFSL_ECUDA;
    }
    std::vector<int64_t> ms(Mp + 1, 0), lo(Mp, 0);
    int64_t lu_total = 0;
    for (int64_t l = 0; l < Mp; ++l) {
        if (hc[l] < 1) { set_error("pu_build: a patch contains no node"); return RBFSL_EINVAL; }
        if (hc[l] > kPuMaxMembers || hc[l] + u->M > RBFSL_MAX_SYSTEM) {
            set_error("pu_build: a patch holds more nodes than RBFSL_MAX_SYSTEM allows");
            return RBFSL_EINVAL;
        }
        u->max_members = std::max(u->max_members, hc[l]);
        ms[l + 1] = ms[l] + hc[l];
        lo[l] = lu_total;
        const int64_t m = hc[l] + u->M;
        lu_total += m * m;
    }
    if ((rc = alloc((void **)&u->members, ms[Mp] * sizeof(int32_t)))) return rc;
    if ((rc = alloc((void **)&u->LU, lu_total * sizeof(double)))) return rc;
    if ((rc = alloc((void **)&u->perm, (ms[Mp] + Mp * u->M) * sizeof(int32_t)))) return rc;
    RBFSL_CUDA_TRY(cudaMemcpyAsync(u->mstart, ms.data(), (Mp + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    RBFSL_CUDA_TRY(cudaMemcpyAsync(u->lu_off, lo.data(), Mp * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    RBFSL_CUDA_TRY(cudaMemsetAsync(u->status, 0, sizeof(int32_t), s));
    pu_members_kernel<<<blocks, 128, 0, s>>>(grid_view(u->nodes_ix), u->centers, Mp, R, nullptr, u->mstart, u->members);
    if ((rc = launch_stencil_factor(u->X, u->mstart, u->members, u->lu_off, Mp, u->max_members, u->M, ell,
                                    power, u->LU, u->perm, u->status, s, 0)))
        return rc;
    int32_t bad = 0;
    RBFSL_CUDA_TRY(cudaMemcpyAsync(&bad, u->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    RBFSL_CUDA_TRY(cudaStreamSynchronize(s));
    if (bad) {
        set_error("pu_build: " + std::to_string(bad) + " singular patch systems");
        return RBFSL_ESINGULAR;
    }
    return RBFSL_OK;
}

int pu_apply(rbfsl_pu *u, const double *q, int T, const double *p, int64_t Nq, int wkind, int dtype,
             void *out, int32_t *status, cudaStream_t s) {
    if (T != u->coef_T) {
        cudaFree(u->coef); cudaFree(u->coef32);
        u->coef = nullptr; u->coef32 = nullptr;
        int64_t tot = 0;
        RBFSL_CUDA_TRY(cudaMemcpy(&tot, u->mstart + u->Mp, sizeof(int64_t), cudaMemcpyDeviceToHost));
        tot = (tot + u->Mp * u->M) * T;
        if (cudaMalloc(&u->coef, tot * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&u->coef32, tot * sizeof(float2)) != cudaSuccess) {
            cudaGetLastError();
            set_error("pu_apply: out of device memory");
            return RBFSL_ENOMEM;
        }
        u->coef_T = T;
        u->coef_len = tot;
    }
    const int mmax = u->max_members + u->M;
    const int smem = mmax * T * (int)sizeof(double);
    RBFSL_CUDA_TRY(cudaFuncSetAttribute(pu_coef_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    pu_coef_kernel<<<(unsigned)u->Mp, 128, smem, s>>>(u->mstart, u->members, u->lu_off, u->M, u->LU, u->perm,
                                                      q, T, u->coef);
    int rc = launch_status("pu_coef");
    if (rc) return rc;
    if (Nq == 0) return RBFSL_OK;
    const unsigned blocks = (unsigned)((Nq + 3) / 4);
    const KnnGrid cg = grid_view(u->centers_ix);
    const int half = (u->power - 1) / 2;
    if (dtype == RBFSL_F64) {
        pu_eval_kernel<double><<<blocks, 128, 0, s>>>(cg, u->R, wkind, u->X, u->mstart, u->members,
                                                      u->M, u->ell, half, u->coef, T, p, Nq, (double *)out, status);
    } else if (dtype == RBFSL_F32) {
        pu_convert<double, float><<<(unsigned)((u->coef_len + 255) / 256), 256, 0, s>>>(u->coef, (float *)u->coef32,
                                                                                       u->coef_len);
        pu_eval_kernel<float><<<blocks, 128, 0, s>>>(cg, u->R, wkind, u->X, u->mstart, u->members,
                                                     u->M, u->ell, half, (const float *)u->coef32, T, p, Nq,
                                                     (float *)out, status);
    } else {
        pu_to_pairs<<<(unsigned)((u->coef_len + 255) / 256), 256, 0, s>>>(u->coef, (float2 *)u->coef32, u->coef_len);
        pu_eval_pair_kernel<<<blocks, 128, 0, s>>>(cg, u->R, wkind, u->X, u->mstart, u->members, u->M, u->ell,
                                                   half, (const float2 *)u->coef32, T, p, Nq, (float2 *)out, status);
    }
    return launch_status("pu_eval");
}

}  // namespace rbfsl

extern "C" int rbfsl_pu_create(rbfsl_pu **out, const double *x, int64_t N, const double *centers,
                               int64_t Mp, double radius, int ell, int kernel, double kparam,
                               void *stream) {
    using namespace rbfsl;
    RBFSL_CHECK_ARG(out && x && centers, "pu_create: null pointer");
    RBFSL_CHECK_ARG(N >= 1 && N < ((int64_t)1 << 31) && Mp >= 1 && Mp < ((int64_t)1 << 31),
                    "pu_create: bad sizes");
    RBFSL_CHECK_ARG(radius > 0 && radius <= 2.0, "pu_create: radius must be in (0, 2]");
    RBFSL_CHECK_ARG(ell >= 0 && ell <= RBFSL_MAX_SH_DEGREE, "pu_create: ell out of range");
    const int pw = (int)kparam;
    RBFSL_CHECK_ARG(kernel == RBFSL_PHS && (double)pw == kparam && pw >= 1 && (pw & 1),
                    "pu_create: only the PHS kernel r^p with odd p is supported");
    auto *u = new rbfsl_pu();
    RBFSL_CUDA_TRY(cudaGetDevice(&u->device));
    const int rc = pu_build(u, x, N, centers, Mp, radius, ell, pw, (cudaStream_t)stream);
    if (rc != RBFSL_OK) {
        pu_free(u);
        delete u;
        return rc;
    }
    *out = u;
    return RBFSL_OK;
}

extern "C" int rbfsl_pu_destroy(rbfsl_pu *u) {
    if (!u) return RBFSL_OK;
    rbfsl::pu_free(u);
    delete u;
    return RBFSL_OK;
}

extern "C" int rbfsl_pu_apply(rbfsl_pu *u, const double *q, int T, const double *p, int64_t Nq,
                              int weight_kind, int dtype, void *out, int32_t *status, void *stream) {
    using namespace rbfsl;
    RBFSL_CHECK_ARG(u != nullptr, "pu_apply: null handle");
    RBFSL_CHECK_ARG(T >= 1 && Nq >= 0, "pu_apply: bad sizes");
    RBFSL_CHECK_ARG(q && (Nq == 0 || (p && out)), "pu_apply: null pointer");
    RBFSL_CHECK_ARG(weight_kind == RBFSL_PU_WENDLAND || weight_kind == RBFSL_PU_BSPLINE, "pu_apply: bad weight kind");
    RBFSL_CHECK_ARG(dtype == RBFSL_F64 || dtype == RBFSL_F32 || dtype == RBFSL_F32X2, "pu_apply: bad dtype");
    const int mmax = u->max_members + u->M;
    RBFSL_CHECK_ARG((size_t)mmax * T * sizeof(double) <= 200 * 1024, "pu_apply: too many tracers for one call");
    return pu_apply(u, q, T, p, Nq, weight_kind, dtype, out, status, (cudaStream_t)stream);
}
