// Cardinal form of the global interpolant (Sec. 2.1, Eqs. srbfinterp and rbf_linsys).
//
// The interpolant of a field q at a point p is phi(p, X) c with A_X c = q, so at a fixed set of
// points P it is E q with E = Phi(P, X) A_X^-1 (Nq x N), the values of the N cardinal functions
// at the points. Under a steady flow the departure points are the same at every step, so E is
// formed once and each semi-Lagrangian step becomes one dense product q <- E q: the per-step
// triangular solves (2 N^2 T FP64 flops, latency-bound) and the kernel evaluations go away.
//
// Build: A_X is symmetric (phi depends on |x_i - x_j| only, and the assembly forms the same
// squared distance for (i, j) and (j, i)), so E^T = A_X^-1 Phi(P, X)^T. Blocks of kCardChunk
// points are solved with the LU factor of rbfsl_global_factor (forward and backward
// substitution, as the per-step solve) and transposed into E, FP64 or FP32 pairs.
//
// Apply: out = E q, 32 x 64 output tiles per block (eight warps of four rows, two columns per
// lane), K staged through shared memory with cp.async double buffering, split over K so that
// the grid covers the SMs evenly; the partial sums are added in split order by cardinal_reduce
// (deterministic). FP64: one DFMA per term, bound by GB300's FP64 rate. FP32 pairs: each term
// in pair arithmetic (pair_fma's 12 FP32 operations), issued as packed FP32x2 instructions for
// a lane's two columns, bound by the FP32 pipe; the rounding is ~2^-48 relative per term,
// FP64-like, because the cardinal values are O(1) and do not cancel (unlike the coefficients c,
// which grow as A_X becomes singular).
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "kernels.cuh"

namespace rbfsl {

namespace {

constexpr int kCardChunk = 512;  // points per block of right-hand sides in the build
constexpr int kApWarps = 8, kApRows = 4, kApBM = kApWarps * kApRows, kApBK = 32, kApCols = 64;
constexpr int kApMaxSplit = 16;

__device__ __forceinline__ double card_radial(int kind, double eps2, double d2) {
    return kind == RBFSL_GAUSS ? exp(-eps2 * d2) : rsqrt(1.0 + eps2 * d2);
}

// B[j][ii] = phi(|x_j - p_(i0+ii)|), N x nc row-major: the right-hand sides A_X E^T = Phi^T.
__global__ void cardinal_rhs(const double *__restrict__ X, int64_t N, const double *__restrict__ P,
                             int64_t i0, int nc, int kind, double eps2, double *__restrict__ B) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N * nc) return;
    const int64_t j = e / nc, ii = e - j * nc;
    const double *p = P + 3 * (i0 + ii);
    const double dx = X[3 * j] - p[0], dy = X[3 * j + 1] - p[1], dz = X[3 * j + 2] - p[2];
    B[e] = card_radial(kind, eps2, dx * dx + dy * dy + dz * dz);
}

// E[i0 + ii][j] = C[j][ii] through a 32 x 32 shared tile (both sides coalesced), converted to
// the storage type (FP64, or an FP32 pair hi = fl(e), lo = fl(e - hi)).
template <typename V>
__global__ void cardinal_store(const double *__restrict__ C, int64_t N, int nc, int64_t i0,
                               V *__restrict__ E) {
    __shared__ double tile[32][33];
    const int64_t j0 = blockIdx.x * 32ll;
    const int ii0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int r = ty; r < 32; r += 8) {
        const int64_t j = j0 + r;
        const int ii = ii0 + tx;
        tile[r][tx] = (j < N && ii < nc) ? C[j * nc + ii] : 0.0;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int ii = ii0 + r;
        const int64_t j = j0 + tx;
        if (ii < nc && j < N) E[(i0 + ii) * N + j] = wcast<V>(tile[tx][r]);
    }
}

__device__ __forceinline__ void cp_async8(void *smem, const void *g, bool valid) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(g), "r"(valid ? 8 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Two adjacent elements of a 16-byte aligned shared row in one 16-byte load.
__device__ __forceinline__ void load_two(const double *p, double &a, double &b) {
    const double2 t = *reinterpret_cast<const double2 *>(p);
    a = t.x;
    b = t.y;
}

// FP64 out = E q over rows [32 bx, 32 bx + 32), columns [64 by, 64 by + 64) and the K range of
// split bz. With one split the sums go to `out` (Nq x T); otherwise to part + bz * Nq * T, and
// cardinal_reduce adds them.
__global__ void __launch_bounds__(kApWarps * 32, 4) cardinal_apply_f64_kernel(
    const double *__restrict__ E, int64_t Nq, int64_t N, const double *__restrict__ q, int T, int64_t kspan,
    double *__restrict__ out, double *__restrict__ part) {
    using V = double;
    __shared__ __align__(16) V Es[2][kApBM][kApBK];
    __shared__ __align__(16) V Qs[2][kApBK][kApCols];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t row0 = blockIdx.x * (int64_t)kApBM;
    const int col0 = blockIdx.y * kApCols;
    const int64_t kb = blockIdx.z * kspan, ke = std::min<int64_t>(N, kb + kspan);
    const int nchunks = (int)((ke - kb + kApBK - 1) / kApBK);

    auto load = [&](int st, int64_t k0) {
#pragma unroll
        for (int u = 0; u < kApBM * kApBK / (kApWarps * 32); ++u) {
            const int e = tid + u * kApWarps * 32;
            const int r = e / kApBK, kk = e % kApBK;
            const int64_t row = row0 + r, k = k0 + kk;
            const bool ok = row < Nq && k < ke;
            cp_async8(&Es[st][r][kk], ok ? E + row * N + k : E, ok);
        }
#pragma unroll
        for (int u = 0; u < kApBK * kApCols / (kApWarps * 32); ++u) {
            const int e = tid + u * kApWarps * 32;
            const int kk = e / kApCols, c = e % kApCols;
            const int64_t k = k0 + kk;
            const bool ok = k < ke && col0 + c < T;
            cp_async8(&Qs[st][kk][c], ok ? q + k * T + col0 + c : q, ok);
        }
    };

    double acc[kApRows][2] = {};
    if (nchunks > 0) load(0, kb);
    cp_async_commit();
    for (int ch = 0; ch < nchunks; ++ch) {
        const int st = ch & 1;
        if (ch + 1 < nchunks) load(st ^ 1, kb + (int64_t)(ch + 1) * kApBK);
        cp_async_commit();
        cp_async_wait1();  // this thread's copies of chunk ch have landed
        __syncthreads();   // and everyone else's
#pragma unroll 4
        for (int kk = 0; kk < kApBK; ++kk) {
            V q0, q1;
            load_two(&Qs[st][kk][2 * lane], q0, q1);
#pragma unroll
            for (int r = 0; r < kApRows; ++r) {
                const V e = Es[st][warp * kApRows + r][kk];  // same address in every lane: broadcast
                acc[r][0] = fma(e, q0, acc[r][0]);
                acc[r][1] = fma(e, q1, acc[r][1]);
            }
        }
        __syncthreads();  // stage st is refilled by the next iteration's load
    }
#pragma unroll
    for (int r = 0; r < kApRows; ++r) {
        const int64_t row = row0 + warp * kApRows + r;
        if (row >= Nq) continue;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int c = col0 + 2 * lane + u;
            if (c >= T) continue;
            if (part) part[(int64_t)blockIdx.z * Nq * T + row * T + c] = acc[r][u];
            else out[row * T + c] = acc[r][u];
        }
    }
}

// ---- FP32-pair product with packed FP32x2 instructions. Each lane owns two columns and the
// pair arithmetic of pair_fma is the same for both, so every operation is issued once for the
// two columns (add/sub/mul/fma .rn.f32x2: two IEEE round-to-nearest FP32 operations). The
// shared tiles hold the operands already packed: a cardinal value e as (e.hi, e.hi, e.lo, e.lo)
// and the two columns' field values as (q0.hi, q1.hi, q0.lo, q1.lo), filled by 4-byte cp.async
// copies. pe (the exact error of the high product and the cross terms) is carried negated,
// using the negated field: round-to-nearest is symmetric, so each rounding equals pair_fma's.
constexpr int kAp2BK = 16;
typedef unsigned long long f2_t;  // two packed FP32 values, element 0 in the low half

__device__ __forceinline__ f2_t f2_mul(f2_t a, f2_t b) {
    f2_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c) {
    f2_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2_t f2_add(f2_t a, f2_t b) {
    f2_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2_t f2_sub(f2_t a, f2_t b) {
    f2_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ void f2_unpack(f2_t v, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}

__device__ __forceinline__ void cp_async4(void *smem, const void *g, bool valid) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(g), "r"(valid ? 4 : 0)
                 : "memory");
}

// (sh, sl) += e * q for both columns: pair_fma's operations, packed.
__device__ __forceinline__ void pair_fma2(f2_t ex, f2_t ey, f2_t qh, f2_t nqh, f2_t nql, f2_t &sh, f2_t &sl) {
    const f2_t p = f2_mul(ex, qh);
    f2_t npe = f2_fma(ex, nqh, p);  // -(e.hi q.hi - p), exact
    npe = f2_fma(ex, nql, npe);     // -(pe + e.hi q.lo)
    npe = f2_fma(ey, nqh, npe);     // -(pe + e.hi q.lo + e.lo q.hi)
    const f2_t s = f2_add(sh, p);   // two-sum of sh and p
    const f2_t bp = f2_sub(s, sh);
    const f2_t err = f2_add(f2_sub(sh, f2_sub(s, bp)), f2_sub(p, bp));
    sl = f2_add(sl, f2_sub(err, npe));
    sh = s;
}

__global__ void __launch_bounds__(kApWarps * 32, 4) cardinal_apply_pair_kernel(
    const float2 *__restrict__ E, int64_t Nq, int64_t N, const float2 *__restrict__ q, int T, int64_t kspan,
    float2 *__restrict__ out, float2 *__restrict__ part) {
    __shared__ __align__(16) float4 Es[3][kApBM][kAp2BK];
    __shared__ __align__(16) float4 Qs[3][kAp2BK][kApCols / 2];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t row0 = blockIdx.x * (int64_t)kApBM;
    const int col0 = blockIdx.y * kApCols;
    const int64_t kb = blockIdx.z * kspan, ke = std::min<int64_t>(N, kb + kspan);
    const int nchunks = (int)((ke - kb + kAp2BK - 1) / kAp2BK);

    auto load = [&](int st, int64_t k0) {
#pragma unroll
        for (int u = 0; u < kApBM * kAp2BK / (kApWarps * 32); ++u) {
            const int e = tid + u * kApWarps * 32;
            const int r = e / kAp2BK, kk = e % kAp2BK;
            const int64_t row = row0 + r, k = k0 + kk;
            const bool ok = row < Nq && k < ke;
            const float *src = ok ? reinterpret_cast<const float *>(E + row * N + k) : reinterpret_cast<const float *>(E);
            float *dst = reinterpret_cast<float *>(&Es[st][r][kk]);
            cp_async4(dst + 0, src, ok);
            cp_async4(dst + 1, src, ok);
            cp_async4(dst + 2, src + (ok ? 1 : 0), ok);
            cp_async4(dst + 3, src + (ok ? 1 : 0), ok);
        }
#pragma unroll
        for (int u = 0; u < kAp2BK * kApCols / (kApWarps * 32); ++u) {
            const int e = tid + u * kApWarps * 32;
            const int kk = e / kApCols, c = e % kApCols;
            const int64_t k = k0 + kk;
            const bool ok = k < ke && col0 + c < T;
            const float *src = ok ? reinterpret_cast<const float *>(q + k * T + col0 + c) : reinterpret_cast<const float *>(q);
            float *dst = reinterpret_cast<float *>(&Qs[st][kk][c >> 1]);
            cp_async4(dst + (c & 1), src, ok);
            cp_async4(dst + 2 + (c & 1), src + (ok ? 1 : 0), ok);
        }
    };

    const f2_t minus_one = 0xBF800000BF800000ull;  // (-1, -1): negation is exact
    f2_t sh[kApRows], sl[kApRows];
#pragma unroll
    for (int r = 0; r < kApRows; ++r) sh[r] = sl[r] = 0ull;
    // three-stage ring, one barrier per chunk: the barrier that publishes chunk ch also
    // guarantees that every warp has finished chunk ch - 1, whose stage the load of ch + 2 reuses
    if (nchunks > 0) load(0, kb);
    cp_async_commit();
    if (nchunks > 1) load(1, kb + kAp2BK);
    cp_async_commit();
    int st = 0;
    for (int ch = 0; ch < nchunks; ++ch) {
        cp_async_wait1();  // this thread's copies of chunk ch have landed
        __syncthreads();
        if (ch + 2 < nchunks) load(st == 0 ? 2 : st - 1, kb + (int64_t)(ch + 2) * kAp2BK);
        cp_async_commit();
#pragma unroll
        for (int kk = 0; kk < kAp2BK; ++kk) {
            const ulonglong2 qv = *reinterpret_cast<const ulonglong2 *>(&Qs[st][kk][lane]);
            const f2_t nqh = f2_mul(qv.x, minus_one), nql = f2_mul(qv.y, minus_one);
#pragma unroll
            for (int r = 0; r < kApRows; ++r) {
                const ulonglong2 ev = *reinterpret_cast<const ulonglong2 *>(&Es[st][warp * kApRows + r][kk]);
                pair_fma2(ev.x, ev.y, qv.x, nqh, nql, sh[r], sl[r]);
            }
        }
        st = st == 2 ? 0 : st + 1;
    }
#pragma unroll
    for (int r = 0; r < kApRows; ++r) {
        const int64_t row = row0 + warp * kApRows + r;
        if (row >= Nq) continue;
        float h[2], l[2];
        f2_unpack(sh[r], h[0], h[1]);
        f2_unpack(sl[r], l[0], l[1]);
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int c = col0 + 2 * lane + u;
            if (c >= T) continue;
            if (part) part[(int64_t)blockIdx.z * Nq * T + row * T + c] = make_float2(h[u], l[u]);
            else out[row * T + c] = pair_norm(h[u], l[u]);
        }
    }
}

// out[e] = sum over splits s = 0..S-1 (in that order) of part[s][e].
__global__ void cardinal_reduce_f64(const double *__restrict__ part, int64_t cnt, int S, double *__restrict__ out) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= cnt) return;
    double s = part[e];
    for (int k = 1; k < S; ++k) s += part[k * cnt + e];
    out[e] = s;
}
__global__ void cardinal_reduce_pair(const float2 *__restrict__ part, int64_t cnt, int S, float2 *__restrict__ out) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= cnt) return;
    float h = part[e].x, l = part[e].y;
    for (int k = 1; k < S; ++k) {
        const float2 p = part[k * cnt + e];
        const float s = h + p.x;  // two-sum of the high parts, low parts added
        const float bp = s - h;
        const float err = (h - (s - bp)) + (p.x - bp);
        l = l + (err + p.y);
        h = s;
    }
    out[e] = pair_norm(h, l);
}

struct ApPlan {
    int S = 1;
    int64_t kspan = 0;
    size_t ws = 0;
};

// Splits of K: the block count (row tiles x column tiles x S) as close below a whole number of
// SM-loads as possible, each split at least eight chunks long.
ApPlan ap_plan(int64_t Nq, int64_t N, int T) {
    ApPlan p;
    int sms = 152, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t tiles = ((Nq + kApBM - 1) / kApBM) * ((T + kApCols - 1) / kApCols);
    double best = -1.0;
    for (int S = 1; S <= kApMaxSplit; ++S) {
        const int64_t span = ((N + S - 1) / S + kApBK - 1) / kApBK * kApBK;
        if (S > 1 && span < 8 * kApBK) break;
        const int64_t splits = (N + span - 1) / span;
        if (splits != S) continue;
        const double waves = (double)(tiles * S) / sms;
        const double eff = waves / std::ceil(waves);
        if (eff > best + 1e-9) { best = eff; p.S = S; p.kspan = span; }
    }
    if (p.kspan == 0) p.kspan = N;
    p.ws = p.S > 1 ? (size_t)p.S * (size_t)Nq * (size_t)T * 8 : 0;
    return p;
}

}  // namespace

int global_cardinal_build(const double *LU, const int32_t *perm, const double *X, int64_t N, int kind,
                          double eps, const double *P, int64_t Nq, void *E, int e_dtype, cudaStream_t s) {
    if (Nq == 0) return RBFSL_OK;
    const int ncmax = (int)std::min<int64_t>(kCardChunk, Nq);
    double *B = nullptr, *C = nullptr;
    RBFSL_CUDA_TRY(cudaMalloc(&B, (size_t)N * ncmax * sizeof(double)));
    if (cudaMalloc(&C, (size_t)N * ncmax * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(B);
        set_error("global_cardinal: cudaMalloc failed");
        return RBFSL_ENOMEM;
    }
    int rc = RBFSL_OK;
    for (int64_t i0 = 0; i0 < Nq && rc == RBFSL_OK; i0 += ncmax) {
        const int nc = (int)std::min<int64_t>(ncmax, Nq - i0);
        const int64_t cnt = N * nc;
        cardinal_rhs<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(X, N, P, i0, nc, kind, eps * eps, B);
        rc = global_solve(LU, perm, N, B, nc, C, s);
        if (rc) break;
        dim3 grid((unsigned)((N + 31) / 32), (unsigned)((nc + 31) / 32)), block(32, 8);
        if (e_dtype == RBFSL_F64) cardinal_store<double><<<grid, block, 0, s>>>(C, N, nc, i0, (double *)E);
        else cardinal_store<float2><<<grid, block, 0, s>>>(C, N, nc, i0, (float2 *)E);
        rc = launch_status("global_cardinal");
    }
    const cudaError_t e = cudaStreamSynchronize(s);
    cudaFree(B);
    cudaFree(C);
    if (rc == RBFSL_OK && e != cudaSuccess) {
        set_error(std::string("global_cardinal: ") + cudaGetErrorString(e));
        rc = RBFSL_ECUDA;
    }
    return rc;
}

size_t cardinal_apply_workspace(int64_t Nq, int64_t N, int T) { return ap_plan(Nq, N, T).ws; }

int launch_cardinal_apply(const void *E, int64_t Nq, int64_t N, const void *q, int T, int dtype, void *out,
                          void *ws, size_t ws_bytes, cudaStream_t s) {
    if (Nq == 0) return RBFSL_OK;
    const ApPlan p = ap_plan(Nq, N, T);
    if (ws_bytes < p.ws || (p.ws && !ws)) {
        set_error("cardinal_apply: workspace too small");
        return RBFSL_EINVAL;
    }
    void *part = p.S > 1 ? ws : nullptr;
    dim3 grid((unsigned)((Nq + kApBM - 1) / kApBM), (unsigned)((T + kApCols - 1) / kApCols), (unsigned)p.S);
    const int64_t cnt = Nq * (int64_t)T;
    const unsigned rb = (unsigned)((cnt + 255) / 256);
    if (dtype == RBFSL_F64) {
        cardinal_apply_f64_kernel<<<grid, kApWarps * 32, 0, s>>>((const double *)E, Nq, N, (const double *)q, T,
                                                                p.kspan, (double *)out, (double *)part);
        if (part) cardinal_reduce_f64<<<rb, 256, 0, s>>>((const double *)part, cnt, p.S, (double *)out);
    } else {
        cardinal_apply_pair_kernel<<<grid, kApWarps * 32, 0, s>>>((const float2 *)E, Nq, N, (const float2 *)q, T,
                                                                 p.kspan, (float2 *)out, (float2 *)part);
        if (part) cardinal_reduce_pair<<<rb, 256, 0, s>>>((const float2 *)part, cnt, p.S, (float2 *)out);
    }
    return launch_status("cardinal_apply");
}

}  // namespace rbfsl

extern "C" int rbfsl_global_cardinal(const double *LU, const int32_t *perm, const double *x, int64_t N,
                                     int kernel, double eps, const double *p, int64_t Nq, void *E,
                                     int e_dtype, void *stream) {
    using namespace rbfsl;
    RBFSL_CHECK_ARG(N >= 1 && Nq >= 0, "global_cardinal: bad sizes");
    RBFSL_CHECK_ARG(kernel == RBFSL_GAUSS || kernel == RBFSL_IMQ, "global_cardinal: kernel must be GAUSS or IMQ");
    RBFSL_CHECK_ARG(eps > 0 && std::isfinite(eps), "global_cardinal: eps must be positive");
    RBFSL_CHECK_ARG(e_dtype == RBFSL_F64 || e_dtype == RBFSL_F32X2, "global_cardinal: bad e_dtype");
    RBFSL_CHECK_ARG(Nq == 0 || (LU && perm && x && p && E), "global_cardinal: null pointer");
    return global_cardinal_build(LU, perm, x, N, kernel, eps, p, Nq, E, e_dtype, (cudaStream_t)stream);
}

extern "C" size_t rbfsl_cardinal_apply_workspace_bytes(int64_t Nq, int64_t N, int T) {
    if (Nq < 0 || N < 1 || T < 1) return 0;
    return rbfsl::cardinal_apply_workspace(Nq, N, T);
}

extern "C" int rbfsl_cardinal_apply(const void *E, int64_t Nq, int64_t N, const void *q, int T, int dtype,
                                    void *q_out, void *workspace, size_t workspace_bytes, void *stream) {
    using namespace rbfsl;
    RBFSL_CHECK_ARG(Nq >= 0 && N >= 1 && T >= 1, "cardinal_apply: bad sizes");
    RBFSL_CHECK_ARG(dtype == RBFSL_F64 || dtype == RBFSL_F32X2, "cardinal_apply: bad dtype");
    RBFSL_CHECK_ARG(Nq == 0 || (E && q && q_out), "cardinal_apply: null pointer");
    RBFSL_CHECK_ARG(q_out != q, "cardinal_apply: q_out may not alias q");
    return launch_cardinal_apply(E, Nq, N, q, T, dtype, q_out, workspace, workspace_bytes, (cudaStream_t)stream);
}
