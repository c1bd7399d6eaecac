// Gather-dot W.q (Algorithm 1, "interpolate q^m to the departure points"): for each output
// row i, q_out[i, :] = sum_j w[i, j] q[idx[i, j], :]. Memory-bound: per row it streams n
// weights and n indices once and gathers n rows of q (T contiguous values each, so a row
// group of lanes reads whole rows coalesced).
//
// A row group of L lanes (L = the power of two >= min(T, 32)) serves one output row; the
// group's first n (w, idx) pairs are loaded cooperatively, one per lane, and broadcast with
// warp shuffles. FP32 uses the difference form q_c + sum_j w_j (q_j - q_c), c = idx[i, 0];
// FP32 pairs (the mixed-precision storage) use pair arithmetic.
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"

namespace rbfsl {

template <typename R, bool kDiff>
__global__ void __launch_bounds__(256) gather_dot_kernel(const int32_t *__restrict__ idx,
                                                         const R *__restrict__ W, int64_t Nq,
                                                         int n, const R *__restrict__ q, int T,
                                                         int L, R *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int rows_per_warp = kWarp / L;
    const int sub = lane % L, grp = lane / L;
    const int64_t i = gwarp * rows_per_warp + grp;
    const bool active = i < Nq;
    if (__all_sync(0xffffffffu, !active)) return;
    for (int t0 = 0; t0 < T; t0 += L) {
        const int t = t0 + sub;
        R acc = R(0), qc = R(0);
        if (kDiff && active && t < T) {
            const int c = idx[i * n];
            qc = c >= 0 ? q[(int64_t)c * T + t] : R(NAN);
        }
        for (int j0 = 0; j0 < n; j0 += L) {
            // cooperative load of up to L (w, idx) pairs of row i
            R wj = R(0);
            int sj = 0;
            if (active && j0 + sub < n) {
                wj = W[i * n + j0 + sub];
                sj = idx[i * n + j0 + sub];
            }
            const int cnt = min(L, n - j0);
            for (int jj = 0; jj < cnt; ++jj) {
                const R w = __shfl_sync(0xffffffffu, wj, grp * L + jj);
                const int s = __shfl_sync(0xffffffffu, sj, grp * L + jj);
                if (active && t < T) {
                    const R v = s >= 0 ? q[(int64_t)s * T + t] : R(NAN);  // failed stencil
                    acc = fma(w, kDiff ? (v - qc) : v, acc);
                }
            }
        }
        if (active && t < T) out[i * T + t] = kDiff ? qc + acc : acc;
    }
}

// Vectorised variant for T a multiple of the vector width V (4 floats or 2 doubles = 16 B):
// a row group of G = T / V lanes serves one row (32 / G rows per warp), every lane owning V
// consecutive tracers, so each gathered q row is read as G 16-byte pieces. Members are taken in
// batches of kGatherBatch: the batch's indices and weights are loaded first (the G lanes of a
// row group read the same words), then all its q pieces are requested before the first is
// used, so a lane keeps kGatherBatch gathers in flight instead of one; with 16-byte aligned rows
// (n a multiple of 4) a batch's indices and weights come in 16-byte loads. A negative member
// (failed stencil) is flagged once per row and gives a NaN row. Same summation order as the
// scalar kernel (j ascending, one fma per term). Four blocks of 256 threads per SM (64
// registers): 32 resident warps to hide the gather latency.
constexpr int kGatherBatch = 8;

template <typename R, typename RV, int V, bool kDiff, bool kVecLoads>
__global__ void __launch_bounds__(256, 4) gather_dot_vec_kernel(const int32_t *__restrict__ idx,
                                                             const R *__restrict__ W, int64_t Nq,
                                                             int n, const R *__restrict__ q, int T,
                                                             int G, R *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int rows_per_warp = kWarp / G;
    const int sub = lane % G, grp = lane / G;
    const int64_t i = gwarp * rows_per_warp + grp;
    if (grp >= rows_per_warp || i >= Nq) return;
    const RV *qv = reinterpret_cast<const RV *>(q);
    const int Tv = T / V;
    const int32_t *Ir = idx + i * n;
    const R *Wr = W + i * n;
    bool failed = false;  // a negative member (failed stencil): the row is NaN
    R acc[V], qc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) { acc[v] = R(0); qc[v] = R(0); }
    if (kDiff) {
        const int c = Ir[0];
        failed = c < 0;
        const RV x = qv[(int64_t)(c < 0 ? 0 : c) * Tv + sub];
        const R *xr = reinterpret_cast<const R *>(&x);
#pragma unroll
        for (int v = 0; v < V; ++v) qc[v] = xr[v];
    }
    auto term = [&](R w, const RV &x) {
        const R *xr = reinterpret_cast<const R *>(&x);
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = fma(w, kDiff ? (xr[v] - qc[v]) : xr[v], acc[v]);
    };
    int j0 = 0;
    for (; j0 + kGatherBatch <= n; j0 += kGatherBatch) {
        int sb[kGatherBatch];
        R wb[kGatherBatch];
        RV xb[kGatherBatch];
        if (kVecLoads) {  // 16-byte loads of the batch's indices and weights (rows 16-byte aligned)
#pragma unroll
            for (int b = 0; b < kGatherBatch; b += 4) {
                const int4 iv = *reinterpret_cast<const int4 *>(Ir + j0 + b);
                sb[b] = iv.x; sb[b + 1] = iv.y; sb[b + 2] = iv.z; sb[b + 3] = iv.w;
            }
            constexpr int WV = 16 / (int)sizeof(R);
#pragma unroll
            for (int b = 0; b < kGatherBatch; b += WV) {
                const RV wv = *reinterpret_cast<const RV *>(Wr + j0 + b);
                const R *wr = reinterpret_cast<const R *>(&wv);
#pragma unroll
                for (int u = 0; u < WV; ++u) wb[b + u] = wr[u];
            }
        } else {
#pragma unroll
            for (int b = 0; b < kGatherBatch; ++b) { sb[b] = Ir[j0 + b]; wb[b] = Wr[j0 + b]; }
        }
#pragma unroll
        for (int b = 0; b < kGatherBatch; ++b) {
            failed |= sb[b] < 0;
            xb[b] = qv[(int64_t)(sb[b] < 0 ? 0 : sb[b]) * Tv + sub];
        }
#pragma unroll
        for (int b = 0; b < kGatherBatch; ++b) term(wb[b], xb[b]);
    }
    for (; j0 < n; ++j0) {
        const int sidx = Ir[j0];
        failed |= sidx < 0;
        term(Wr[j0], qv[(int64_t)(sidx < 0 ? 0 : sidx) * Tv + sub]);
    }
    RV o;
    R *orr = reinterpret_cast<R *>(&o);
#pragma unroll
    for (int v = 0; v < V; ++v) orr[v] = failed ? R(NAN) : (kDiff ? qc[v] + acc[v] : acc[v]);
    reinterpret_cast<RV *>(out)[i * Tv + sub] = o;
}

// FP32 pairs (mixed precision): weights and field stored as (hi, lo) pairs and the sum
// formed in pair arithmetic (pair_fma), FP32 operations only. Each lane owns V consecutive
// tracers (V = 2: one 16-byte load per gathered row piece; V = 1 for odd T); a row group of G
// lanes covers G * V tracers per pass. Members in batches of kGatherBatch as in
// gather_dot_vec_kernel (16-byte index and weight loads, one failure flag per row). Same element
// order (j ascending) as the batched path. Four blocks of 256 threads per SM (64 registers, no
// spills): 32 resident warps to hide the gather latency (measured against three: 1.48 against
// 1.22 TB/s at N = 655,362, T = 16).
template <int V, bool kVecLoads>
__global__ void __launch_bounds__(256, 4) gather_dot_pair_kernel(const int32_t *__restrict__ idx,
                                                              const float2 *__restrict__ W, int64_t Nq,
                                                              int n, const float2 *__restrict__ q,
                                                              int T, int G, float2 *__restrict__ out) {
    using Vec = typename std::conditional<V == 2, float4, float2>::type;
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int rows_per_warp = kWarp / G;
    const int sub = lane % G, grp = lane / G;
    const int64_t i = gwarp * rows_per_warp + grp;
    if (grp >= rows_per_warp || i >= Nq) return;
    const int32_t *Ir = idx + i * n;
    const float2 *Wr = W + i * n;
    for (int t0 = 0; t0 < T; t0 += G * V) {
        const int t = t0 + sub * V;
        if (t >= T) continue;  // V = 2 only for even T, so t + 1 < T too
        bool failed = false;   // a negative member (failed stencil): the row is NaN
        float sh[V], sl[V];
#pragma unroll
        for (int v = 0; v < V; ++v) { sh[v] = 0.f; sl[v] = 0.f; }
        auto term = [&](float2 w, const Vec &x) {
            const float2 *xp = reinterpret_cast<const float2 *>(&x);
#pragma unroll
            for (int v = 0; v < V; ++v) pair_fma(w, xp[v], sh[v], sl[v]);
        };
        int j0 = 0;
        for (; j0 + kGatherBatch <= n; j0 += kGatherBatch) {
            int sb[kGatherBatch];
            float2 wb[kGatherBatch];
            Vec xb[kGatherBatch];
            if (kVecLoads) {  // 16-byte loads of the batch's indices and weight pairs
#pragma unroll
                for (int b = 0; b < kGatherBatch; b += 4) {
                    const int4 iv = *reinterpret_cast<const int4 *>(Ir + j0 + b);
                    sb[b] = iv.x; sb[b + 1] = iv.y; sb[b + 2] = iv.z; sb[b + 3] = iv.w;
                }
#pragma unroll
                for (int b = 0; b < kGatherBatch; b += 2) {
                    const float4 wv = *reinterpret_cast<const float4 *>(Wr + j0 + b);
                    wb[b] = make_float2(wv.x, wv.y);
                    wb[b + 1] = make_float2(wv.z, wv.w);
                }
            } else {
#pragma unroll
                for (int b = 0; b < kGatherBatch; ++b) { sb[b] = Ir[j0 + b]; wb[b] = Wr[j0 + b]; }
            }
#pragma unroll
            for (int b = 0; b < kGatherBatch; ++b) {
                failed |= sb[b] < 0;
                xb[b] = *reinterpret_cast<const Vec *>(q + (int64_t)(sb[b] < 0 ? 0 : sb[b]) * T + t);
            }
#pragma unroll
            for (int b = 0; b < kGatherBatch; ++b) term(wb[b], xb[b]);
        }
        for (; j0 < n; ++j0) {
            const int sidx = Ir[j0];
            failed |= sidx < 0;
            term(Wr[j0], *reinterpret_cast<const Vec *>(q + (int64_t)(sidx < 0 ? 0 : sidx) * T + t));
        }
        Vec o;
        float2 *op = reinterpret_cast<float2 *>(&o);
#pragma unroll
        for (int v = 0; v < V; ++v) op[v] = failed ? make_float2(NAN, NAN) : pair_norm(sh[v], sl[v]);
        *reinterpret_cast<Vec *>(out + i * T + t) = o;
    }
}

int launch_gather(const int32_t *idx, const void *w, int64_t Nq, int n, const void *q, int T,
                  int dtype, void *q_out, cudaStream_t s) {
    if (Nq == 0) return RBFSL_OK;
    if (dtype == RBFSL_F32X2) {
        const bool vec2 = T % 2 == 0 && ((uintptr_t)q % 16 == 0) && ((uintptr_t)q_out % 16 == 0);
        const int per_lane = vec2 ? 2 : 1;
        const int need = (T + per_lane - 1) / per_lane;
        int G = 1;
        while (G < need && G < 32) G <<= 1;
        const int rows_per_warp = kWarp / G;
        const int threads = 256;
        const int64_t warps = (Nq + rows_per_warp - 1) / rows_per_warp;
        const unsigned blocks = (unsigned)((warps * kWarp + threads - 1) / threads);
        const bool vl = n % 4 == 0 && (uintptr_t)idx % 16 == 0 && (uintptr_t)w % 16 == 0;
        auto go = [&](auto k) {
            k<<<blocks, threads, 0, s>>>(idx, (const float2 *)w, Nq, n, (const float2 *)q, T, G, (float2 *)q_out);
        };
        if (vec2 && vl) go(gather_dot_pair_kernel<2, true>);
        else if (vec2) go(gather_dot_pair_kernel<2, false>);
        else if (vl) go(gather_dot_pair_kernel<1, true>);
        else go(gather_dot_pair_kernel<1, false>);
        return launch_status("gather_dot_pair");
    }
    const int V = dtype == RBFSL_F64 ? 2 : 4;
    const bool aligned = ((uintptr_t)q % 16 == 0) && ((uintptr_t)q_out % 16 == 0);
    if (T % V == 0 && T / V <= 32 && aligned) {
        int G = 1;
        while (G < T / V) G <<= 1;  // a power of two >= T / V lanes per row
        if (G == T / V) {
            const int rows_per_warp = kWarp / G;
            const int threads = 256;
            const int64_t warps = (Nq + rows_per_warp - 1) / rows_per_warp;
            const unsigned blocks = (unsigned)((warps * kWarp + threads - 1) / threads);
            const bool vl = n % 4 == 0 && (uintptr_t)idx % 16 == 0 && (uintptr_t)w % 16 == 0;
            if (dtype == RBFSL_F64 && vl)
                gather_dot_vec_kernel<double, double2, 2, false, true><<<blocks, threads, 0, s>>>(
                    idx, (const double *)w, Nq, n, (const double *)q, T, G, (double *)q_out);
            else if (dtype == RBFSL_F64)
                gather_dot_vec_kernel<double, double2, 2, false, false><<<blocks, threads, 0, s>>>(
                    idx, (const double *)w, Nq, n, (const double *)q, T, G, (double *)q_out);
            else if (vl)
                gather_dot_vec_kernel<float, float4, 4, true, true><<<blocks, threads, 0, s>>>(
                    idx, (const float *)w, Nq, n, (const float *)q, T, G, (float *)q_out);
            else
                gather_dot_vec_kernel<float, float4, 4, true, false><<<blocks, threads, 0, s>>>(
                    idx, (const float *)w, Nq, n, (const float *)q, T, G, (float *)q_out);
            return launch_status("gather_dot_vec");
        }
    }
    int L = 1;
    while (L < T && L < 32) L <<= 1;
    const int rows_per_warp = kWarp / L;
    const int threads = 256;
    const int64_t warps = (Nq + rows_per_warp - 1) / rows_per_warp;
    const unsigned blocks = (unsigned)((warps * kWarp + threads - 1) / threads);
    if (dtype == RBFSL_F64)
        gather_dot_kernel<double, false><<<blocks, threads, 0, s>>>(
            idx, (const double *)w, Nq, n, (const double *)q, T, L, (double *)q_out);
    else
        gather_dot_kernel<float, true><<<blocks, threads, 0, s>>>(
            idx, (const float *)w, Nq, n, (const float *)q, T, L, (float *)q_out);
    return launch_status("gather_dot");
}

}  // namespace rbfsl

extern "C" int rbfsl_gather_dot(const int32_t *idx, const void *w, int64_t Nq, int n,
                                const void *q, int T, int dtype, void *q_out, void *stream) {
    using namespace rbfsl;
    RBFSL_CHECK_ARG(Nq >= 0 && n >= 1 && T >= 1, "gather_dot: bad sizes");
    RBFSL_CHECK_ARG(dtype == RBFSL_F64 || dtype == RBFSL_F32 || dtype == RBFSL_F32X2, "gather_dot: bad dtype");
    RBFSL_CHECK_ARG(Nq == 0 || (idx && w && q && q_out), "gather_dot: null pointer");
    RBFSL_CHECK_ARG(q != q_out, "gather_dot: q_out aliases q");
    return launch_gather(idx, w, Nq, n, q, T, dtype, q_out, (cudaStream_t)stream);
}
