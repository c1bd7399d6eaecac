// Global RBF evaluation on the tensor cores (tcgen05, split TF32, FP32 accumulation):
//   out[i][t] = sum_j phi(|p_i - x_j|) c[j][t]          (Eq. srbfinterp at the departure points)
// Each block owns 128 points x 32 tracers; the accumulator (128 x 32 FP32) lives in tensor
// memory. Per chunk of 32 nodes, the 128 threads compute the kernel values of their point row
// (FP32), split each into a TF32 high part and the FP32 remainder, and store both in shared
// memory in the no-swizzle K-major core-matrix layout; the coefficient chunk (pre-split and
// transposed by tc_split_coefficients) is staged the same way. One thread then issues the MMAs
// hi*hi + hi*lo + lo*hi (M = 128, N = 32, K = 8 each) and commits them to an mbarrier; two
// shared-memory stages let the next chunk's kernel values be computed while the MMAs run.
// Every wait on an mbarrier is bounded: on timeout the block records an error, releases its
// tensor memory and returns.
#include <cstdint>

#include "common.cuh"
#include "kernels.cuh"

namespace rbfsl {

constexpr int kTcM = 128, kTcN = 32, kTcK = 32;  // block tile: points x tracers x node chunk
constexpr int kTcStageFloats = 2 * kTcM * kTcK + 2 * kTcN * kTcK;  // Ahi, Alo, Bhi, Blo
constexpr long long kTcWaitLimit = 1LL << 22;
constexpr uint32_t kTcLbo = 128, kTcSbo = (kTcK / 4) * 128;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Offset (in floats) of element (row, k) of a K-major operand tile with 32 K-elements per row,
// no swizzle: core matrices of 8 rows x 4 floats (16 B per row, 128 B per core matrix), core
// (row/8, k/4) at byte ((row/8) * 8 + k/4) * 128.
__device__ __forceinline__ int core_off(int row, int k) {
    return (((row >> 3) * (kTcK / 4) + (k >> 2)) << 5) + ((row & 7) << 2) + (k & 3);
}

// Shared-memory matrix descriptor (tcgen05): start >> 4 (bits 0-13), leading-dimension byte
// offset >> 4 (16-29, the step between core matrices along K), stride-dimension byte offset
// >> 4 (32-45, the step between 8-row groups), version 1 (46-47), no swizzle (61-63 = 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor, kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32 (7-9, 10-12 = 2),
// both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t tc_idesc() {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
        :
        : "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (long long it = 0; it < kTcWaitLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// c (N x T, FP64 or FP32, row-major) -> hi, lo ([Tpad][Npad] transposed, zero padded):
// hi = TF32 rounding of c, lo = c - hi in FP32.
template <typename R>
__global__ void tc_split_coefficients(const R *__restrict__ c, int64_t N, int T, int64_t Npad, int Tpad,
                                      float *__restrict__ hi, float *__restrict__ lo) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= Npad * Tpad) return;
    const int64_t t = e / Npad, k = e - t * Npad;
    const float v = (k < N && t < T) ? (float)c[k * T + t] : 0.f;
    const float h = tf32_rna(v);
    hi[e] = h;
    lo[e] = v - h;
}

__global__ void __launch_bounds__(128) global_eval_tc_kernel(const double *__restrict__ P, int64_t Nq,
                                                             const double *__restrict__ X, int64_t N,
                                                             int kind, float eps2,
                                                             const float *__restrict__ Chi,
                                                             const float *__restrict__ Clo, int64_t Npad,
                                                             int T, float *__restrict__ out,
                                                             int32_t *__restrict__ err, uint32_t lbo,
                                                             uint32_t sbo) {
    extern __shared__ __align__(1024) float tsm[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t p0 = (int64_t)blockIdx.x * kTcM;
    const int t0 = blockIdx.y * kTcN;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(32)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;

    const int64_t pi = p0 + tid < Nq ? p0 + tid : (Nq > 0 ? Nq - 1 : 0);
    const float px = (float)P[3 * pi], py = (float)P[3 * pi + 1], pz = (float)P[3 * pi + 2];
    const int64_t nchunks = Npad / kTcK;
    const uint32_t idesc = tc_idesc();
    bool ok = true;
    for (int64_t c = 0; c < nchunks && ok; ++c) {
        const int s = (int)(c & 1);
        float *Ahi = tsm + s * kTcStageFloats, *Alo = Ahi + kTcM * kTcK;
        float *Bhi = Alo + kTcM * kTcK, *Blo = Bhi + kTcN * kTcK;
        if (c >= 2) {  // the MMAs that read this stage two chunks ago have completed
            ok = mbar_wait(smem_u32(&mbar[s]), (uint32_t)(((c - 2) >> 1) & 1));
            ok = __syncthreads_and(ok);  // one decision for the whole block
            if (!ok) break;
        }
        // kernel values of this thread's point against 32 nodes
#pragma unroll 4
        for (int k = 0; k < kTcK; ++k) {
            const int64_t j = c * kTcK + k;
            float v = 0.f;
            if (j < N) {
                const float dx = px - (float)X[3 * j], dy = py - (float)X[3 * j + 1], dz = pz - (float)X[3 * j + 2];
                const float d2 = dx * dx + dy * dy + dz * dz;
                v = kind == RBFSL_GAUSS ? __expf(-eps2 * d2) : rsqrtf(1.0f + eps2 * d2);
            }
            const float h = tf32_rna(v);
            Ahi[core_off(tid, k)] = h;
            Alo[core_off(tid, k)] = v - h;
        }
        // coefficient chunk: tracers t0..t0+31 (rows of B) x nodes (K)
        for (int e = tid; e < kTcN * kTcK; e += 128) {
            const int n = e / kTcK, k = e % kTcK;
            const int64_t g = (int64_t)(t0 + n) * Npad + c * kTcK + k;
            Bhi[core_off(n, k)] = Chi[g];
            Blo[core_off(n, k)] = Clo[g];
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a_hi = smem_u32(Ahi), a_lo = smem_u32(Alo), b_hi = smem_u32(Bhi), b_lo = smem_u32(Blo);
#pragma unroll
            for (int ks = 0; ks < kTcK / 8; ++ks) {
                const uint32_t koff = ks * 2 * 128;  // two core matrices (8 TF32) per k-step
                mma_tf32(tmem, smem_desc(a_hi + koff, lbo, sbo), smem_desc(b_hi + koff, lbo, sbo), idesc,
                         (c > 0 || ks > 0) ? 1u : 0u);
                mma_tf32(tmem, smem_desc(a_hi + koff, lbo, sbo), smem_desc(b_lo + koff, lbo, sbo), idesc, 1u);
                mma_tf32(tmem, smem_desc(a_lo + koff, lbo, sbo), smem_desc(b_hi + koff, lbo, sbo), idesc, 1u);
            }
            mma_commit(smem_u32(&mbar[s]));
        }
        __syncthreads();
    }
    // drain: the last commit of each stage (also after a timeout, so that no MMA is still
    // writing tensor memory when it is released; this wait is bounded too)
    bool drained = true;
    for (int64_t c = (nchunks >= 2 ? nchunks - 2 : 0); c < nchunks; ++c)
        drained = mbar_wait(smem_u32(&mbar[c & 1]), (uint32_t)((c >> 1) & 1)) && drained;
    ok = __syncthreads_and(ok && drained);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        uint32_t r[32];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
              "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
              "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
              "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int64_t row = p0 + warp * 32 + lane;
        if (row < Nq) {
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (t0 + j < T) out[row * T + t0 + j] = __uint_as_float(r[j]);
        }
    } else if (tid == 0) {
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32) : "memory");
}

size_t global_eval_tc_workspace(int64_t N, int T) {
    const int64_t Npad = (N + kTcK - 1) / kTcK * kTcK;
    const int64_t Tpad = (T + kTcN - 1) / kTcN * kTcN;
    return (size_t)(2 * Npad * Tpad) * sizeof(float) + 256;
}

int launch_global_eval_tc(const double *P, int64_t Nq, const double *X, int64_t N, int kind, double eps,
                          const void *C, int c_dtype, int T, float *out, void *workspace, cudaStream_t s) {
    if (Nq == 0) return RBFSL_OK;
    const int64_t Npad = (N + kTcK - 1) / kTcK * kTcK;
    const int Tpad = (T + kTcN - 1) / kTcN * kTcN;
    float *hi = reinterpret_cast<float *>(workspace);
    float *lo = hi + Npad * Tpad;
    int32_t *err = reinterpret_cast<int32_t *>(lo + Npad * Tpad);
    const int64_t tot = Npad * Tpad;
    if (c_dtype == RBFSL_F64)
        tc_split_coefficients<double><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>((const double *)C, N, T, Npad, Tpad, hi, lo);
    else
        tc_split_coefficients<float><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>((const float *)C, N, T, Npad, Tpad, hi, lo);
    RBFSL_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int32_t), s));
    const int smem = 2 * kTcStageFloats * (int)sizeof(float);
    RBFSL_CUDA_TRY(cudaFuncSetAttribute(global_eval_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    dim3 grid((unsigned)((Nq + kTcM - 1) / kTcM), (unsigned)(Tpad / kTcN));
    // LBO: byte step between core matrices along K; SBO: byte step between 8-row groups
    global_eval_tc_kernel<<<grid, 128, smem, s>>>(P, Nq, X, N, kind, (float)(eps * eps), hi, lo, Npad, T, out, err,
                                                  kTcLbo, kTcSbo);
    return launch_status("global_eval_tc");
}

}  // namespace rbfsl

extern "C" size_t rbfsl_global_eval_tc_workspace_bytes(int64_t N, int T) {
    return rbfsl::global_eval_tc_workspace(N, T);
}

extern "C" int rbfsl_global_eval_tc(const double *p, int64_t Nq, const double *x, int64_t N, int kernel,
                                    double eps, const void *c, int c_dtype, int T, float *out,
                                    void *workspace, size_t workspace_bytes, void *stream) {
    using namespace rbfsl;
    RBFSL_CHECK_ARG(Nq >= 0 && N >= 1 && T >= 1, "global_eval_tc: bad sizes");
    RBFSL_CHECK_ARG(Nq == 0 || (p && x && c && out && workspace), "global_eval_tc: null pointer");
    RBFSL_CHECK_ARG((kernel == RBFSL_GAUSS || kernel == RBFSL_IMQ) && eps > 0, "global_eval_tc: bad kernel");
    RBFSL_CHECK_ARG(c_dtype == RBFSL_F64 || c_dtype == RBFSL_F32, "global_eval_tc: bad dtype");
    RBFSL_CHECK_ARG(workspace_bytes >= global_eval_tc_workspace(N, T), "global_eval_tc: workspace too small");
    RBFSL_CHECK_ARG(((uintptr_t)workspace & 15) == 0, "global_eval_tc: workspace must be 16-byte aligned");
    return launch_global_eval_tc(p, Nq, x, N, kernel, eps, c, c_dtype, T, out, workspace, (cudaStream_t)stream);
}
