// Global RBF evaluation on the tensor cores (tcgen05, split TF32, FP32 accumulation):
//   out[i][t] = sum_j phi(|p_i - x_j|) c[j][t]          (Eq. srbfinterp at the departure points)
//
// Formulation: the transposed product D^T = C^T Phi^T with both factors split into a TF32 high
// part and the FP32 remainder. The A operand is [c_hi ; c_lo] (M = 128: 64 tracers twice), the
// B operand is phi_hi or phi_lo of 256 points (N = 256), K = 8 nodes per MMA; two MMAs per k-step
// accumulate [c_hi ; c_lo] (phi_hi + phi_lo) into 128 lanes x 256 columns of tensor memory, and
// the result is the sum of the two lane halves (c_hi phi + c_lo phi: all four hi/lo products).
// Large MMAs (N = 256) keep the single issuing thread ahead of the tensor pipe.
//
// Work: items (256-point tile, node range, 64-tracer tile); the node range is split ksplit ways
// so that equal numbers of items go to persistent CTAs, one per SM. Each item writes its two
// lane halves as partial tiles and a second kernel adds the 2 ksplit slices in a fixed order
// (deterministic). Within an item the CTA walks its range in chunks of 32 nodes; two
// accumulators, so that an item's epilogue overlaps the next item's MMAs.
//
// Warp roles (576 threads); two phi stages, up to 6 coefficient stages:
//   warps 0-15  producers: per chunk, the kernel values of 256 points x 32 nodes in FP32 (each
//               thread one point and 16 nodes, read from the chunk's coefficient block once its
//               copy has landed), split into hi and lo and stored in the no-swizzle K-major
//               core-matrix layout; after an item, the epilogue (tensor memory -> registers ->
//               partial tiles, 128-byte rows per warp).
//   warp 16     MMA issuer (one lane): allocates tensor memory; per chunk waits for the
//               producers (whose arrival implies the coefficient copy) and issues the MMAs, then
//               commits them to the stages' "empty" barriers and, after an item's last chunk,
//               to the accumulator's barrier.
//   warp 17     copy issuer (one lane): streams the coefficient blocks (laid out by tc_prepare)
//               with one bulk TMA copy per chunk, up to the ring's depth ahead.
// Every wait is bounded: on timeout the CTA records RBFSL_ETIMEDOUT, stops, waits (bounded) for
// the copies and MMAs it started, releases its tensor memory and returns.
#include <cstdint>

#include "common.cuh"
#include "kernels.cuh"

namespace rbfsl {

constexpr int kTcPts = 256, kTcK = 32;  // points per tile (MMA N), nodes per chunk
constexpr int kTcTn = 64;               // tracers per tile: the A operand is [c_hi ; c_lo], M = 128
constexpr int kTcProducerWarps = 16, kTcThreads = 32 * (kTcProducerWarps + 2);
constexpr int kTcMaxCStages = 6;
constexpr long long kTcWaitLimit = 1LL << 22;
constexpr uint32_t kTcLbo = 128;               // byte step between core matrices along K
constexpr uint32_t kTcSbo = (kTcK / 4) * 128;  // byte step between 8-row groups

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// 2^x by the hardware approximation (PTX ex2.approx).
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Offset (in floats) of element (row, k) of a K-major operand tile with kTcK elements per row,
// no swizzle: core matrices of 8 rows x 4 floats (16 B per row, 128 B per core matrix), core
// (row/8, k/4) at byte ((row/8) * (kTcK/4) + k/4) * 128.
__host__ __device__ __forceinline__ int core_off(int row, int k) {
    return (((row >> 3) * (kTcK / 4) + (k >> 2)) << 5) + ((row & 7) << 2) + (k & 3);
}

// Shared-memory matrix descriptor (tcgen05): start >> 4 (bits 0-13), leading-dimension byte
// offset >> 4 (16-29), stride-dimension byte offset >> 4 (32-45), version 1 (46-47), no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((kTcLbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((kTcSbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor, kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32 (7-9, 10-12 = 2),
// both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t tc_idesc(int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
        :
        : "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// Wait for the phase of the given parity to complete; false after kTcWaitLimit polls.
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

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

// One bulk (non-tensor) TMA copy, global -> this CTA's shared memory, completing on mbar.
__device__ __forceinline__ void tma_bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(mbar)
        : "memory");
}

// 32 lanes x 16 consecutive 32-bit columns of tensor memory -> 16 registers per thread.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}

struct TcArgs {
    const double *P;   // Nq x 3 evaluation points
    int64_t Nq;
    const float *B;    // coefficient blocks [ttile][chunk] (tc_cblock_floats floats each)
    int64_t nchunks;
    int ksplit, ptiles, ttiles;
    int64_t nitems;    // ptiles * ksplit * ttiles work items (point tile, node range, tracer tile)
    int T, Tpad;       // tracers, padded to whole tiles of kTcTn
    int sc;            // coefficient stages in shared memory (2..kTcMaxCStages)
    int kind;
    float karg;        // Gaussian: -eps^2 log2(e) (base-2 exponent); IMQ: eps^2
    float *part;       // partial tiles [2 ksplit][Nq][Tpad]: slice 2 kz + h holds c_h x phi
    int32_t *status;   // RBFSL_ETIMEDOUT after a timed-out wait
};

// Floats of one coefficient block: the A operand [c_hi ; c_lo] (128 rows = 2 x kTcTn tracers,
// kTcK nodes, core-matrix order), then the chunk's kTcK nodes as float4 (x, y, z, 0).
__host__ __device__ __forceinline__ constexpr int tc_cblock_floats() { return 2 * kTcTn * kTcK + 4 * kTcK; }

// The CTA's work in order: items blockIdx.x, blockIdx.x + gridDim.x, ...; within an item its
// node chunks c..c1-1. Item it: node range kz = it % ksplit, point tile (it / ksplit) % ptiles,
// tracer tile it / (ksplit * ptiles).
struct TcCursor {
    int64_t it;
    int c, c1;
    int j;  // item ordinal within this CTA
    int kz, pt, tt;
    __device__ __forceinline__ void load(const TcArgs &a) {
        kz = (int)(it % a.ksplit);
        const int64_t rest = it / a.ksplit;
        pt = (int)(rest % a.ptiles);
        tt = (int)(rest / a.ptiles);
        c = (int)(a.nchunks * kz / a.ksplit);
        c1 = (int)(a.nchunks * (kz + 1) / a.ksplit);
    }
    __device__ __forceinline__ void start(const TcArgs &a) {
        it = blockIdx.x;
        j = 0;
        if (it < a.nitems) load(a);
    }
    __device__ __forceinline__ bool valid(const TcArgs &a) const { return it < a.nitems; }
    __device__ __forceinline__ void next(const TcArgs &a) {
        if (++c < c1) return;
        it += gridDim.x;
        ++j;
        if (it < a.nitems) load(a);
    }
};

__global__ void __launch_bounds__(kTcThreads, 1) global_eval_tc_kernel(TcArgs a) {
    extern __shared__ __align__(128) float tsm[];
    __shared__ __align__(8) uint64_t phi_full[2], phi_empty[2];                 // B operand stages
    __shared__ __align__(8) uint64_t c_full[kTcMaxCStages], c_empty[kTcMaxCStages];  // coefficient stages
    __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2];
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int SC = a.sc;
    constexpr int phi_floats = kTcPts * kTcK;           // hi or lo half of a phi stage
    constexpr int cblk = tc_cblock_floats();
    float *phi_base = tsm;                              // 2 stages x (hi, lo)
    float *c_base = tsm + 4 * phi_floats;               // SC stages x cblk
    constexpr uint32_t acc_cols = kTcPts;               // one accumulator: 128 lanes x 256 columns
    constexpr uint32_t ncols = 2 * acc_cols;

    if (warp == kTcProducerWarps) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(smem_u32(&phi_full[s]), kTcProducerWarps);
            mbar_init(smem_u32(&phi_empty[s]), 1);
            mbar_init(smem_u32(&acc_full[s]), 1);
            mbar_init(smem_u32(&acc_empty[s]), kTcProducerWarps);
        }
        for (int s = 0; s < kTcMaxCStages; ++s) {
            mbar_init(smem_u32(&c_full[s]), 1);
            mbar_init(smem_u32(&c_empty[s]), 1);
        }
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;

    if (warp < kTcProducerWarps) {
        // ---------------------------------------------------------------- producers
        const int row = tid & (kTcPts - 1), kh = (tid >> 8) * (kTcK / 2);  // one point, 16 nodes
        const int q = warp & 3, cg = warp >> 2;  // epilogue: tensor-memory lane quarter, column group
        int pend_j = -1, pend_pt = 0, pend_kz = 0, pend_tt = 0;  // item whose epilogue is due
        auto epilogue = [&](int jj, int pt, int kz, int tt) {
            const int acc = jj & 1;
            if (!mbar_wait(smem_u32(&acc_full[acc]), (uint32_t)((jj >> 1) & 1))) {
                s_abort = 1;
                atomicExch(a.status, RBFSL_ETIMEDOUT);
                return;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // lanes 0-63: c_hi x phi for tracers 0-63, lanes 64-127: c_lo x phi; columns: points
            const int h = q >> 1, t = tt * kTcTn + (q & 1) * 32 + lane;
            float *dst = a.part + (int64_t)(2 * kz + h) * a.Nq * a.Tpad + t;
            const int64_t p0 = (int64_t)pt * kTcPts;
            const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + acc * acc_cols;
            for (int cc = cg * 64; cc < cg * 64 + 64; cc += 16) {
                uint32_t v[16];
                tmem_ld16(tbase + (uint32_t)cc, v);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int64_t pidx = p0 + cc + u;
                    if (pidx < a.Nq) dst[pidx * a.Tpad] = __uint_as_float(v[u]);  // 32 lanes: 128 B
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&acc_empty[acc]));
        };
        TcCursor cur;
        cur.start(a);
        float px = 0.f, py = 0.f, pz = 0.f;
        int cur_j = -1, sc = 0;
        uint32_t pc = 0;  // chunk g's coefficient stage g % SC and its phase parity (g / SC) & 1
        for (int g = 0; cur.valid(a); ++g, cur.next(a)) {
            const int sp = g & 1;
            const bool first = cur.j != cur_j;
            if (first) {  // a new item: this thread's point
                cur_j = cur.j;
                const int64_t p = (int64_t)cur.pt * kTcPts + row;
                const int64_t pi = p < a.Nq ? p : a.Nq - 1;
                px = (float)a.P[3 * pi]; py = (float)a.P[3 * pi + 1]; pz = (float)a.P[3 * pi + 2];
            }
            bool ok = true;
            if (g >= 2) ok = mbar_wait(smem_u32(&phi_empty[sp]), (uint32_t)(((g - 2) >> 1) & 1));
            ok = ok && mbar_wait(smem_u32(&c_full[sc]), pc);  // the chunk's nodes are in
            if (!ok) {
                s_abort = 1;
                atomicExch(a.status, RBFSL_ETIMEDOUT);
                break;
            }
            float *Bhi = phi_base + sp * 2 * phi_floats, *Blo = Bhi + phi_floats;
            const float4 *xc = reinterpret_cast<const float4 *>(c_base + sc * cblk + 2 * kTcTn * kTcK) + kh;
#pragma unroll
            for (int gk = 0; gk < kTcK / 2; gk += 4) {
                float v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float4 x = xc[gk + u];
                    const float dx = px - x.x, dy = py - x.y, dz = pz - x.z;
                    const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                    v[u] = a.kind == RBFSL_GAUSS ? ex2_approx(a.karg * d2) : rsqrtf(fmaf(a.karg, d2, 1.0f));
                }
                float4 hv, lv;
                hv.x = tf32_rna(v[0]); hv.y = tf32_rna(v[1]); hv.z = tf32_rna(v[2]); hv.w = tf32_rna(v[3]);
                lv.x = v[0] - hv.x; lv.y = v[1] - hv.y; lv.z = v[2] - hv.z; lv.w = v[3] - hv.w;
                const int off = core_off(row, kh + gk);
                *reinterpret_cast<float4 *>(Bhi + off) = hv;
                *reinterpret_cast<float4 *>(Blo + off) = lv;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&phi_full[sp]));
            // the previous item's epilogue, once this item's first chunk is produced
            if (first && pend_j >= 0) epilogue(pend_j, pend_pt, pend_kz, pend_tt);
            if (first) { pend_j = cur.j; pend_pt = cur.pt; pend_kz = cur.kz; pend_tt = cur.tt; }
            if (++sc == SC) { sc = 0; pc ^= 1u; }
            if (s_abort) break;
        }
        if (pend_j >= 0 && !s_abort) epilogue(pend_j, pend_pt, pend_kz, pend_tt);
    } else if (warp == kTcProducerWarps && lane == 0) {
        // ---------------------------------------------------------------- MMA issuer
        // Per k-step: [c_hi ; c_lo] x phi_hi and [c_hi ; c_lo] x phi_lo (M = 128, N = 256, K = 8)
        // into the item's accumulator. The producers arrive on phi_full only after the chunk's
        // coefficient block has landed, so phi_full alone orders both operands.
        const uint32_t idesc = tc_idesc(kTcPts);
        TcCursor cur;
        cur.start(a);
        int cur_j = -1, sc = 0;
        int g = 0;
        bool ok = true;
        for (; cur.valid(a); ++g, cur.next(a)) {
            const int sp = g & 1;
            const bool first = cur.j != cur_j;
            cur_j = cur.j;
            const int acc = cur.j & 1;
            if (first && cur.j >= 2) ok = mbar_wait(smem_u32(&acc_empty[acc]), (uint32_t)(((cur.j - 2) >> 1) & 1));
            ok = ok && mbar_wait(smem_u32(&phi_full[sp]), (uint32_t)((g >> 1) & 1));
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t dc = smem_desc(smem_u32(c_base + sc * cblk));
            const uint64_t dh = smem_desc(smem_u32(phi_base + sp * 2 * phi_floats));
            const uint64_t dl = dh + (uint64_t)(phi_floats * 4 >> 4);
            const uint32_t d = tmem + acc * acc_cols;
#pragma unroll
            for (int ks = 0; ks < kTcK / 8; ++ks) {
                const uint64_t ko = (uint64_t)(ks * 2 * 128 >> 4);  // two core matrices (8 TF32) per k-step
                mma_tf32(d, dc + ko, dh + ko, idesc, (first && ks == 0) ? 0u : 1u);
                mma_tf32(d, dc + ko, dl + ko, idesc, 1u);
            }
            mma_commit(smem_u32(&phi_empty[sp]));
            mma_commit(smem_u32(&c_empty[sc]));
            if (cur.c + 1 == cur.c1) mma_commit(smem_u32(&acc_full[acc]));
            if (++sc == SC) sc = 0;
            if (s_abort) break;
        }
        if (!ok || s_abort) {
            s_abort = 1;
            atomicExch(a.status, RBFSL_ETIMEDOUT);
        }
        // every MMA of the CTA has completed once the last commit has
        if (g > 0) {
            const int gl = g - 1;
            mbar_wait(smem_u32(&phi_empty[gl & 1]), (uint32_t)((gl >> 1) & 1));
        }
    } else if (warp == kTcProducerWarps + 1 && lane == 0) {
        // ---------------------------------------------------------------- copy issuer
        constexpr uint32_t blk_bytes = (uint32_t)(cblk * sizeof(float));
        TcCursor cur;
        cur.start(a);
        int sc = 0;
        uint32_t pc = 0;
        int g = 0;
        for (; cur.valid(a); ++g, cur.next(a)) {
            if (g >= SC && !mbar_wait(smem_u32(&c_empty[sc]), pc ^ 1u)) {  // chunk g - SC's MMAs done
                s_abort = 1;
                atomicExch(a.status, RBFSL_ETIMEDOUT);
                break;
            }
            mbar_arrive_tx(smem_u32(&c_full[sc]), blk_bytes);
            const float *src = a.B + ((int64_t)cur.tt * a.nchunks + cur.c) * cblk;
            tma_bulk_g2s(smem_u32(c_base + sc * cblk), src, blk_bytes, smem_u32(&c_full[sc]));
            if (++sc == SC) { sc = 0; pc ^= 1u; }
            if (s_abort) break;
        }
        // wait (bounded) for the copies still in flight before the CTA's memory goes
        for (int gg = g - SC < 0 ? 0 : g - SC; gg < g; ++gg)
            mbar_wait(smem_u32(&c_full[gg % SC]), (uint32_t)((gg / SC) & 1));
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == kTcProducerWarps)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// Sum of the partial tiles in slice order: out[i][t] = sum_z part[z][i][t], z < nslices.
__global__ void tc_reduce_kernel(const float *__restrict__ part, int nslices, int64_t Nq, int T, int Tpad,
                                 float *__restrict__ out) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= Nq * T) return;
    const int64_t i = e / T, t = e - i * T;
    float s = 0.f;
    for (int z = 0; z < nslices; ++z) s += part[((int64_t)z * Nq + i) * Tpad + t];
    out[e] = s;
}

// Coefficients c (N x T, row-major, FP64 or FP32) and nodes X -> blocks [ttile][chunk] of
// tc_cblock_floats() floats: the A operand, rows 0..kTcTn-1 the TF32 rounding c_hi of the tile's
// tracers and rows kTcTn..2 kTcTn-1 the FP32 remainder c_lo = c - c_hi, kTcK nodes each, in
// core-matrix order (zero beyond N and T); then the chunk's kTcK nodes as FP32 float4 (zero
// beyond N). One thread per float of the blocks.
template <typename R>
__global__ void tc_prepare(const R *__restrict__ c, const double *__restrict__ X, int64_t N, int T, int ttiles,
                           int64_t nchunks, float *__restrict__ B) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    constexpr int cblk = tc_cblock_floats(), amat = 2 * kTcTn * kTcK;
    if (e >= (int64_t)ttiles * nchunks * cblk) return;
    const int64_t blk = e / cblk;
    const int w = (int)(e - blk * cblk);
    const int tt = (int)(blk / nchunks);
    const int64_t ch = blk - (int64_t)tt * nchunks;
    if (w >= amat) {  // node part
        const int f = w - amat, k = f >> 2, comp = f & 3;
        const int64_t j = ch * kTcK + k;
        B[e] = (comp < 3 && j < N) ? (float)X[3 * j + comp] : 0.f;
        return;
    }
    // invert core_off: w = ((n/8)*(kTcK/4) + k/4)*32 + (n%8)*4 + k%4, n the operand row
    const int core = w >> 5, in_core = w & 31;
    const int n = (core / (kTcK / 4)) * 8 + (in_core >> 2);
    const int k = (core % (kTcK / 4)) * 4 + (in_core & 3);
    const int half = n >= kTcTn;
    const int64_t j = ch * kTcK + k;
    const int t = tt * kTcTn + (n - half * kTcTn);
    const float v = (j < N && t < T) ? (float)c[j * T + t] : 0.f;
    const float h = tf32_rna(v);
    B[e] = half ? v - h : h;
}

struct TcPlan {
    int ttiles, Tpad, ksplit, ptiles, sc, grid;
    int64_t nchunks, nitems;
    size_t b_bytes, part_bytes, total, smem;
};

// Tiles, split and schedule: tracer tiles of kTcTn (T padded), point tiles of kTcPts; two phi
// stages and as many coefficient stages as fit (at most kTcMaxCStages); the node range split
// ksplit ways so that the persistent CTAs (one per SM) get equal numbers of items while each
// item keeps enough chunks: minimise waves x (chunks per item + 2), the 2 standing for an item's
// fixed cost (epilogue, pipeline refill), then prefer fewer splits.
TcPlan tc_plan(int64_t Nq, int64_t N, int T, int sms, int smem_optin) {
    TcPlan p{};
    p.ttiles = (T + kTcTn - 1) / kTcTn;
    p.Tpad = p.ttiles * kTcTn;
    p.nchunks = (N + kTcK - 1) / kTcK;
    p.ptiles = (int)((Nq + kTcPts - 1) / kTcPts);
    const size_t phi_bytes = (size_t)4 * kTcPts * kTcK * sizeof(float);
    const size_t cbytes = (size_t)tc_cblock_floats() * sizeof(float);
    const int sc = (int)(((size_t)smem_optin - 1024 - phi_bytes) / cbytes);
    p.sc = sc > kTcMaxCStages ? kTcMaxCStages : sc;
    p.smem = phi_bytes + (size_t)p.sc * cbytes;
    const int64_t tiles = (int64_t)p.ptiles * p.ttiles;
    double best = 1e300;
    p.ksplit = 1;
    for (int ks = 1; ks <= 64 && ks <= p.nchunks; ++ks) {
        const int64_t items = tiles * ks;
        const int64_t waves = (items + sms - 1) / sms;
        const double cost = (double)waves * ((double)((p.nchunks + ks - 1) / ks) + 2.0);
        if (cost < best * 0.98) {
            best = cost;
            p.ksplit = ks;
        }
    }
    p.nitems = tiles * p.ksplit;
    p.grid = (int)(p.nitems < sms ? p.nitems : sms);
    p.b_bytes = (size_t)p.ttiles * p.nchunks * cbytes;
    p.part_bytes = (size_t)2 * p.ksplit * Nq * p.Tpad * sizeof(float);
    p.total = p.b_bytes + p.part_bytes + 256;
    return p;
}

static void tc_device(int &sms, int &optin) {
    int dev = 0;
    sms = 152;
    optin = 232448;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        sms = 152;
        optin = 232448;
    }
}

size_t global_eval_tc_workspace(int64_t Nq, int64_t N, int T) {
    int sms, optin;
    tc_device(sms, optin);
    return tc_plan(Nq, N, T, sms, optin).total;
}

int launch_global_eval_tc(const double *P, int64_t Nq, const double *X, int64_t N, int kind, double eps,
                          const void *C, int c_dtype, int T, float *out, void *workspace, int32_t *status,
                          cudaStream_t s) {
    if (Nq == 0) return RBFSL_OK;
    int sms, optin;
    tc_device(sms, optin);
    const TcPlan p = tc_plan(Nq, N, T, sms, optin);
    if (p.sc < 2) {
        set_error("global_eval_tc: two coefficient stages do not fit in shared memory");
        return RBFSL_EINVAL;
    }
    char *ws = reinterpret_cast<char *>(workspace);
    float *B = reinterpret_cast<float *>(ws);
    float *part = reinterpret_cast<float *>(ws + p.b_bytes);
    if (!status) {  // the caller does not want the status: a word of the workspace takes it
        status = reinterpret_cast<int32_t *>(ws + p.b_bytes + p.part_bytes);
        RBFSL_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int32_t), s));
    }
    const int64_t tot = (int64_t)p.ttiles * p.nchunks * tc_cblock_floats();
    if (c_dtype == RBFSL_F64)
        tc_prepare<double><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>((const double *)C, X, N, T, p.ttiles,
                                                                         p.nchunks, B);
    else
        tc_prepare<float><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>((const float *)C, X, N, T, p.ttiles,
                                                                        p.nchunks, B);
    RBFSL_CUDA_TRY(cudaFuncSetAttribute(global_eval_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)p.smem));
    TcArgs a{};
    a.P = P; a.Nq = Nq; a.B = B; a.nchunks = p.nchunks; a.ksplit = p.ksplit; a.ptiles = p.ptiles;
    a.ttiles = p.ttiles; a.nitems = p.nitems; a.T = T; a.Tpad = p.Tpad; a.sc = p.sc; a.kind = kind;
    a.karg = kind == RBFSL_GAUSS ? (float)(-eps * eps * 1.4426950408889634) : (float)(eps * eps);
    a.part = part;
    a.status = status;
    global_eval_tc_kernel<<<p.grid, kTcThreads, p.smem, s>>>(a);
    RBFSL_CUDA_TRY(cudaGetLastError());
    tc_reduce_kernel<<<(unsigned)((Nq * T + 255) / 256), 256, 0, s>>>(part, 2 * p.ksplit, Nq, T, p.Tpad, out);
    return launch_status("global_eval_tc");
}

}  // namespace rbfsl

extern "C" size_t rbfsl_global_eval_tc_workspace_bytes(int64_t Nq, int64_t N, int T) {
    if (Nq < 0 || N < 1 || T < 1) return 0;
    return rbfsl::global_eval_tc_workspace(Nq, N, T);
}

extern "C" int rbfsl_global_eval_tc(const double *p, int64_t Nq, const double *x, int64_t N, int kernel,
                                    double eps, const void *c, int c_dtype, int T, float *out,
                                    void *workspace, size_t workspace_bytes, int32_t *status, void *stream) {
    using namespace rbfsl;
    RBFSL_CHECK_ARG(Nq >= 0 && N >= 1 && T >= 1, "global_eval_tc: bad sizes");
    RBFSL_CHECK_ARG(Nq == 0 || (p && x && c && out && workspace), "global_eval_tc: null pointer");
    RBFSL_CHECK_ARG((kernel == RBFSL_GAUSS || kernel == RBFSL_IMQ) && eps > 0, "global_eval_tc: bad kernel");
    RBFSL_CHECK_ARG(c_dtype == RBFSL_F64 || c_dtype == RBFSL_F32, "global_eval_tc: bad dtype");
    RBFSL_CHECK_ARG(workspace_bytes >= global_eval_tc_workspace(Nq, N, T), "global_eval_tc: workspace too small");
    RBFSL_CHECK_ARG(((uintptr_t)workspace & 15) == 0, "global_eval_tc: workspace must be 16-byte aligned");
    return launch_global_eval_tc(p, Nq, x, N, kernel, eps, c, c_dtype, T, out, workspace, status,
                                 (cudaStream_t)stream);
}
