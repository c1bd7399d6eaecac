// Batched local RBF-SL: many independent problems (own nodes, stencil size n, degree ell,
// velocity, tracers, precision, stencil mode) advanced together, one SL step (Algorithm 1)
// per graph replay:
//   1. batch_trace_kernel     departure points of every node of every active problem;
//   2. batch_solve_kernel     one persistent fused kernel per stencil class (mode, n, ell),
//                             the classes on parallel graph branches: blocks take tiles of the
//                             class's points from its counter; per point the k-NN stencil, the
//                             FP64 weights (direct solve or stored centre-stencil LU) and the
//                             gather-dot into the next field, with stencil and weights kept on
//                             chip. Each class's launch has its own block shared memory and
//                             grid, so a small class is not held to the largest class's
//                             occupancy;
//   3. batch_finalize_kernel  per-problem failure counters, time and step advance, counter
//                             reset.
// The per-point arithmetic is the same device code as the single-problem kernels
// (device_ops.cuh), so a problem's result is bit-identical alone or in any batch.
// Tile shape per (n, ell) class: one warp per point (four points per 128-thread block) or four
// warps per point; chosen by rbfsl_batch_autotune (timed) or by a size rule.
#include <algorithm>
#include <cmath>
#include <map>
#include <string>
#include <vector>

#include "common.cuh"
#include "device_ops.cuh"
#include "kernels.cuh"

namespace rbfsl {

struct BatchDesc {
    int64_t N;
    int n, ell, half, m, ld, T;
    int mode, mixed, ppt, active;
    int vel_kind;
    double vel[4];   // as given (kernel-ready forms are built on the device)
    double t, dt;    // t = time of the current field
    int64_t step;
    const double *X;
    KnnGrid grid;
    const double *LU;
    const int32_t *perm, *Ik;
    void *q[2];      // field ping-pong: input q[step & 1]
    double *xi;
    int32_t *status;
    unsigned long long *ctr;  // [singular, knn failures]
    int64_t node0, tile0;     // prefix offsets of this problem's nodes and tiles
};

__device__ __forceinline__ int find_problem(const BatchDesc *__restrict__ d, int np, int64_t g, bool tiles) {
    int lo = 0, hi = np - 1;
    while (lo < hi) {  // last problem whose offset <= g
        const int mid = (lo + hi + 1) >> 1;
        const int64_t off = tiles ? d[mid].tile0 : d[mid].node0;
        if (off <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ Vel<double> dev_vel64(const BatchDesc &p) {
    Vel<double> u{p.vel_kind, p.vel[0], p.vel[1], 0.0, 0.0};
    if (p.vel_kind == RBFSL_VEL_RIGID) { u.p2 = p.vel[2]; u.p3 = p.vel[3]; }
    else u.p1 = 3.14159265358979323846 / p.vel[1];
    return u;
}

__global__ void batch_trace_kernel(const BatchDesc *__restrict__ d, int np, int64_t total) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= total) return;
    const int p = find_problem(d, np, g, false);
    const BatchDesc &b = d[p];
    if (!b.active) return;
    const int64_t j = g - b.node0;
    const double t1 = b.t + b.dt;
    const double *X = b.X;
    double *Xi = b.xi;
    if (!b.mixed)
        rk4_point_f64(dev_vel64(b), X[3 * j], X[3 * j + 1], X[3 * j + 2], t1, -b.dt, Xi[3 * j], Xi[3 * j + 1], Xi[3 * j + 2]);
    else
        rk4_point_mixed(dev_vel64(b), X[3 * j], X[3 * j + 1], X[3 * j + 2], t1, -b.dt, Xi[3 * j], Xi[3 * j + 1],
                        Xi[3 * j + 2]);
}

// Shared memory of one point. Direct mode: system region (ldl_doubles), then the stencil (n
// int). Centre mode: right-hand side and solution (2 m double). The k-NN buffers (cap double +
// cap int + 1 int) alias the start of the region: the search ends, and its result is copied
// out, before the system or the right-hand side is written. A 109 x 109 system then takes
// 55.6 KB, four points per SM.
__host__ __device__ inline int batch_region_doubles(int mode, int n, int m, int ld) {
    return mode == RBFSL_DIRECT ? ldl_doubles(n, m) + (n + 1) / 2 : 2 * m;
}
__host__ __device__ inline int batch_point_doubles(int mode, int n, int m, int ld, int cap) {
    const int region = batch_region_doubles(mode, n, m, ld), knn = cap + (cap + 2) / 2;
    return region > knn ? region : knn;
}

// Gather-dot of one row from a point's weights (FP64 solution, split into FP32 pairs in mixed
// precision as the single-problem path stores them).
__device__ __forceinline__ void batch_gather(const BatchDesc &b, const double *w, const int32_t *S, int64_t i,
                                             int lane) {
    const int in = (int)(b.step & 1);
    if (!b.mixed) {
        gather_row<double, double>(w, S, b.n, (const double *)b.q[in], b.T, (double *)b.q[in ^ 1] + i * b.T, lane);
    } else {
        // FP32 pairs: each weight split into a pair exactly as a stored pair weight row, then
        // the same element arithmetic as gather_dot_pair_kernel
        const float2 *q = (const float2 *)b.q[in];
        float2 *out = (float2 *)b.q[in ^ 1] + i * b.T;
        for (int t = lane; t < b.T; t += 32) {
            float sh = 0.f, sl = 0.f;
            for (int j = 0; j < b.n; ++j) pair_fma(pair_from(w[j]), q[(int64_t)S[j] * b.T + t], sh, sl);
            out[t] = pair_norm(sh, sl);
        }
    }
}

// Tiles [tile_begin, tile_end) of the table's problems [p_begin, p_begin + np) (one class).
__global__ void __launch_bounds__(128, 4) batch_solve_kernel(const BatchDesc *__restrict__ d, int p_begin, int np,
                                                          int64_t tile_begin, int64_t tile_end,
                                                          unsigned long long *__restrict__ counter) {
    extern __shared__ double sm[];
    __shared__ long long s_tile;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    for (;;) {
        if (t == 0) s_tile = (long long)atomicAdd(counter, 1ULL);
        __syncthreads();
        const int64_t tile = tile_begin + s_tile;
        __syncthreads();
        if (tile >= tile_end) break;
        const int p = p_begin + find_problem(d + p_begin, np, tile, true);
        const BatchDesc &b = d[p];
        if (!b.active) continue;
        const int n = b.n, m = b.m, ld = b.ld, cap = knn_cap(b.mode == RBFSL_DIRECT ? n : 1);
        const int per = batch_point_doubles(b.mode, n, m, ld, cap);
        const int k = b.mode == RBFSL_DIRECT ? n : 1;
        if (b.ppt == 4 || b.mode == RBFSL_CENTER) {
            // one warp per point
            const int64_t i = (tile - b.tile0) * 4 + warp;
            if (i >= b.N) continue;
            double *base = sm + (size_t)warp * per;
            double *A = base;
            int32_t *S = reinterpret_cast<int32_t *>(base + ldl_doubles(n, m));  // direct only
            double *bd = base;  // aliases the region (see batch_point_doubles)
            int *bi = reinterpret_cast<int *>(bd + cap);
            int *cnt = bi + cap;
            const double px = b.xi[3 * i], py = b.xi[3 * i + 1], pz = b.xi[3 * i + 2];
            const bool ok = knn_warp(b.grid, px, py, pz, k, cap, bd, bi, cnt, lane);
            int rc = RBFSL_OK;
            if (!ok) {
                rc = RBFSL_EKNN;
            } else if (b.mode == RBFSL_DIRECT) {
                for (int j = lane; j < n; j += 32) S[j] = bi[j];
                __syncwarp();
                double *wv = nullptr;
                rc = weights_point_ldl<1>(A, b.X, S, n, m, b.ell, b.half, px, py, pz, lane, wv);
                if (rc == RBFSL_OK) batch_gather(b, wv, S, i, lane);
            } else {
                const int64_t kc = bi[0];
                const int32_t *Sg = b.Ik + kc * n;
                double *bb = A, *y = A + m;
                center_point(b.X, Sg, b.LU + (size_t)kc * m * m, b.perm + (size_t)kc * m, n, m, b.ell, b.half,
                             px, py, pz, bb, y, lane);
                batch_gather(b, y, Sg, i, lane);
            }
            if (rc != RBFSL_OK) {
                const int in = (int)(b.step & 1);
                for (int c = lane; c < b.T; c += 32) {
                    if (b.mixed) ((float2 *)b.q[in ^ 1])[i * b.T + c] = make_float2(NAN, NAN);
                    else ((double *)b.q[in ^ 1])[i * b.T + c] = NAN;
                }
            }
            if (lane == 0) b.status[i] = rc;
        } else {
            // four warps per point (direct mode)
            const int64_t i = tile - b.tile0;
            double *A = sm;
            int32_t *S = reinterpret_cast<int32_t *>(sm + ldl_doubles(n, m));
            double *bd = sm;  // aliases the region (see batch_point_doubles)
            int *bi = reinterpret_cast<int *>(bd + cap);
            int *cnt = bi + cap;
            const double px = b.xi[3 * i], py = b.xi[3 * i + 1], pz = b.xi[3 * i + 2];
            if (warp == 0) {
                const bool ok = knn_warp(b.grid, px, py, pz, k, cap, bd, bi, cnt, lane);
                for (int j = lane; j < n; j += 32) S[j] = ok ? bi[j] : -1;
            }
            __syncthreads();
            double *wv = nullptr;
            const int rc = weights_point_ldl<4>(A, b.X, S, n, m, b.ell, b.half, px, py, pz, t, wv);
            if (warp == 0) {
                if (rc == RBFSL_OK) {
                    batch_gather(b, wv, S, i, lane);
                } else {
                    const int in = (int)(b.step & 1);
                    for (int c = lane; c < b.T; c += 32) {
                        if (b.mixed) ((float2 *)b.q[in ^ 1])[i * b.T + c] = make_float2(NAN, NAN);
                        else ((double *)b.q[in ^ 1])[i * b.T + c] = NAN;
                    }
                }
                if (lane == 0) b.status[i] = rc;
            }
            __syncthreads();
        }
    }
}

__global__ void batch_count_kernel(BatchDesc *__restrict__ d, int np, int64_t total) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= total) return;
    const int p = find_problem(d, np, g, false);
    const BatchDesc &b = d[p];
    if (!b.active) return;
    const int32_t s = b.status[g - b.node0];
    if (s == RBFSL_ESINGULAR) atomicAdd(&b.ctr[0], 1ULL);
    else if (s == RBFSL_EKNN) atomicAdd(&b.ctr[1], 1ULL);
}

__global__ void batch_finalize_kernel(BatchDesc *__restrict__ d, int np, unsigned long long *__restrict__ counters,
                                      int nc) {
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
        if (!d[p].active) continue;
        d[p].t = d[p].t + d[p].dt;
        d[p].step += 1;
    }
    for (int c = threadIdx.x; c < nc; c += blockDim.x) counters[c] = 0ULL;
}

// One persistent launch per stencil class: its table range, tile range and launch shape.
struct ClassLaunch {
    int p0 = 0, np = 0;
    int64_t t0 = 0, t1 = 0;
    int smem = 0, grid = 0;
    long long key = 0;
};
constexpr int kMaxClasses = 64;  // class counters allocated with the batch

struct HostProblem {
    bool used = false;
    BatchDesc d{};
    rbfsl_knn_index *knn = nullptr;
    double *X = nullptr, *LU = nullptr, *xi = nullptr;
    int32_t *perm = nullptr, *Ik = nullptr, *status = nullptr;
    void *q[2] = {nullptr, nullptr};
    unsigned long long *ctr = nullptr;
    size_t bytes = 0;
};

}  // namespace rbfsl

struct rbfsl_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::vector<rbfsl::HostProblem> probs;
    rbfsl::BatchDesc *d_table = nullptr;
    int table_cap = 0;
    unsigned long long *d_counter = nullptr;  // kMaxClasses tile counters, one per class
    int np = 0;                    // slots in the device table (used problems, grouped by class)
    std::vector<int> slot_of;      // problem id -> table slot (-1 if not in the table)
    int64_t total_nodes = 0, total_tiles = 0;
    std::vector<rbfsl::ClassLaunch> classes;
    std::vector<cudaStream_t> side;      // class c > 0 runs on side[c - 1] (fork / join by events)
    std::vector<cudaEvent_t> side_done;
    cudaEvent_t fork = nullptr;
    bool dirty = true;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool use_graph = true;
    std::map<long long, int> tile_rule;  // (n, ell) -> points per tile (autotuned)
    size_t bytes = 0;
};

namespace rbfsl {
namespace {

long long class_key(int n, int ell) { return (long long)n * 64 + ell; }
long long group_key(const BatchDesc &d) { return (long long)d.mode * 1000000 + class_key(d.n, d.ell); }

int default_ppt(const rbfsl_batch *b, int n, int ell, int mode) {
    if (mode == RBFSL_CENTER) return 4;
    auto it = b->tile_rule.find(class_key(n, ell));
    if (it != b->tile_rule.end()) return it->second;
    const int m = n + (ell + 1) * (ell + 1);
    return ldl_doubles(n, m) * 8 > kWeightsSmallBytes ? 1 : 4;  // the single-problem rule
}

void free_problem(HostProblem &h) {
    if (h.knn) rbfsl_knn_index_destroy(h.knn);
    cudaFree(h.X); cudaFree(h.LU); cudaFree(h.xi); cudaFree(h.perm); cudaFree(h.Ik);
    cudaFree(h.status); cudaFree(h.q[0]); cudaFree(h.q[1]); cudaFree(h.ctr);
    h = HostProblem();
}

// Rebuild the device table (used problems grouped by stencil class, in id order within a
// class), prefix offsets, and each class's launch shape.
int rebuild(rbfsl_batch *b) {
    std::vector<BatchDesc> tab;
    b->slot_of.assign(b->probs.size(), -1);
    b->classes.clear();
    std::vector<long long> keys;
    for (auto &h : b->probs)
        if (h.used && std::find(keys.begin(), keys.end(), group_key(h.d)) == keys.end()) keys.push_back(group_key(h.d));
    std::sort(keys.begin(), keys.end());
    if ((int)keys.size() > kMaxClasses) {
        set_error("batch: more than 64 stencil classes");
        return RBFSL_EINVAL;
    }
    int64_t nodes = 0, tiles = 0;
    int max_smem = 0, sms = 0;
    RBFSL_CUDA_TRY(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device));
    RBFSL_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
    for (long long key : keys) {
        ClassLaunch cl;
        cl.key = key;
        cl.p0 = (int)tab.size();
        cl.t0 = tiles;
        for (size_t id = 0; id < b->probs.size(); ++id) {
            HostProblem &h = b->probs[id];
            if (!h.used || group_key(h.d) != key) continue;
            BatchDesc d = h.d;
            d.ppt = default_ppt(b, d.n, d.ell, d.mode);
            h.d.ppt = d.ppt;
            d.node0 = nodes;
            d.tile0 = tiles;
            nodes += d.N;
            tiles += d.ppt == 4 ? (d.N + 3) / 4 : d.N;
            const int cap = knn_cap(d.mode == RBFSL_DIRECT ? d.n : 1);
            const int per = batch_point_doubles(d.mode, d.n, d.m, d.ld, cap) * 8;
            cl.smem = std::max(cl.smem, d.ppt == 4 ? 4 * per : per);
            b->slot_of[id] = (int)tab.size();
            tab.push_back(d);
        }
        cl.np = (int)tab.size() - cl.p0;
        cl.t1 = tiles;
        if (cl.smem > max_smem) {
            set_error("batch: a problem's per-block shared memory (" + std::to_string(cl.smem) +
                      " bytes) exceeds the device limit");
            return RBFSL_EINVAL;
        }
        b->classes.push_back(cl);
    }
    if ((int)tab.size() > b->table_cap) {
        cudaFree(b->d_table);
        b->d_table = nullptr;
        b->table_cap = std::max<int>((int)tab.size(), 2 * b->table_cap);
        if (cudaMalloc(&b->d_table, b->table_cap * sizeof(BatchDesc)) != cudaSuccess) {
            cudaGetLastError();
            b->table_cap = 0;
            set_error("batch: out of device memory for the problem table");
            return RBFSL_ENOMEM;
        }
    }
    if (!tab.empty())
        RBFSL_CUDA_TRY(cudaMemcpyAsync(b->d_table, tab.data(), tab.size() * sizeof(BatchDesc),
                                       cudaMemcpyHostToDevice, b->stream));
    b->np = (int)tab.size();
    b->total_nodes = nodes;
    b->total_tiles = tiles;
    int smem_set = 0;
    for (auto &cl : b->classes) {
        if (cl.smem > smem_set) {  // the attribute is per kernel: the largest class's size
            RBFSL_CUDA_TRY(cudaFuncSetAttribute(batch_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, cl.smem));
            smem_set = cl.smem;
        }
    }
    for (auto &cl : b->classes) {
        int per_sm = 0;
        RBFSL_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_solve_kernel, 128, cl.smem));
        const int64_t g = (int64_t)std::max(1, per_sm) * sms;
        cl.grid = (int)std::max<int64_t>(1, std::min<int64_t>(g, cl.t1 - cl.t0));
    }
    while (b->side.size() + 1 < b->classes.size()) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        RBFSL_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaStreamDestroy(st);
            return launch_status("batch: event creation");
        }
        b->side.push_back(st);
        b->side_done.push_back(ev);
    }
    if (!b->fork) RBFSL_CUDA_TRY(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    b->dirty = false;
    return RBFSL_OK;
}

void launch_class(rbfsl_batch *b, int c, cudaStream_t s) {
    const ClassLaunch &cl = b->classes[c];
    batch_solve_kernel<<<cl.grid, 128, cl.smem, s>>>(b->d_table, cl.p0, cl.np, cl.t0, cl.t1, b->d_counter + c);
}

int enqueue_step(rbfsl_batch *b) {
    if (b->np == 0) return RBFSL_OK;
    const unsigned tb = (unsigned)((b->total_nodes + 255) / 256);
    batch_trace_kernel<<<tb, 256, 0, b->stream>>>(b->d_table, b->np, b->total_nodes);
    const int nc = (int)b->classes.size();
    if (nc > 1) {  // classes 1.. on side streams, forked from and joined back into the stream
        RBFSL_CUDA_TRY(cudaEventRecord(b->fork, b->stream));
        for (int c = 1; c < nc; ++c) {
            RBFSL_CUDA_TRY(cudaStreamWaitEvent(b->side[c - 1], b->fork, 0));
            launch_class(b, c, b->side[c - 1]);
            RBFSL_CUDA_TRY(cudaEventRecord(b->side_done[c - 1], b->side[c - 1]));
        }
    }
    if (nc > 0) launch_class(b, 0, b->stream);
    for (int c = 1; c < nc; ++c) RBFSL_CUDA_TRY(cudaStreamWaitEvent(b->stream, b->side_done[c - 1], 0));
    batch_count_kernel<<<tb, 256, 0, b->stream>>>(b->d_table, b->np, b->total_nodes);
    batch_finalize_kernel<<<1, 256, 0, b->stream>>>(b->d_table, b->np, b->d_counter, nc);
    return launch_status("batch step");
}

// The table keeps the device copy of time and step; pull them back before the host edits it.
int sync_table_to_host(rbfsl_batch *b) {
    if (b->np == 0) return RBFSL_OK;
    std::vector<BatchDesc> tab(b->np);
    RBFSL_CUDA_TRY(cudaMemcpyAsync(tab.data(), b->d_table, b->np * sizeof(BatchDesc), cudaMemcpyDeviceToHost, b->stream));
    RBFSL_CUDA_TRY(cudaStreamSynchronize(b->stream));
    for (size_t id = 0; id < b->probs.size(); ++id) {
        const int s = id < b->slot_of.size() ? b->slot_of[id] : -1;
        if (s < 0 || !b->probs[id].used) continue;
        b->probs[id].d.t = tab[s].t;
        b->probs[id].d.step = tab[s].step;
    }
    return RBFSL_OK;
}

}  // namespace
}  // namespace rbfsl

using namespace rbfsl;

extern "C" {

int rbfsl_batch_create(rbfsl_batch **out, int device, void *stream) {
    RBFSL_CHECK_ARG(out != nullptr, "batch_create: out is null");
    int ndev = 0;
    RBFSL_CUDA_TRY(cudaGetDeviceCount(&ndev));
    RBFSL_CHECK_ARG(device >= 0 && device < ndev, "batch_create: no such device");
    RBFSL_CUDA_TRY(cudaSetDevice(device));
    int rc = sh_tables_init();
    if (rc) return rc;
    auto *b = new rbfsl_batch();
    b->device = device;
    b->stream = (cudaStream_t)stream;
    if (cudaMalloc(&b->d_counter, kMaxClasses * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        set_error("batch_create: out of device memory");
        return RBFSL_ENOMEM;
    }
    RBFSL_CUDA_TRY(cudaMemset(b->d_counter, 0, kMaxClasses * sizeof(unsigned long long)));
    *out = b;
    return RBFSL_OK;
}

int rbfsl_batch_destroy(rbfsl_batch *b) {
    if (!b) return RBFSL_OK;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    for (auto &h : b->probs) free_problem(h);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaFree(b->d_table);
    cudaFree(b->d_counter);
    for (auto st : b->side) cudaStreamDestroy(st);
    for (auto ev : b->side_done) cudaEventDestroy(ev);
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
    return RBFSL_OK;
}

int rbfsl_batch_add(rbfsl_batch *b, const rbfsl_problem *pr, int *id_out) {
    RBFSL_CHECK_ARG(b && pr && id_out, "batch_add: null argument");
    RBFSL_CHECK_ARG(pr->N >= 1 && pr->N < ((int64_t)1 << 31) && pr->nodes && pr->q0, "batch_add: bad nodes or field");
    RBFSL_CHECK_ARG(pr->n >= 1 && pr->n <= pr->N && pr->ell >= 0 && pr->ell <= RBFSL_MAX_SH_DEGREE,
                    "batch_add: bad stencil size or degree");
    const int M = (pr->ell + 1) * (pr->ell + 1), m = pr->n + M;
    RBFSL_CHECK_ARG(m <= RBFSL_MAX_SYSTEM, "batch_add: n + (ell+1)^2 exceeds RBFSL_MAX_SYSTEM");
    const int pw = (int)pr->phs_power;
    RBFSL_CHECK_ARG((double)pw == pr->phs_power && pw >= 1 && (pw & 1), "batch_add: PHS power must be odd");
    RBFSL_CHECK_ARG(pr->mode == RBFSL_DIRECT || pr->mode == RBFSL_CENTER, "batch_add: bad stencil mode");
    RBFSL_CHECK_ARG(pr->precision == RBFSL_FP64 || pr->precision == RBFSL_MIXED, "batch_add: bad precision");
    RBFSL_CHECK_ARG(pr->vel_kind == RBFSL_VEL_RIGID || pr->vel_kind == RBFSL_VEL_DEFORM_Y2, "batch_add: bad velocity");
    RBFSL_CHECK_ARG(pr->T >= 1 && pr->T <= 256 && pr->dt > 0, "batch_add: bad T or dt");
    RBFSL_CUDA_TRY(cudaSetDevice(b->device));
    int rc;
    if ((rc = sync_table_to_host(b))) return rc;
    HostProblem h;
    h.used = true;
    const int64_t N = pr->N, n = pr->n;
    auto alloc = [&](void **p, size_t bytes) {
        if (cudaMalloc(p, bytes ? bytes : 1) != cudaSuccess) {
            cudaGetLastError();
            set_error("batch_add: out of device memory");
            return RBFSL_ENOMEM;
        }
        h.bytes += bytes;
        return RBFSL_OK;
    };
    const size_t es = 8;  // FP64, or an FP32 pair (mixed)
    if ((rc = alloc((void **)&h.X, N * 3 * sizeof(double))) || (rc = alloc((void **)&h.xi, N * 3 * sizeof(double))) ||
        (rc = alloc((void **)&h.status, N * sizeof(int32_t))) || (rc = alloc(&h.q[0], N * pr->T * es)) ||
        (rc = alloc(&h.q[1], N * pr->T * es)) || (rc = alloc((void **)&h.ctr, 2 * sizeof(unsigned long long)))) {
        free_problem(h);
        return rc;
    }
    cudaStream_t s = b->stream;
    RBFSL_CUDA_TRY(cudaMemcpyAsync(h.X, pr->nodes, N * 3 * sizeof(double), cudaMemcpyHostToDevice, s));
    RBFSL_CUDA_TRY(cudaMemsetAsync(h.ctr, 0, 2 * sizeof(unsigned long long), s));
    if (pr->precision == RBFSL_FP64) {
        RBFSL_CUDA_TRY(cudaMemcpyAsync(h.q[0], pr->q0, N * pr->T * 8, cudaMemcpyHostToDevice, s));
    } else {
        std::vector<float> q32((size_t)N * pr->T * 2);
        for (size_t e = 0; e < (size_t)N * pr->T; ++e) {
            const float hi = (float)pr->q0[e];
            q32[2 * e] = hi;
            q32[2 * e + 1] = (float)(pr->q0[e] - (double)hi);
        }
        RBFSL_CUDA_TRY(cudaMemcpyAsync(h.q[0], q32.data(), q32.size() * 4, cudaMemcpyHostToDevice, s));
        RBFSL_CUDA_TRY(cudaStreamSynchronize(s));
    }
    if ((rc = rbfsl_knn_index_create(&h.knn, h.X, N, pr->n, s))) { free_problem(h); return rc; }
    h.bytes += h.knn->bytes;
    if (pr->mode == RBFSL_CENTER) {
        if ((rc = alloc((void **)&h.Ik, N * n * sizeof(int32_t))) ||
            (rc = alloc((void **)&h.LU, (size_t)N * m * m * sizeof(double))) ||
            (rc = alloc((void **)&h.perm, (size_t)N * m * sizeof(int32_t)))) {
            free_problem(h);
            return rc;
        }
        if ((rc = launch_knn(h.knn, h.X, N, (int)n, h.Ik, h.status, s))) { free_problem(h); return rc; }
        std::vector<int64_t> ms(N + 1), lo(N);
        for (int64_t k = 0; k <= N; ++k) ms[k] = k * n;
        for (int64_t k = 0; k < N; ++k) lo[k] = k * (int64_t)m * m;
        int64_t *d_ms = nullptr, *d_lo = nullptr;
        int32_t *d_bad = nullptr;
        if (cudaMalloc(&d_ms, (N + 1) * sizeof(int64_t)) != cudaSuccess || cudaMalloc(&d_lo, N * sizeof(int64_t)) != cudaSuccess ||
            cudaMalloc(&d_bad, sizeof(int32_t)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(d_ms); cudaFree(d_lo);
            free_problem(h);
            set_error("batch_add: out of device memory");
            return RBFSL_ENOMEM;
        }
        cudaMemcpyAsync(d_ms, ms.data(), (N + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_lo, lo.data(), N * sizeof(int64_t), cudaMemcpyHostToDevice, s);
        cudaMemsetAsync(d_bad, 0, sizeof(int32_t), s);
        rc = launch_stencil_factor(h.X, d_ms, h.Ik, d_lo, N, (int)n, M, pr->ell, pw, h.LU, h.perm, d_bad, s, 1);
        int32_t bad = 0;
        if (rc == RBFSL_OK && (cudaMemcpyAsync(&bad, d_bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                               cudaStreamSynchronize(s) != cudaSuccess)) {
            cudaGetLastError();
            set_error("batch_add: centre factorisation failed");
            rc = RBFSL_ECUDA;
        }
        cudaFree(d_ms); cudaFree(d_lo); cudaFree(d_bad);
        if (rc == RBFSL_OK && bad) { set_error("batch_add: singular centre stencil"); rc = RBFSL_ESINGULAR; }
        if (rc) { free_problem(h); return rc; }
    }
    RBFSL_CUDA_TRY(cudaStreamSynchronize(s));
    BatchDesc &d = h.d;
    d.N = N; d.n = (int)n; d.ell = pr->ell; d.half = (pw - 1) / 2; d.m = m; d.ld = (m + 1) | 1; d.T = pr->T;
    d.mode = pr->mode; d.mixed = pr->precision == RBFSL_MIXED; d.active = 1;
    d.vel_kind = pr->vel_kind;
    for (int i = 0; i < 4; ++i) d.vel[i] = pr->vel_params[i];
    d.t = pr->t0; d.dt = pr->dt; d.step = 0;
    d.X = h.X; d.grid = grid_view(h.knn); d.LU = h.LU; d.perm = h.perm; d.Ik = h.Ik;
    d.q[0] = h.q[0]; d.q[1] = h.q[1]; d.xi = h.xi; d.status = h.status; d.ctr = h.ctr;
    int id = -1;
    for (size_t i = 0; i < b->probs.size(); ++i)
        if (!b->probs[i].used) { id = (int)i; break; }
    if (id < 0) { id = (int)b->probs.size(); b->probs.emplace_back(); }
    b->probs[id] = h;
    b->bytes += h.bytes;
    b->dirty = true;
    *id_out = id;
    return RBFSL_OK;
}

int rbfsl_batch_remove(rbfsl_batch *b, int id) {
    RBFSL_CHECK_ARG(b && id >= 0 && id < (int)b->probs.size() && b->probs[id].used, "batch_remove: no such problem");
    RBFSL_CUDA_TRY(cudaSetDevice(b->device));
    int rc;
    if ((rc = sync_table_to_host(b))) return rc;
    b->bytes -= b->probs[id].bytes;
    free_problem(b->probs[id]);
    b->dirty = true;
    return RBFSL_OK;
}

int rbfsl_batch_step(rbfsl_batch *b, int nsteps) {
    RBFSL_CHECK_ARG(b && nsteps >= 0, "batch_step: bad arguments");
    RBFSL_CUDA_TRY(cudaSetDevice(b->device));
    int rc;
    if (b->dirty && (rc = rebuild(b))) return rc;
    if (b->np == 0 || nsteps == 0) return RBFSL_OK;
    if (b->use_graph && !b->exec) {
        // one SL step of every problem as a graph, replayed per step
        RBFSL_CUDA_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        rc = enqueue_step(b);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
        if (rc || e != cudaSuccess) {
            cudaGetLastError();
            if (g) cudaGraphDestroy(g);
            b->use_graph = false;  // fall back to eager launches of the same kernels
        } else {
            b->graph = g;
            if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
                cudaGetLastError();
                b->use_graph = false;
                b->exec = nullptr;
            }
        }
    }
    for (int k = 0; k < nsteps; ++k) {
        if (b->exec) RBFSL_CUDA_TRY(cudaGraphLaunch(b->exec, b->stream));
        else if ((rc = enqueue_step(b))) return rc;
    }
    return RBFSL_OK;
}

int rbfsl_batch_get_q(rbfsl_batch *b, int id, double *out) {
    RBFSL_CHECK_ARG(b && out && id >= 0 && id < (int)b->probs.size() && b->probs[id].used, "batch_get_q: no such problem");
    RBFSL_CUDA_TRY(cudaSetDevice(b->device));
    int rc;
    if ((rc = sync_table_to_host(b))) return rc;
    HostProblem &h = b->probs[id];
    const size_t cnt = (size_t)h.d.N * h.d.T;
    const void *src = h.q[h.d.step & 1];
    if (!h.d.mixed) {
        RBFSL_CUDA_TRY(cudaMemcpyAsync(out, src, cnt * 8, cudaMemcpyDeviceToHost, b->stream));
        RBFSL_CUDA_TRY(cudaStreamSynchronize(b->stream));
    } else {
        std::vector<float> tmp(cnt * 2);
        RBFSL_CUDA_TRY(cudaMemcpyAsync(tmp.data(), src, cnt * 8, cudaMemcpyDeviceToHost, b->stream));
        RBFSL_CUDA_TRY(cudaStreamSynchronize(b->stream));
        for (size_t e = 0; e < cnt; ++e) out[e] = (double)tmp[2 * e] + (double)tmp[2 * e + 1];
    }
    return RBFSL_OK;
}

int rbfsl_batch_problem_stats(rbfsl_batch *b, int id, rbfsl_stats *out) {
    RBFSL_CHECK_ARG(b && out && id >= 0 && id < (int)b->probs.size() && b->probs[id].used, "batch_stats: no such problem");
    RBFSL_CUDA_TRY(cudaSetDevice(b->device));
    int rc;
    if ((rc = sync_table_to_host(b))) return rc;
    HostProblem &h = b->probs[id];
    unsigned long long c[2] = {0, 0};
    RBFSL_CUDA_TRY(cudaMemcpy(c, h.ctr, sizeof(c), cudaMemcpyDeviceToHost));
    *out = rbfsl_stats{};
    out->steps_done = h.d.step;
    out->singular_points = (int64_t)c[0];
    out->knn_failures = (int64_t)c[1];
    out->time = h.d.t;
    out->device_bytes = h.bytes;
    return RBFSL_OK;
}

int rbfsl_batch_set_graph(rbfsl_batch *b, int use_graph) {
    RBFSL_CHECK_ARG(b != nullptr, "batch_set_graph: null batch");
    b->use_graph = use_graph != 0;
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    return RBFSL_OK;
}

// Time the persistent solve kernel for each direct-mode (n, ell) class of the batch with one
// warp per point and with four warps per point, keep the faster. The timing launches run on
// the current departure points and leave the fields, times and step counters unchanged.
int rbfsl_batch_autotune(rbfsl_batch *b, int *choices, int max_choices) {
    RBFSL_CHECK_ARG(b != nullptr, "batch_autotune: null batch");
    RBFSL_CUDA_TRY(cudaSetDevice(b->device));
    int rc;
    if ((rc = sync_table_to_host(b))) return rc;
    std::vector<long long> classes;
    for (auto &h : b->probs)
        if (h.used && h.d.mode == RBFSL_DIRECT) {
            const long long key = class_key(h.d.n, h.d.ell);
            if (std::find(classes.begin(), classes.end(), key) == classes.end()) classes.push_back(key);
        }
    cudaEvent_t e0, e1;
    RBFSL_CUDA_TRY(cudaEventCreate(&e0));
    RBFSL_CUDA_TRY(cudaEventCreate(&e1));
    int max_smem = 0;
    RBFSL_CUDA_TRY(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device));
    int nout = 0;
    for (long long key : classes) {
        float best_ms = 1e30f;
        int best = 1;
        const int kn = (int)(key / 64), kell = (int)(key % 64), km = kn + (kell + 1) * (kell + 1);
        const int per_bytes = batch_point_doubles(RBFSL_DIRECT, kn, km, (km + 1) | 1, knn_cap(kn)) * 8;
        for (int ppt : {4, 1}) {
            if (ppt == 4 && 4 * per_bytes > max_smem) continue;
            // only this class active, with the candidate tile shape
            std::vector<int> saved;
            for (auto &h : b->probs) {
                saved.push_back(h.d.active);
                if (h.used) h.d.active = (h.d.mode == RBFSL_DIRECT && class_key(h.d.n, h.d.ell) == key) ? 1 : 0;
            }
            b->tile_rule[key] = ppt;
            if ((rc = rebuild(b))) break;
            int c = 0;
            while (c < (int)b->classes.size() && b->classes[c].key != (long long)RBFSL_DIRECT * 1000000 + key) ++c;
            if (c == (int)b->classes.size()) { rc = RBFSL_EINVAL; set_error("batch_autotune: class not found"); break; }
            const unsigned tb = (unsigned)((b->total_nodes + 255) / 256);
            batch_trace_kernel<<<tb, 256, 0, b->stream>>>(b->d_table, b->np, b->total_nodes);
            cudaMemsetAsync(b->d_counter + c, 0, sizeof(unsigned long long), b->stream);
            launch_class(b, c, b->stream);
            cudaMemsetAsync(b->d_counter + c, 0, sizeof(unsigned long long), b->stream);
            cudaEventRecord(e0, b->stream);
            launch_class(b, c, b->stream);
            cudaEventRecord(e1, b->stream);
            cudaMemsetAsync(b->d_counter + c, 0, sizeof(unsigned long long), b->stream);
            if ((rc = launch_status("batch_autotune"))) break;
            RBFSL_CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_ms) { best_ms = ms; best = ppt; }
            size_t k = 0;
            for (auto &h : b->probs) h.d.active = saved[k++];
        }
        if (rc) break;
        b->tile_rule[key] = best;
        if (choices && nout + 2 < max_choices) {
            choices[nout++] = (int)(key / 64);
            choices[nout++] = (int)(key % 64);
            choices[nout++] = best;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->dirty = true;
    if (rc == RBFSL_OK) rc = rebuild(b);
    return rc;
}

}  // extern "C"
