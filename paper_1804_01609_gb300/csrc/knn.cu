// k-nearest-neighbour search on S^2 (stencil selection, Sec. 2.2 and 3.3; the paper uses a
// kd-tree). Here a uniform grid over [-1,1]^3 holds the nodes sorted by cell; a query
// brackets its k nearest nodes by collecting every node with d2 <= r^2 from the cells that
// overlap the ball of radius r (r grown or shrunk until the count lies in [k, CAP]), then
// sorts the candidates by the key (d2, index). The candidates with d2 <= r^2 contain the k
// smallest keys, so the result equals a brute-force search bit for bit, with d2 computed in
// a fixed rounding order and ties broken by the smaller node index.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "device_ops.cuh"

namespace rbfsl {

__global__ void knn_cell_count(const double *__restrict__ X, int64_t N, int G, double inv_cell,
                               int32_t *__restrict__ cell_of, int32_t *__restrict__ counts) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= N) return;
    const int cx = cell_coord(X[3 * j], inv_cell, G);
    const int cy = cell_coord(X[3 * j + 1], inv_cell, G);
    const int cz = cell_coord(X[3 * j + 2], inv_cell, G);
    const int c = (cz * G + cy) * G + cx;
    cell_of[j] = c;
    atomicAdd(&counts[c], 1);
}

// Exclusive scan of counts[0..C) into start[0..C] by one block (set-up only).
__global__ void knn_scan_single_block(const int32_t *__restrict__ counts, int64_t C,
                                      int32_t *__restrict__ start) {
    __shared__ int64_t part[1024];
    const int t = threadIdx.x;
    const int64_t chunk = (C + blockDim.x - 1) / blockDim.x;
    const int64_t b = t * chunk, e = min(C, b + chunk);
    int64_t s = 0;
    for (int64_t i = b; i < e; ++i) s += counts[i];
    part[t] = s;
    __syncthreads();
    if (t == 0) {
        int64_t acc = 0;
        for (int i = 0; i < (int)blockDim.x; ++i) {
            const int64_t v = part[i];
            part[i] = acc;
            acc += v;
        }
        start[C] = (int32_t)acc;
    }
    __syncthreads();
    int64_t acc = part[t];
    for (int64_t i = b; i < e; ++i) {
        start[i] = (int32_t)acc;
        acc += counts[i];
    }
}

__global__ void knn_scatter(const double *__restrict__ X, int64_t N,
                            const int32_t *__restrict__ cell_of,
                            const int32_t *__restrict__ start, int32_t *__restrict__ fill,
                            double *__restrict__ sx, double *__restrict__ sy,
                            double *__restrict__ sz, int32_t *__restrict__ sid) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= N) return;
    const int c = cell_of[j];
    const int pos = start[c] + atomicAdd(&fill[c], 1);
    sx[pos] = X[3 * j];
    sy[pos] = X[3 * j + 1];
    sz[pos] = X[3 * j + 2];
    sid[pos] = (int32_t)j;
}

int knn_index_build(rbfsl_knn_index *ix, const double *x, int64_t N, int k_hint,
                    cudaStream_t s) {
    ix->N = N;
    ix->r2_per_k = 4.0 * 1.3 / (double)N;  // a chord-ball of radius r holds ~N r^2 / 4 nodes
    const double r0 = std::sqrt(ix->r2_per_k * std::max(1, k_hint));
    int G = (int)std::ceil(2.0 / (0.5 * r0));
    ix->G = std::min(256, std::max(1, G));
    ix->cell = 2.0 / ix->G;
    const int64_t C = (int64_t)ix->G * ix->G * ix->G;
    int32_t *cell_of = nullptr, *counts = nullptr;
    ix->bytes = (size_t)N * (3 * sizeof(double) + sizeof(int32_t)) + (C + 1) * sizeof(int32_t);
    if (cudaMalloc(&ix->sx, N * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&ix->sy, N * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&ix->sz, N * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&ix->sid, N * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&ix->cell_start, (C + 1) * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&cell_of, N * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&counts, C * sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(cell_of);
        cudaFree(counts);
        set_error("knn_index_create: out of device memory");
        return RBFSL_ENOMEM;
    }
    int rc = RBFSL_OK;
    const double inv_cell = ix->G / 2.0;
    const unsigned blocks = (unsigned)((N + 255) / 256);
    if (cudaMemsetAsync(counts, 0, C * sizeof(int32_t), s) != cudaSuccess) rc = RBFSL_ECUDA;
    if (rc == RBFSL_OK) {
        knn_cell_count<<<blocks, 256, 0, s>>>(x, N, ix->G, inv_cell, cell_of, counts);
        knn_scan_single_block<<<1, 1024, 0, s>>>(counts, C, ix->cell_start);
        if (cudaMemsetAsync(counts, 0, C * sizeof(int32_t), s) != cudaSuccess) rc = RBFSL_ECUDA;
    }
    if (rc == RBFSL_OK) {
        knn_scatter<<<blocks, 256, 0, s>>>(x, N, cell_of, ix->cell_start, counts, ix->sx, ix->sy,
                                           ix->sz, ix->sid);
        rc = launch_status("knn_index_build");
    }
    if (rc == RBFSL_OK && cudaStreamSynchronize(s) != cudaSuccess) {
        set_error(std::string("knn_index_build: ") + cudaGetErrorString(cudaGetLastError()));
        rc = RBFSL_ECUDA;
    }
    cudaFree(cell_of);
    cudaFree(counts);
    return rc;
}

void knn_index_free(rbfsl_knn_index *ix) {
    cudaFree(ix->sx);
    cudaFree(ix->sy);
    cudaFree(ix->sz);
    cudaFree(ix->sid);
    cudaFree(ix->cell_start);
    ix->sx = ix->sy = ix->sz = nullptr;
    ix->sid = ix->cell_start = nullptr;
}

// One warp per query. Shared memory per warp: cap doubles + cap ints + 1 counter.
__global__ void __launch_bounds__(128) knn_query_kernel(KnnGrid g, const double *__restrict__ Q,
                                                        int64_t Nq, int k, int cap,
                                                        int32_t *__restrict__ idx,
                                                        int32_t *__restrict__ status) {
    extern __shared__ unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    double *bd = reinterpret_cast<double *>(smem_raw) + (size_t)warp * cap;
    int *bi = reinterpret_cast<int *>(reinterpret_cast<double *>(smem_raw) + (size_t)wpb * cap) +
              (size_t)warp * cap;
    int *cnt = reinterpret_cast<int *>(reinterpret_cast<double *>(smem_raw) + (size_t)wpb * cap) +
               (size_t)wpb * cap + warp;
    const int64_t q = (int64_t)blockIdx.x * wpb + warp;
    if (q >= Nq) return;
    const bool ok = knn_warp(g, Q[3 * q], Q[3 * q + 1], Q[3 * q + 2], k, cap, bd, bi, cnt, lane);
    for (int r = lane; r < k; r += kWarp) idx[q * k + r] = ok ? bi[r] : -1;
    if (status && lane == 0) status[q] = ok ? RBFSL_OK : RBFSL_EKNN;
}

int launch_knn(const rbfsl_knn_index *ix, const double *q, int64_t Nq, int k, int32_t *idx,
               int32_t *status, cudaStream_t s) {
    if (Nq == 0) return RBFSL_OK;
    const int cap = knn_cap(k);
    const int wpb = 4;
    const size_t smem = (size_t)wpb * cap * (sizeof(double) + sizeof(int)) + wpb * sizeof(int);
    const KnnGrid g = grid_view(ix);
    if (smem > 48 * 1024)
        RBFSL_CUDA_TRY(cudaFuncSetAttribute(knn_query_kernel,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const unsigned blocks = (unsigned)((Nq + wpb - 1) / wpb);
    knn_query_kernel<<<blocks, wpb * kWarp, smem, s>>>(g, q, Nq, k, cap, idx, status);
    return launch_status("knn_query");
}

}  // namespace rbfsl

extern "C" int rbfsl_knn_index_create(rbfsl_knn_index **out, const double *x, int64_t N,
                                      int k_hint, void *stream) {
    using namespace rbfsl;
    RBFSL_CHECK_ARG(out != nullptr, "knn_index_create: out is null");
    RBFSL_CHECK_ARG(N >= 1 && N < (int64_t)1 << 31, "knn_index_create: N out of range");
    RBFSL_CHECK_ARG(x != nullptr, "knn_index_create: x is null");
    auto *ix = new rbfsl_knn_index{};
    RBFSL_CUDA_TRY(cudaGetDevice(&ix->device));
    int rc = knn_index_build(ix, x, N, k_hint, (cudaStream_t)stream);
    if (rc != RBFSL_OK) {
        knn_index_free(ix);
        delete ix;
        return rc;
    }
    *out = ix;
    return RBFSL_OK;
}

extern "C" int rbfsl_knn_index_destroy(rbfsl_knn_index *ix) {
    if (!ix) return RBFSL_OK;
    rbfsl::knn_index_free(ix);
    delete ix;
    return RBFSL_OK;
}

extern "C" int rbfsl_knn_query(const rbfsl_knn_index *ix, const double *q, int64_t Nq, int k,
                               int32_t *idx, int32_t *status, void *stream) {
    using namespace rbfsl;
    RBFSL_CHECK_ARG(ix != nullptr, "knn_query: index is null");
    RBFSL_CHECK_ARG(Nq >= 0, "knn_query: Nq < 0");
    RBFSL_CHECK_ARG(k >= 1 && k <= RBFSL_MAX_K && k <= ix->N, "knn_query: k out of range");
    RBFSL_CHECK_ARG(Nq == 0 || (q && idx), "knn_query: null pointer");
    return launch_knn(ix, q, Nq, k, idx, status, (cudaStream_t)stream);
}
