// Internal launchers shared by the C-ABI entry points and the context.
#pragma once

#include "common.cuh"

struct rbfsl_knn_index {
    int device;
    int64_t N;
    int G;                 // cells per axis over [-1, 1]^3
    double cell;           // cell edge 2 / G
    double r2_per_k;       // initial squared search radius per neighbour: 4 * 1.3 / N
    double *sx, *sy, *sz;  // node coordinates sorted by cell (SoA)
    int32_t *sid;          // original node index of each sorted entry
    int32_t *cell_start;   // G^3 + 1 offsets into the sorted arrays
    size_t bytes;
};

namespace rbfsl {

int launch_trace(const double *x, int64_t N, int vel_kind, const double *prm, double t1,
                 double dt, int precision, double *xi, cudaStream_t s);

int knn_index_build(rbfsl_knn_index *ix, const double *x, int64_t N, int k_hint, cudaStream_t s);
void knn_index_free(rbfsl_knn_index *ix);
int launch_knn(const rbfsl_knn_index *ix, const double *q, int64_t Nq, int k, int32_t *idx,
               int32_t *status, cudaStream_t s);

int launch_weights(const double *x, const int32_t *idx, int64_t Nq, int n, int ell, int power,
                   const double *p, void *w, int w_dtype, int32_t *status, cudaStream_t s);

int launch_gather(const int32_t *idx, const void *w, int64_t Nq, int n, const void *q, int T,
                  int dtype, void *q_out, cudaStream_t s);

int global_factor_full(const double *x, int64_t N, int kernel, double eps, double *LU, int32_t *perm,
                       int32_t *piv, int32_t *status, cudaStream_t s);
int global_solve(const double *LU, const int32_t *perm, int64_t N, const double *Q, int T,
                 double *C, cudaStream_t s);
int launch_global_eval(const double *P, int64_t Nq, const double *X, int64_t N, int kind,
                       double eps, const void *C, int T, int dtype, void *out, int out_dtype,
                       cudaStream_t s);

}  // namespace rbfsl
