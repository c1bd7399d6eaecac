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

// RBF-PU patches and factors (pu.cu).
struct rbfsl_pu {
    int device = 0;
    int64_t N = 0, Mp = 0;
    double R = 0;
    int ell = 0, power = 0, M = 0, max_members = 0;
    double *X = nullptr, *centers = nullptr;
    int64_t *mstart = nullptr;   // Mp + 1 (device)
    int32_t *members = nullptr;  // mstart[Mp] (device), ascending node index per patch
    int64_t *lu_off = nullptr;   // Mp (device): offset of patch l's m_l x m_l factor
    double *LU = nullptr;
    int32_t *perm = nullptr;     // row order of each factor, at mstart[l] + l * M
    rbfsl_knn_index *nodes_ix = nullptr, *centers_ix = nullptr;
    double *coef = nullptr;      // (mstart[Mp] + Mp M) x coef_T
    void *coef32 = nullptr;      // FP32 or FP32-pair copy of coef for the mixed evaluations
    int coef_T = 0;
    int64_t coef_len = 0;        // values in coef
    int32_t *status = nullptr;
    size_t bytes = 0;
};

namespace rbfsl {

// Device view of a grid index (see knn.cu).
struct KnnGrid {
    const double *sx, *sy, *sz;
    const int32_t *sid, *cell_start;
    int G;
    double inv_cell;
    double r2_per_k;
};

inline KnnGrid grid_view(const rbfsl_knn_index *ix) {
    return KnnGrid{ix->sx, ix->sy, ix->sz, ix->sid, ix->cell_start, ix->G, ix->G / 2.0, ix->r2_per_k};
}

__device__ __forceinline__ int cell_coord(double v, double inv_cell, int G) {
    int c = (int)floor((v + 1.0) * inv_cell);
    return c < 0 ? 0 : (c >= G ? G - 1 : c);
}

// Calls f(sorted_position) for every indexed point in the cells that overlap the ball of
// radius rb around (qx, qy, qz); the cells are dealt to the lanes of a warp (lane, lane+32..).
template <typename F>
__device__ __forceinline__ void grid_ball_foreach(const KnnGrid &g, double qx, double qy, double qz,
                                                  double rb, int lane, F f) {
    const int x0 = cell_coord(qx - rb, g.inv_cell, g.G), x1 = cell_coord(qx + rb, g.inv_cell, g.G);
    const int y0 = cell_coord(qy - rb, g.inv_cell, g.G), y1 = cell_coord(qy + rb, g.inv_cell, g.G);
    const int z0 = cell_coord(qz - rb, g.inv_cell, g.G), z1 = cell_coord(qz + rb, g.inv_cell, g.G);
    const int nx = x1 - x0 + 1, ny = y1 - y0 + 1, nz = z1 - z0 + 1;
    const int nb = nx * ny * nz;
    for (int t = lane; t < nb; t += 32) {
        const int cx = x0 + t % nx, cy = y0 + (t / nx) % ny, cz = z0 + t / (nx * ny);
        const int c = (cz * g.G + cy) * g.G + cx;
        const int b = g.cell_start[c], e = g.cell_start[c + 1];
        for (int p = b; p < e; ++p) f(p);
    }
}

int launch_trace(const double *x, int64_t N, int vel_kind, const double *prm, double t1,
                 double dt, int precision, double *xi, cudaStream_t s);

int knn_index_build(rbfsl_knn_index *ix, const double *x, int64_t N, int k_hint, cudaStream_t s);
void knn_index_free(rbfsl_knn_index *ix);
int launch_knn(const rbfsl_knn_index *ix, const double *q, int64_t Nq, int k, int32_t *idx,
               int32_t *status, cudaStream_t s);

int launch_weights(const double *x, const int32_t *idx, int64_t Nq, int n, int ell, int power,
                   const double *p, void *w, int w_dtype, int32_t *status, cudaStream_t s);

int launch_trace_order(const double *x, int64_t N, int vel_kind, const double *prm, double t1, double dt,
                       int precision, int order, double *xi, cudaStream_t s);

int launch_gather(const int32_t *idx, const void *w, int64_t Nq, int n, const void *q, int T,
                  int dtype, void *q_out, cudaStream_t s);

int sh_tables_init();

int launch_stencil_factor(const double *X, const int64_t *mstart, const int32_t *members,
                          const int64_t *lu_off, int64_t count, int max_n, int M, int ell,
                          int power, double *LU, int32_t *perm, int32_t *status, cudaStream_t s,
                          int colmajor);
int launch_center_weights(const double *X, const int32_t *K, const int32_t *Ik, const double *LU,
                          const int32_t *perm, int64_t Nq, int n, int ell, int power,
                          const double *p, int32_t *I, void *w, int w_dtype, int32_t *status,
                          cudaStream_t s);

int global_factor_full(const double *x, int64_t N, int kernel, double eps, double *LU, int32_t *perm,
                       int32_t *piv, int32_t *status, cudaStream_t s);
int global_factor_chol_full(const double *x, int64_t N, int kernel, double eps, double *LU, int32_t *perm,
                            cudaStream_t s);
int global_solve(const double *LU, const int32_t *perm, int64_t N, const double *Q, int T,
                 double *C, cudaStream_t s);
int launch_global_eval(const double *P, int64_t Nq, const double *X, int64_t N, int kind,
                       double eps, const void *C, int T, int dtype, void *out, int out_dtype,
                       cudaStream_t s);
size_t global_eval_tc_workspace(int64_t Nq, int64_t N, int T);
int launch_global_eval_tc(const double *P, int64_t Nq, const double *X, int64_t N, int kind, double eps,
                          const void *C, int c_dtype, int T, float *out, void *workspace, int32_t *status,
                          cudaStream_t s);

size_t global_eval_pairs_workspace(int64_t Nq, int64_t N, int T);
int launch_global_eval_pairs(const double *P, int64_t Nq, const double *X, int64_t N, int kind, double eps,
                             const double *C, int T, float2 *out, void *ws, size_t ws_bytes, cudaStream_t s);

int global_cardinal_build(const double *LU, const int32_t *perm, const double *X, int64_t N, int kind,
                          double eps, const double *P, int64_t Nq, void *E, int e_dtype, cudaStream_t s);
size_t cardinal_apply_workspace(int64_t Nq, int64_t N, int T);
int launch_cardinal_apply(const void *E, int64_t Nq, int64_t N, const void *q, int T, int dtype, void *out,
                          void *ws, size_t ws_bytes, cudaStream_t s);

}  // namespace rbfsl
