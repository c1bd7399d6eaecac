// Departure-point tracing (Sec. 3.2, Eq. sl_ode): RK4 backward in time with an orthogonal
// projection onto S^2 at every stage and of the result. One thread per node: the work per
// node is ~200 flops with no reuse, so the kernel is bound by the FP64 pipe (FP64 mode) or
// by the 24+24 bytes per node it moves (mixed mode, where ~50 of the flops are FP64).
#include "common.cuh"
#include "kernels.cuh"
#include "device_ops.cuh"

namespace rbfsl {

// FP64 tracer.
__global__ void trace_rk4_f64(const double *__restrict__ X, int64_t N, Vel<double> u, double t1,
                              double h, double *__restrict__ Xi) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= N) return;
    rk4_point_f64(u, X[3 * j], X[3 * j + 1], X[3 * j + 2], t1, h, Xi[3 * j], Xi[3 * j + 1], Xi[3 * j + 2]);
}

// Mixed tracer: FP32 stage increments, FP64 node velocity, final add and projection.
__global__ void trace_rk4_mixed(const double *__restrict__ X, int64_t N, Vel<double> u, double t1,
                                double h, double *__restrict__ Xi) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= N) return;
    rk4_point_mixed(u, X[3 * j], X[3 * j + 1], X[3 * j + 2], t1, h, Xi[3 * j], Xi[3 * j + 1], Xi[3 * j + 2]);
}

// Fehlberg fifth-order tracers (the paper's final integrator), FP64 and mixed.
__global__ void trace_rk5_f64(const double *__restrict__ X, int64_t N, Vel<double> u, double t1, double h,
                              double *__restrict__ Xi) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= N) return;
    rk5_point_f64(u, X[3 * j], X[3 * j + 1], X[3 * j + 2], t1, h, Xi[3 * j], Xi[3 * j + 1], Xi[3 * j + 2]);
}

__global__ void trace_rk5_mixed(const double *__restrict__ X, int64_t N, Vel<double> u, double t1, double h,
                                double *__restrict__ Xi) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= N) return;
    rk5_point_mixed(u, X[3 * j], X[3 * j + 1], X[3 * j + 2], t1, h, Xi[3 * j], Xi[3 * j + 1], Xi[3 * j + 2]);
}

int launch_trace_order(const double *x, int64_t N, int vel_kind, const double *prm, double t1, double dt,
                       int precision, int order, double *xi, cudaStream_t s) {
    if (order != 5) return launch_trace(x, N, vel_kind, prm, t1, dt, precision, xi, s);
    if (N == 0) return RBFSL_OK;
    const unsigned blocks = (unsigned)((N + 255) / 256);
    if (precision == RBFSL_FP64) trace_rk5_f64<<<blocks, 256, 0, s>>>(x, N, make_vel64(vel_kind, prm), t1, -dt, xi);
    else trace_rk5_mixed<<<blocks, 256, 0, s>>>(x, N, make_vel64(vel_kind, prm), t1, -dt, xi);
    return launch_status("trace_rk5");
}

int launch_trace(const double *x, int64_t N, int vel_kind, const double *prm, double t1,
                 double dt, int precision, double *xi, cudaStream_t s) {
    if (N == 0) return RBFSL_OK;
    const int threads = 256;
    const unsigned blocks = (unsigned)((N + threads - 1) / threads);
    if (precision == RBFSL_FP64) {
        trace_rk4_f64<<<blocks, threads, 0, s>>>(x, N, make_vel64(vel_kind, prm), t1, -dt, xi);
    } else {
        trace_rk4_mixed<<<blocks, threads, 0, s>>>(x, N, make_vel64(vel_kind, prm), t1, -dt, xi);
    }
    return launch_status("trace_rk4");
}

}  // namespace rbfsl

extern "C" int rbfsl_trace_rk4(const double *x, int64_t N, int vel_kind, const double *vel_params,
                               double t1, double dt, int precision, double *xi, void *stream) {
    using namespace rbfsl;
    RBFSL_CHECK_ARG(N >= 0, "trace_rk4: N < 0");
    RBFSL_CHECK_ARG(N == 0 || (x && xi && vel_params), "trace_rk4: null pointer");
    RBFSL_CHECK_ARG(vel_kind == RBFSL_VEL_RIGID || vel_kind == RBFSL_VEL_DEFORM_Y2 || vel_kind == RBFSL_VEL_NL,
                    "trace_rk4: unknown velocity kind");
    RBFSL_CHECK_ARG(precision == RBFSL_FP64 || precision == RBFSL_MIXED,
                    "trace_rk4: unknown precision");
    return launch_trace(x, N, vel_kind, vel_params, t1, dt, precision, xi, (cudaStream_t)stream);
}

extern "C" int rbfsl_trace_rk5(const double *x, int64_t N, int vel_kind, const double *vel_params,
                               double t1, double dt, int precision, double *xi, void *stream) {
    using namespace rbfsl;
    RBFSL_CHECK_ARG(N >= 0, "trace_rk5: N < 0");
    RBFSL_CHECK_ARG(N == 0 || (x && xi && vel_params), "trace_rk5: null pointer");
    RBFSL_CHECK_ARG(vel_kind == RBFSL_VEL_RIGID || vel_kind == RBFSL_VEL_DEFORM_Y2 || vel_kind == RBFSL_VEL_NL,
                    "trace_rk5: unknown velocity kind");
    RBFSL_CHECK_ARG(precision == RBFSL_FP64 || precision == RBFSL_MIXED, "trace_rk5: unknown precision");
    return launch_trace_order(x, N, vel_kind, vel_params, t1, dt, precision, 5, xi, (cudaStream_t)stream);
}
