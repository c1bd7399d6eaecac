// Departure-point tracing (Sec. 3.2, Eq. sl_ode): RK4 backward in time with an orthogonal
// projection onto S^2 at every stage and of the result. One thread per node: the work per
// node is ~200 flops with no reuse, so the kernel is bound by the FP64 pipe (FP64 mode) or
// by the 24+24 bytes per node it moves (mixed mode).
#include "common.cuh"
#include "kernels.cuh"

namespace rbfsl {

template <typename R>
struct Vel {
    int kind;
    R p0, p1, p2, p3;  // rigid: a_x, a_y, a_z, omega; deform: kappa, pi / T_f
    __device__ __forceinline__ void operator()(R x, R y, R z, R t, R &ux, R &uy, R &uz) const {
        if (kind == RBFSL_VEL_RIGID) {
            const R w0 = p3 * p0, w1 = p3 * p1, w2 = p3 * p2;
            ux = w1 * z - w2 * y;
            uy = w2 * x - w0 * z;
            uz = w0 * y - w1 * x;
        } else {
            const R g = R(2) * p0 * y * cos(p1 * t);
            ux = -g * z;
            uy = R(0);
            uz = g * x;
        }
    }
};

template <typename R>
__device__ __forceinline__ void normalize3(R &x, R &y, R &z) {
    const R inv = R(1) / sqrt(x * x + y * y + z * z);
    x *= inv;
    y *= inv;
    z *= inv;
}

// FP64 tracer.
__global__ void trace_rk4_f64(const double *__restrict__ X, int64_t N, Vel<double> u, double t1,
                              double h, double *__restrict__ Xi) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= N) return;
    const double x = X[3 * j], y = X[3 * j + 1], z = X[3 * j + 2];
    double k1x, k1y, k1z, k2x, k2y, k2z, k3x, k3y, k3z, k4x, k4y, k4z;
    u(x, y, z, t1, k1x, k1y, k1z);
    double sx = x + 0.5 * h * k1x, sy = y + 0.5 * h * k1y, sz = z + 0.5 * h * k1z;
    normalize3(sx, sy, sz);
    u(sx, sy, sz, t1 + 0.5 * h, k2x, k2y, k2z);
    sx = x + 0.5 * h * k2x; sy = y + 0.5 * h * k2y; sz = z + 0.5 * h * k2z;
    normalize3(sx, sy, sz);
    u(sx, sy, sz, t1 + 0.5 * h, k3x, k3y, k3z);
    sx = x + h * k3x; sy = y + h * k3y; sz = z + h * k3z;
    normalize3(sx, sy, sz);
    u(sx, sy, sz, t1 + h, k4x, k4y, k4z);
    const double c = h / 6.0;
    double ox = x + c * (k1x + 2.0 * k2x + 2.0 * k3x + k4x);
    double oy = y + c * (k1y + 2.0 * k2y + 2.0 * k3y + k4y);
    double oz = z + c * (k1z + 2.0 * k2z + 2.0 * k3z + k4z);
    normalize3(ox, oy, oz);
    Xi[3 * j] = ox;
    Xi[3 * j + 1] = oy;
    Xi[3 * j + 2] = oz;
}

// Mixed tracer: stages in FP32; the displacement d = (h/6)(k1 + 2k2 + 2k3 + k4) is added to
// the FP64 node and projected in FP64, so the FP32 rounding scales with |d|, not with |x|.
__global__ void trace_rk4_mixed(const double *__restrict__ X, int64_t N, Vel<float> u, float t1,
                                float h, double *__restrict__ Xi) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= N) return;
    const double xd = X[3 * j], yd = X[3 * j + 1], zd = X[3 * j + 2];
    const float x = (float)xd, y = (float)yd, z = (float)zd;
    float k1x, k1y, k1z, k2x, k2y, k2z, k3x, k3y, k3z, k4x, k4y, k4z;
    u(x, y, z, t1, k1x, k1y, k1z);
    float sx = x + 0.5f * h * k1x, sy = y + 0.5f * h * k1y, sz = z + 0.5f * h * k1z;
    normalize3(sx, sy, sz);
    u(sx, sy, sz, t1 + 0.5f * h, k2x, k2y, k2z);
    sx = x + 0.5f * h * k2x; sy = y + 0.5f * h * k2y; sz = z + 0.5f * h * k2z;
    normalize3(sx, sy, sz);
    u(sx, sy, sz, t1 + 0.5f * h, k3x, k3y, k3z);
    sx = x + h * k3x; sy = y + h * k3y; sz = z + h * k3z;
    normalize3(sx, sy, sz);
    u(sx, sy, sz, t1 + h, k4x, k4y, k4z);
    const float c = h / 6.0f;
    double ox = xd + (double)(c * (k1x + 2.0f * k2x + 2.0f * k3x + k4x));
    double oy = yd + (double)(c * (k1y + 2.0f * k2y + 2.0f * k3y + k4y));
    double oz = zd + (double)(c * (k1z + 2.0f * k2z + 2.0f * k3z + k4z));
    normalize3(ox, oy, oz);
    Xi[3 * j] = ox;
    Xi[3 * j + 1] = oy;
    Xi[3 * j + 2] = oz;
}

int launch_trace(const double *x, int64_t N, int vel_kind, const double *prm, double t1,
                 double dt, int precision, double *xi, cudaStream_t s) {
    if (N == 0) return RBFSL_OK;
    const int threads = 256;
    const unsigned blocks = (unsigned)((N + threads - 1) / threads);
    const double pi = 3.14159265358979323846;
    if (precision == RBFSL_FP64) {
        Vel<double> u{vel_kind, prm[0], prm[1], 0.0, 0.0};
        if (vel_kind == RBFSL_VEL_RIGID) { u.p2 = prm[2]; u.p3 = prm[3]; }
        else u.p1 = pi / prm[1];
        trace_rk4_f64<<<blocks, threads, 0, s>>>(x, N, u, t1, -dt, xi);
    } else {
        Vel<float> u{vel_kind, (float)prm[0], (float)prm[1], 0.f, 0.f};
        if (vel_kind == RBFSL_VEL_RIGID) { u.p2 = (float)prm[2]; u.p3 = (float)prm[3]; }
        else u.p1 = (float)(pi / prm[1]);
        // The deformation's time argument enters through cos(pi t / T_f); FP32 t1 is exact
        // to ~1e-7 relative, far below the trajectory error of a step.
        trace_rk4_mixed<<<blocks, threads, 0, s>>>(x, N, u, (float)t1, (float)-dt, xi);
    }
    return launch_status("trace_rk4");
}

}  // namespace rbfsl

extern "C" int rbfsl_trace_rk4(const double *x, int64_t N, int vel_kind, const double *vel_params,
                               double t1, double dt, int precision, double *xi, void *stream) {
    using namespace rbfsl;
    RBFSL_CHECK_ARG(N >= 0, "trace_rk4: N < 0");
    RBFSL_CHECK_ARG(N == 0 || (x && xi && vel_params), "trace_rk4: null pointer");
    RBFSL_CHECK_ARG(vel_kind == RBFSL_VEL_RIGID || vel_kind == RBFSL_VEL_DEFORM_Y2,
                    "trace_rk4: unknown velocity kind");
    RBFSL_CHECK_ARG(precision == RBFSL_FP64 || precision == RBFSL_MIXED,
                    "trace_rk4: unknown precision");
    return launch_trace(x, N, vel_kind, vel_params, t1, dt, precision, xi, (cudaStream_t)stream);
}
