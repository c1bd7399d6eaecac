// Shared device/host helpers of the CUDA library (not shared with any CPU reference code).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>

#include "rbfsl.h"

namespace rbfsl {

// Thread-local message of the last failure of a stateless call.
void set_error(const std::string &msg);
const char *get_error();

#define RBFSL_CUDA_TRY(expr)                                                               \
    do {                                                                                   \
        cudaError_t _e = (expr);                                                           \
        if (_e != cudaSuccess) {                                                           \
            cudaGetLastError();                                                            \
            ::rbfsl::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));        \
            return RBFSL_ECUDA;                                                            \
        }                                                                                  \
    } while (0)

#define RBFSL_CHECK_ARG(cond, msg)                                                         \
    do {                                                                                   \
        if (!(cond)) {                                                                     \
            ::rbfsl::set_error(msg);                                                       \
            return RBFSL_EINVAL;                                                           \
        }                                                                                  \
    } while (0)

inline int launch_status(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string(what) + ": " + cudaGetErrorString(e));
        return RBFSL_ECUDA;
    }
    return RBFSL_OK;
}

constexpr int kWarp = 32;

// ---------------------------------------------------------------------------------------
// Real orthonormal spherical harmonics of degree <= ell as polynomials of (x, y, z) on S^2
// (the augmentation basis {p_i} of Sec. 2.2). Index l*l + l + m, m = -l..l.
// With z = cos(theta), x + iy = sin(theta) e^{i phi}, Q_l^m(z) = P_l^m(z) / sin^m(theta):
//   Q_m^m = (2m-1)!!, Q_{m+1}^m = (2m+1) z Q_m^m,
//   Q_l^m = a_lm z Q_{l-1}^m - b_lm Q_{l-2}^m, a_lm = (2l-1)/(l-m), b_lm = (l+m-1)/(l-m),
//   Y_l^0 = K_l0 Q_l^0, Y_l^{+m} = K_lm Q_l^m Re(x+iy)^m, Y_l^{-m} = K_lm Q_l^m Im(x+iy)^m,
//   K_lm = sqrt((2 - delta_m0) (2l+1)/(4 pi) (l-m)!/(l+m)!).
// The coefficient tables live in constant memory, filled once per device by sh_tables_init.
constexpr int kMaxL = RBFSL_MAX_SH_DEGREE;
constexpr int kMaxM = (kMaxL + 1) * (kMaxL + 1);

struct ShTables {
    double K[kMaxM];   // indexed l*l + l + m, m >= 0
    double a[kMaxM];
    double b[kMaxM];
    double qmm[kMaxL + 1];
};

int sh_tables_init();  // host: upload the tables to the current device (idempotent)

extern __constant__ ShTables c_sh;

// Evaluate all (ell+1)^2 harmonics at (x, y, z); out[c * stride] for c = l*l + l + m.
template <typename Out>
__device__ __forceinline__ void sh_eval(int ell, double x, double y, double z, Out out) {
    double cm = 1.0, sm = 0.0;
    for (int m = 0; m <= ell; ++m) {
        if (m > 0) {
            const double c2 = cm * x - sm * y;
            const double s2 = cm * y + sm * x;
            cm = c2;
            sm = s2;
        }
        double q2 = 0.0, q1 = 0.0;
        for (int l = m; l <= ell; ++l) {
            const int id = l * l + l + m;
            double q;
            if (l == m) q = c_sh.qmm[m];
            else q = c_sh.a[id] * z * q1 - c_sh.b[id] * q2;
            const double kq = c_sh.K[id] * q;
            if (m == 0) {
                out(id, kq);
            } else {
                out(id, kq * cm);
                out(l * l + l - m, kq * sm);
            }
            q2 = q1;
            q1 = q;
        }
    }
}

// sh_eval spread over a warp, one lane per order m (lanes 0..ell; the others return at once):
// lane m forms (x + iy)^m by sh_eval's recurrence and then the degrees l = m..ell, so every
// value comes from the same operations as in sh_eval while the serial chain is one order long.
template <typename Out>
__device__ __forceinline__ void sh_eval_lanes(int ell, double x, double y, double z, int lane, Out out) {
    if (lane > ell) return;
    const int m = lane;
    double cm = 1.0, sm = 0.0;
    for (int mm = 1; mm <= m; ++mm) {
        const double c2 = cm * x - sm * y;
        const double s2 = cm * y + sm * x;
        cm = c2;
        sm = s2;
    }
    double q2 = 0.0, q1 = 0.0;
    for (int l = m; l <= ell; ++l) {
        const int id = l * l + l + m;
        double q;
        if (l == m) q = c_sh.qmm[m];
        else q = c_sh.a[id] * z * q1 - c_sh.b[id] * q2;
        const double kq = c_sh.K[id] * q;
        if (m == 0) {
            out(id, kq);
        } else {
            out(id, kq * cm);
            out(l * l + l - m, kq * sm);
        }
        q2 = q1;
        q1 = q;
    }
}

// Polyharmonic spline r^p (p odd) from the squared distance: r * (r^2)^((p-1)/2).
__device__ __forceinline__ double phs_from_d2(double d2, int half) {
    double v = sqrt(d2);
    for (int i = 0; i < half; ++i) v *= d2;
    return v;
}

// Squared distance with every operation rounded separately (the k-NN key).
__device__ __forceinline__ double sqdist_rn(double ax, double ay, double az, double bx,
                                            double by, double bz) {
    const double dx = __dsub_rn(ax, bx), dy = __dsub_rn(ay, by), dz = __dsub_rn(az, bz);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// ---------------------------------------------------------------------------------------
// Mixed-precision storage of fields and weights: each value is an unevaluated pair of FP32
// numbers (hi, lo), value = hi + lo with |lo| <= ulp(hi) / 2, stored interleaved (8 bytes per
// value). The gather-dot sum is formed in pair arithmetic with FP32 operations only: exact
// products of the high parts (FMA error term), the cross terms, and Knuth's two-sum into the
// accumulator, so a step adds ~n 2^-48 relative rounding instead of the ~2^-24 of plain FP32.

__device__ __forceinline__ float2 pair_from(double v) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}

// (sh, sl) += w * q for pairs w and q; w.lo * q.lo (below 2^-48 |w q|) is dropped.
__device__ __forceinline__ void pair_fma(float2 w, float2 q, float &sh, float &sl) {
    const float p = w.x * q.x;
    float pe = fmaf(w.x, q.x, -p);
    pe = fmaf(w.x, q.y, pe);
    pe = fmaf(w.y, q.x, pe);
    const float s = sh + p;
    const float bp = s - sh;
    const float e = (sh - (s - bp)) + (p - bp);
    sl = sl + (e + pe);
    sh = s;
}

// The accumulator as a normalised pair (fast two-sum).
__device__ __forceinline__ float2 pair_norm(float sh, float sl) {
    const float hi = sh + sl;
    return make_float2(hi, sl - (hi - sh));
}

// Weight and field element conversions from FP64 results.
template <typename WT>
__device__ __forceinline__ WT wcast(double v);
template <>
__device__ __forceinline__ double wcast<double>(double v) { return v; }
template <>
__device__ __forceinline__ float wcast<float>(double v) { return (float)v; }
template <>
__device__ __forceinline__ float2 wcast<float2>(double v) { return pair_from(v); }

}  // namespace rbfsl
