// Per-point device operations shared by the single-problem kernels and the batched
// persistent kernel, so that a problem gives bit-identical results alone or in a batch.
#pragma once

#include "common.cuh"
#include "kernels.cuh"

namespace rbfsl {

template <typename R>
struct Vel {
    int kind;
    R p0, p1, p2, p3;  // rigid: a_x, a_y, a_z, omega; deform / NL: kappa, pi / T_f
    __device__ __forceinline__ void operator()(R x, R y, R z, R t, R &ux, R &uy, R &uz) const {
        if (kind == RBFSL_VEL_RIGID) {
            const R w0 = p3 * p0, w1 = p3 * p1, w2 = p3 * p2;
            ux = w1 * z - w2 * y;
            uy = w2 * x - w0 * z;
            uz = w0 * y - w1 * x;
        } else if (kind == RBFSL_VEL_DEFORM_Y2) {
            const R g = R(2) * p0 * y * cos(p1 * t);
            ux = -g * z;
            uy = R(0);
            uz = g * x;
        } else {
            // the paper's deformational flow (Sec. 4.2) as u = x cross grad(psi) with
            // psi = kappa cos(pi t/T) b^2 - (2 pi / T) z, b = y cos c - x sin c, c = 2 pi t / T:
            // grad(psi) = (-2 k b sin c, 2 k b cos c, -a), a polynomial field, smooth at the poles
            const R c = R(2) * p1 * t, cc = cos(c), sc = sin(c);
            const R k2 = R(2) * p0 * cos(p1 * t), a = R(2) * p1;
            const R b = y * cc - x * sc, q = x * cc + y * sc;
            const R kbz = k2 * b * z;
            ux = -a * y - kbz * cc;
            uy = a * x - kbz * sc;
            uz = k2 * b * q;
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


// One departure point, FP64 (Sec. 3.2, Eq. sl_ode): classical RK4 backward (h = -dt) with an
// orthogonal projection onto S^2 of every stage point and of the result.
__device__ __forceinline__ void rk4_point_f64(const Vel<double> &u, double x, double y, double z,
                                              double t1, double h, double &ox, double &oy,
                                              double &oz) {
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
    ox = x + c * (k1x + 2.0 * k2x + 2.0 * k3x + k4x);
    oy = y + c * (k1y + 2.0 * k2y + 2.0 * k3y + k4y);
    oz = z + c * (k1z + 2.0 * k2z + 2.0 * k3z + k4z);
    normalize3(ox, oy, oz);
}

// Mixed: increment form. The node's own velocity U0 = u(x, t1), the stage displacements' FP64
// parts and the final add and projection are FP64 (a few dozen flops per node); the RK4 stages
// are FP32 increments from the node. A stage point is x + e with e = N(x + a) - x formed in
// FP32 from the stage displacement a (|a| ~ |u| dt), and its velocity is U0 + D with
// D = u(x + e, t_s) - u(x, t1) formed in FP32 from e and the FP64 difference of the time
// factors, so every FP32 rounding error scales with an increment, not with |x| or |u|.
// Unit nodes are assumed (|x| = 1 to FP64 rounding).

// e = N(x + a) - x for unit x: r = |x + a| = sqrt(1 + 2 x.a + a.a),
// e = (a - x (r - 1)) / r with r - 1 = (2 x.a + a.a) / (r + 1).
__device__ __forceinline__ void stage_offset(float x, float y, float z, float ax, float ay, float az,
                                             float &ex, float &ey, float &ez) {
    const float g = 2.0f * (x * ax + y * ay + z * az) + (ax * ax + ay * ay + az * az);
    const float r = sqrtf(1.0f + g);
    const float rm1 = g / (r + 1.0f);
    const float ir = 1.0f / r;
    ex = (ax - x * rm1) * ir;
    ey = (ay - y * rm1) * ir;
    ez = (az - z * rm1) * ir;
}

// D = u(x + e, t_s) - u(x, t1). Rigid rotation: omega x e. Deformation u = c(t) g(x) with
// g = 2 kappa y (-z, 0, x): D = c_s [g(x + e) - g(x)] + (c_s - c_1) g(x), the bracket expanded
// so that it is formed from products with e only.
__device__ __forceinline__ void vel_increment(int kind, float w0, float w1, float w2, float k2,
                                              float cs, float dc, float x, float y, float z,
                                              float ex, float ey, float ez, float &dx, float &dy,
                                              float &dz) {
    if (kind == RBFSL_VEL_RIGID) {
        dx = w1 * ez - w2 * ey;
        dy = w2 * ex - w0 * ez;
        dz = w0 * ey - w1 * ex;
    } else {
        const float gx = -k2 * ((y * ez + ey * z) + ey * ez);  // g(x + e) - g(x), x-component
        const float gz = k2 * ((y * ex + ey * x) + ey * ex);
        const float bx = -k2 * y * z, bz = k2 * y * x;         // g(x)
        dx = cs * gx + dc * bx;
        dy = 0.0f;
        dz = cs * gz + dc * bz;
    }
}

__device__ __forceinline__ void rk4_point_mixed(const Vel<double> &u, double xd, double yd, double zd,
                                                double t1, double h, double &ox, double &oy,
                                                double &oz) {
    if (u.kind == RBFSL_VEL_NL) {  // no FP32 increment form for this field: stages in FP64
        rk4_point_f64(u, xd, yd, zd, t1, h, ox, oy, oz);
        return;
    }
    double U0x, U0y, U0z;
    u(xd, yd, zd, t1, U0x, U0y, U0z);
    // time factors of the deformation at t1, t1 + h/2, t1 + h (FP64); unused for rigid rotation
    float cs2 = 0.f, dc2 = 0.f, cs4 = 0.f, dc4 = 0.f, k2 = 0.f, w0 = 0.f, w1 = 0.f, w2 = 0.f;
    if (u.kind == RBFSL_VEL_RIGID) {
        w0 = (float)(u.p3 * u.p0); w1 = (float)(u.p3 * u.p1); w2 = (float)(u.p3 * u.p2);
    } else {
        const double c1 = cos(u.p1 * t1), c2 = cos(u.p1 * (t1 + 0.5 * h)), c4 = cos(u.p1 * (t1 + h));
        cs2 = (float)c2; dc2 = (float)(c2 - c1);
        cs4 = (float)c4; dc4 = (float)(c4 - c1);
        k2 = (float)(2.0 * u.p0);
    }
    const float x = (float)xd, y = (float)yd, z = (float)zd;
    const float hf = (float)h, hh = (float)(0.5 * h);
    // stage 2: a2 = (h/2) U0
    const float a2x = (float)(0.5 * h * U0x), a2y = (float)(0.5 * h * U0y), a2z = (float)(0.5 * h * U0z);
    float ex, ey, ez, d2x, d2y, d2z, d3x, d3y, d3z, d4x, d4y, d4z;
    stage_offset(x, y, z, a2x, a2y, a2z, ex, ey, ez);
    vel_increment(u.kind, w0, w1, w2, k2, cs2, dc2, x, y, z, ex, ey, ez, d2x, d2y, d2z);
    // stage 3: a3 = (h/2)(U0 + D2)
    stage_offset(x, y, z, a2x + hh * d2x, a2y + hh * d2y, a2z + hh * d2z, ex, ey, ez);
    vel_increment(u.kind, w0, w1, w2, k2, cs2, dc2, x, y, z, ex, ey, ez, d3x, d3y, d3z);
    // stage 4: a4 = h (U0 + D3)
    const float a4x = (float)(h * U0x), a4y = (float)(h * U0y), a4z = (float)(h * U0z);
    stage_offset(x, y, z, a4x + hf * d3x, a4y + hf * d3y, a4z + hf * d3z, ex, ey, ez);
    vel_increment(u.kind, w0, w1, w2, k2, cs4, dc4, x, y, z, ex, ey, ez, d4x, d4y, d4z);
    // d = (h/6)(k1 + 2 k2 + 2 k3 + k4) = h U0 + (h/6)(2 D2 + 2 D3 + D4)
    const float c6 = (float)(h / 6.0);
    const float ix = c6 * (2.0f * (d2x + d3x) + d4x), iy = c6 * (2.0f * (d2y + d3y) + d4y),
                iz = c6 * (2.0f * (d2z + d3z) + d4z);
    ox = xd + (h * U0x + (double)ix);
    oy = yd + (h * U0y + (double)iy);
    oz = zd + (h * U0z + (double)iz);
    normalize3(ox, oy, oz);
}

// Fehlberg's fifth-order formula (Sec. 3.2, the paper's final integrator): six stages with
// nodes c, coupling coefficients a (row i: stage i) and fifth-order weights b, as published.
struct Rk5 {
    __host__ __device__ static constexpr double c(int i) {
        constexpr double v[6] = {0.0, 1.0 / 4.0, 3.0 / 8.0, 12.0 / 13.0, 1.0, 1.0 / 2.0};
        return v[i];
    }
    __host__ __device__ static constexpr double a(int i, int q) {
        constexpr double v[6][5] = {{0, 0, 0, 0, 0},
                                    {1.0 / 4.0, 0, 0, 0, 0},
                                    {3.0 / 32.0, 9.0 / 32.0, 0, 0, 0},
                                    {1932.0 / 2197.0, -7200.0 / 2197.0, 7296.0 / 2197.0, 0, 0},
                                    {439.0 / 216.0, -8.0, 3680.0 / 513.0, -845.0 / 4104.0, 0},
                                    {-8.0 / 27.0, 2.0, -3544.0 / 2565.0, 1859.0 / 4104.0, -11.0 / 40.0}};
        return v[i][q];
    }
    __host__ __device__ static constexpr double b(int i) {
        constexpr double v[6] = {16.0 / 135.0, 0.0, 6656.0 / 12825.0, 28561.0 / 56430.0, -9.0 / 50.0, 2.0 / 55.0};
        return v[i];
    }
};

// One departure point, FP64, Fehlberg's formula backward (h = -dt): stage point i is
// x + h sum_j a_ij k_j projected onto S^2, evaluated at t1 + c_i h; the result is projected too.
__device__ __forceinline__ void rk5_point_f64(const Vel<double> &u, double x, double y, double z, double t1,
                                              double h, double &ox, double &oy, double &oz) {
    double kx[6], ky[6], kz[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        double sx = x, sy = y, sz = z;
        if (i > 0) {
            double ax = 0.0, ay = 0.0, az = 0.0;
#pragma unroll
            for (int q = 0; q < i; ++q) {
                ax = ax + Rk5::a(i, q) * kx[q];
                ay = ay + Rk5::a(i, q) * ky[q];
                az = az + Rk5::a(i, q) * kz[q];
            }
            sx = x + h * ax;
            sy = y + h * ay;
            sz = z + h * az;
            normalize3(sx, sy, sz);
        }
        u(sx, sy, sz, t1 + Rk5::c(i) * h, kx[i], ky[i], kz[i]);
    }
    double dx = 0.0, dy = 0.0, dz = 0.0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        dx = dx + Rk5::b(i) * kx[i];
        dy = dy + Rk5::b(i) * ky[i];
        dz = dz + Rk5::b(i) * kz[i];
    }
    ox = x + h * dx;
    oy = y + h * dy;
    oz = z + h * dz;
    normalize3(ox, oy, oz);
}

// Mixed, increment form as rk4_point_mixed: k_i = U0 + D_i with the node's velocity U0 in FP64
// and the stage increments D_i in FP32; since sum_j a_ij = c_i and sum_i b_i = 1, stage i's
// displacement is c_i h U0 + h sum_j a_ij D_j and the step's is h U0 + h sum_i b_i D_i.
__device__ __forceinline__ void rk5_point_mixed(const Vel<double> &u, double xd, double yd, double zd,
                                                double t1, double h, double &ox, double &oy, double &oz) {
    if (u.kind == RBFSL_VEL_NL) {  // no FP32 increment form for this field: stages in FP64
        rk5_point_f64(u, xd, yd, zd, t1, h, ox, oy, oz);
        return;
    }
    double U0x, U0y, U0z;
    u(xd, yd, zd, t1, U0x, U0y, U0z);
    float w0 = 0.f, w1 = 0.f, w2 = 0.f, k2 = 0.f;
    double c1 = 0.0;
    if (u.kind == RBFSL_VEL_RIGID) {
        w0 = (float)(u.p3 * u.p0); w1 = (float)(u.p3 * u.p1); w2 = (float)(u.p3 * u.p2);
    } else {
        c1 = cos(u.p1 * t1);
        k2 = (float)(2.0 * u.p0);
    }
    const float x = (float)xd, y = (float)yd, z = (float)zd;
    const float hf = (float)h;
    float Dx[6], Dy[6], Dz[6];
    Dx[0] = Dy[0] = Dz[0] = 0.f;
#pragma unroll
    for (int i = 1; i < 6; ++i) {
        float sx = 0.f, sy = 0.f, sz = 0.f;
#pragma unroll
        for (int q = 1; q < i; ++q) {
            sx = sx + (float)Rk5::a(i, q) * Dx[q];
            sy = sy + (float)Rk5::a(i, q) * Dy[q];
            sz = sz + (float)Rk5::a(i, q) * Dz[q];
        }
        const double ch = Rk5::c(i) * h;
        const float ax = (float)(ch * U0x) + hf * sx, ay = (float)(ch * U0y) + hf * sy,
                    az = (float)(ch * U0z) + hf * sz;
        float ex, ey, ez;
        stage_offset(x, y, z, ax, ay, az, ex, ey, ez);
        float cs = 0.f, dc = 0.f;
        if (u.kind != RBFSL_VEL_RIGID) {
            const double ci = cos(u.p1 * (t1 + ch));
            cs = (float)ci;
            dc = (float)(ci - c1);
        }
        vel_increment(u.kind, w0, w1, w2, k2, cs, dc, x, y, z, ex, ey, ez, Dx[i], Dy[i], Dz[i]);
    }
    float ix = 0.f, iy = 0.f, iz = 0.f;
#pragma unroll
    for (int i = 1; i < 6; ++i) {
        ix = ix + (float)Rk5::b(i) * Dx[i];
        iy = iy + (float)Rk5::b(i) * Dy[i];
        iz = iz + (float)Rk5::b(i) * Dz[i];
    }
    ox = xd + (h * U0x + (double)(hf * ix));
    oy = yd + (h * U0y + (double)(hf * iy));
    oz = zd + (h * U0z + (double)(hf * iz));
    normalize3(ox, oy, oz);
}

// Kernel-ready velocity parameters (deformation: p1 = pi / T_f).
inline Vel<double> make_vel64(int kind, const double *prm) {
    const double pi = 3.14159265358979323846;
    Vel<double> u{kind, prm[0], prm[1], 0.0, 0.0};
    if (kind == RBFSL_VEL_RIGID) { u.p2 = prm[2]; u.p3 = prm[3]; }
    else u.p1 = pi / prm[1];
    return u;
}

// Order of the k-NN keys (d^2, index). Squared distances are non-negative (and the padding is
// +infinity), and for such doubles the IEEE bit patterns read as 64-bit integers order exactly as
// the values, so the comparison runs on the integer units instead of the FP64 pipe.
__device__ __forceinline__ bool key_less(long long da, int ia, long long db, int ib) {
    return da < db || (da == db && ia < ib);
}

// k nearest nodes of (qx, qy, qz) by one warp. bd/bi: the warp's candidate buffers (cap
// entries, cap a power of two >= k), cnt: one shared int. On success bi[0..k) holds the node
// indices ascending by (d2, index) and the function returns true; false if no radius in 40
// rescalings brackets between k and cap candidates.
__device__ __forceinline__ bool knn_warp(const KnnGrid &g, double qx, double qy, double qz, int k,
                                         int cap, double *bd, int *bi, int *cnt, int lane) {
    double r2 = g.r2_per_k * k;
    const double target = 1.3 * k;
    long long r2b;  // r2 as key bits
    int total = 0;
    bool ok = false;
    for (int iter = 0; iter < 40; ++iter) {
        if (lane == 0) *cnt = 0;
        __syncwarp();
        const double rb = sqrt(r2) * (1.0 + 1e-9) + 1e-15;
        r2b = __double_as_longlong(r2);
        grid_ball_foreach(g, qx, qy, qz, rb, lane, [&](int p) {
            const double d2 = sqdist_rn(qx, qy, qz, g.sx[p], g.sy[p], g.sz[p]);
            if (__double_as_longlong(d2) <= r2b) {  // d2 <= r2, both non-negative
                const int slot = atomicAdd(cnt, 1);
                if (slot < cap) {
                    bd[slot] = d2;
                    bi[slot] = g.sid[p];
                }
            }
        });
        __syncwarp();
        total = *cnt;
        __syncwarp();
        if (total >= k && total <= cap) {
            ok = true;
            break;
        }
        // Rescale the radius towards ~1.3 k candidates (count grows like r^2).
        double f = total > 0 ? target / (double)total : 4.0;
        f = f < 0.25 ? 0.25 : (f > 4.0 ? 4.0 : f);
        if (total < k && f < 1.05) f = 1.05;
        if (total > cap && f > 0.95) f = 0.95;
        r2 *= f;
    }
    if (!ok) return false;
    // Bitonic sort of the candidates by (d2, index), padded to a power of two.
    int P = 1;
    while (P < total) P <<= 1;
    for (int i = total + lane; i < P; i += kWarp) {
        bd[i] = INFINITY;
        bi[i] = 0x7fffffff;
    }
    __syncwarp();
    for (int len = 2; len <= P; len <<= 1) {
        for (int stride = len >> 1; stride > 0; stride >>= 1) {
            for (int i = lane; i < P; i += kWarp) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool up = (i & len) == 0;
                    const double di = bd[i], dj = bd[j];
                    const int ii = bi[i], ij = bi[j];
                    if (key_less(__double_as_longlong(dj), ij, __double_as_longlong(di), ii) == up) {
                        bd[i] = dj; bi[i] = ij;
                        bd[j] = di; bi[j] = ii;
                    }
                }
            }
            __syncwarp();
        }
    }
    return true;
}

__host__ __device__ inline int knn_cap(int k) {
    int cap = 64;
    while (cap < 3 * k) cap <<= 1;
    return cap;
}

// ---- Weights by symmetric indefinite factorisation. The saddle-point matrix
// A~ = [[A, P], [P^T, 0]] of Eq. rbf_poly_linsys is symmetric, so A~ w~ = b is solved by
// P A~ P^T = L D L^T with Bunch-Kaufman pivoting (1 x 1 and 2 x 2 pivots, symmetric
// interchanges): m^3 / 6 FMAs instead of elimination's m^3 / 3, on the lower triangle only.
// The PHS block has a zero diagonal, so the first pivots are 2 x 2.
//
// Blocked form (delayed trailing updates, LAPACK's panel scheme for the symmetric indefinite
// factorisation): the pivot columns of a panel of up to kPanel columns are updated on the fly
// from the panel's L columns and its W = L D columns (the pivot columns before scaling), and the
// trailing triangle is updated once per panel instead of once per pivot step.
//
// Shared region of one point (doubles): the packed lower triangle (element (i, j), j <= i, at
// i (i + 1) / 2 + j; rows of the trailing triangle hold entries not yet updated by the open
// panel), the right-hand side / solution y (m), the panel's W columns (kPanel x m), the stencil
// coordinates (3 n; afterwards the updated columns k and r, 2 m, and the weights on return), 16
// 64-bit per-warp maxima, then ints: the position -> stencil-row map (m), the pivot kinds (m) and
// eight words of step state.
constexpr int kPanel = 4;
__host__ __device__ inline int ldl_doubles(int n, int m) {
    const int c = 3 * n > 2 * m ? 3 * n : 2 * m;
    return m * (m + 1) / 2 + (1 + kPanel) * m + c + 16 + (2 * m + 8 + 1) / 2;
}
// Shared-memory bytes of one point up to which one warp takes a point (m <~ 45).
constexpr int kWeightsSmallBytes = 12 * 1024;

__device__ __forceinline__ int tri(int i) { return i * (i + 1) / 2; }

// Row of flat index e in a lower triangle of rows of 1, 2, 3, ... elements.
__device__ __forceinline__ int tri_row(int e) {
    int r = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
    if (tri(r) > e) --r;
    if (tri(r + 1) <= e) ++r;
    return r;
}

// |v| / 2^s as an FP32 number, from the bits of the double v with integer operations only
// (the exponent rebased by s, the fraction truncated to 23 bits; 0 below FP32's normal range,
// +inf above it, NaN for NaN). Used for the pivot tests, so that the deciding warp's serial chain
// does not wait on the FP64 pipe, which the other points' trailing updates keep busy.
__device__ __forceinline__ float mag_f32(long long bits, int s) {
    const int e = (int)((bits >> 52) & 0x7ff);
    if (e == 0x7ff) return __int_as_float((bits & 0xfffffffffffffLL) ? 0x7fc00000 : 0x7f800000);
    if (e == 0) return 0.0f;
    const int fe = e - s - 1023 + 127;
    if (fe <= 0) return 0.0f;
    if (fe >= 255) return __int_as_float(0x7f800000);
    return __int_as_float((fe << 23) | (int)((bits >> 29) & 0x7fffff));
}

// Unbiased exponent of a finite nonzero double (0 for zero and subnormals).
__device__ __forceinline__ int exp_of(long long bits) {
    const int e = (int)((bits >> 52) & 0x7ff);
    return e == 0 ? 0 : e - 1023;
}

// Warp-wide maximum of non-negative 64-bit keys (the bit patterns of |a|) with the smallest
// row attaining it: three redux.sync reductions on the 32-bit halves and the row, instead of
// five rounds of 64-bit shuffles (10% of the DIRECT weights launch at m = 109). Lanes without a candidate pass key 0 and row m (a real zero
// entry then wins by its smaller row; a column with no rows gives key 0 and row m).
__device__ __forceinline__ void warp_max_key_row(long long &key, int &row) {
    const unsigned hi = (unsigned)((unsigned long long)key >> 32), lo = (unsigned)key;
    const unsigned mhi = __reduce_max_sync(0xffffffffu, hi);
    const unsigned mlo = __reduce_max_sync(0xffffffffu, hi == mhi ? lo : 0u);
    const bool top = hi == mhi && lo == mlo;
    row = (int)__reduce_min_sync(0xffffffffu, top ? (unsigned)row : 0xffffffffu);
    key = (long long)(((unsigned long long)mhi << 32) | mlo);
}

__device__ __forceinline__ long long warp_max_key(long long key) {
    const unsigned hi = (unsigned)((unsigned long long)key >> 32), lo = (unsigned)key;
    const unsigned mhi = __reduce_max_sync(0xffffffffu, hi);
    const unsigned mlo = __reduce_max_sync(0xffffffffu, hi == mhi ? lo : 0u);
    return (long long)(((unsigned long long)mhi << 32) | mlo);
}

// 1 / d by Newton-Raphson iteration r <- r + r (1 - d r) (the classical reciprocal iteration,
// each step doubling the correct bits) from an FP32 seed: the reciprocal of d's leading 24
// significand bits (rcp.approx.f32, ~23 correct bits) with d's exponent negated, then two
// FMA-based steps in FP64, ~1 ulp. Zero, subnormal, huge or non-finite d take the division.
__device__ __forceinline__ double recip_nr(double d) {
    const long long b = __double_as_longlong(d);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e < 2 || e > 2044) return 1.0 / d;
    const float mf = __int_as_float(0x3f800000 | (int)((b >> 29) & 0x7fffff));  // in [1, 2)
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(mf));                     // in (0.5, 1]
    const int fb = __float_as_int(rf);
    const long long re = (long long)(((fb >> 23) & 0xff) - 127) + 1023 - (e - 1023);
    double r = __longlong_as_double((b & (long long)0x8000000000000000ULL) | (re << 52) |
                                    ((long long)(fb & 0x7fffff) << 29));
    double t = fma(-d, r, 1.0);
    r = fma(r, t, r);
    t = fma(-d, r, 1.0);
    return fma(r, t, r);
}

// Weights of one point by a group of NW warps (thread t of the group). Assembles the packed
// lower triangle of A~ and b (Eqs. rbf_poly, rbf_poly_linsys), factorises with Bunch-Kaufman
// pivoting (alpha = (1 + sqrt 17) / 8; column maximum lambda at row r (smaller row on a tie),
// row maximum sigma of r: 1 x 1 pivot k if |a_kk| >= alpha lambda or |a_kk| sigma >=
// alpha lambda^2, 1 x 1 pivot r if |a_rr| >= alpha sigma, else the 2 x 2 pivot (k, r)),
// applying the forward substitution to b as it goes, then solves D and L^T. Warp 0 takes the
// pivot decisions, interchanges and multipliers; all warps update the trailing triangle, each
// element by the same FMAs whichever thread takes it, so any NW gives the same bits. The
// decision's serial chain keeps off the FP64 pipe where it can (that pipe is the SM's
// bottleneck and queues the other points' updates): the three pivot tests compare FP32 copies
// of the magnitudes rescaled by lambda's exponent (alpha is then honoured to ~1e-7, which the
// method's stability bound does not notice), and pivots are inverted by recip_nr. Each diagonal
// block is overwritten by its inverse once its multipliers are formed, so the final D solve
// multiplies instead of dividing. Returns
// RBFSL_OK with the weights w (n doubles, stencil order) in `out` (valid for warp 0),
// RBFSL_EKNN for a stencil index < 0, RBFSL_ESINGULAR for two coincident stencil nodes or a
// zero or non-finite pivot.
template <int NW>
__device__ __forceinline__ int weights_point_ldl(double *__restrict__ R, const double *__restrict__ X,
                                                 const int32_t *__restrict__ stencil, int n, int m, int ell,
                                                 int half, double px, double py, double pz, int t,
                                                 double *&out) {
    constexpr int GT = NW * kWarp;
    constexpr double kAlpha = 0.6403882032022076;  // (1 + sqrt(17)) / 8
    const int warp = t >> 5, lane = t & 31;
    const int M = m - n;
    const int cdoubles = 3 * n > 2 * m ? 3 * n : 2 * m;
    double *P = R, *y = P + tri(m), *U = y + m;   // U: kPanel columns of W = L D, m each
    double *cx = U + kPanel * m, *cy = cx + n, *cz = cy + n;
    double *wk = cx, *wr = cx + m;                // after the assembly: the updated columns k, r
    long long *slot = reinterpret_cast<long long *>(cx + cdoubles);  // per-warp maxima
    int *perm = reinterpret_cast<int *>(slot + 16), *ptype = perm + m, *st = ptype + m;
    // st[0]: error flag, st[1]: pivot size of the current step, st[2]: close the panel first
    auto gsync = [] {
        if (NW == 1) __syncwarp(); else __syncthreads();
    };
    out = cx;
    if (t == 0) st[0] = 0;
    gsync();
    for (int j = t; j < n; j += GT) {
        const int64_t s = stencil[j];
        if (s < 0) { st[0] = 1; continue; }  // a failed neighbour search leaves -1
        cx[j] = X[3 * s];
        cy[j] = X[3 * s + 1];
        cz[j] = X[3 * s + 2];
    }
    gsync();
    if (st[0]) return RBFSL_EKNN;

    // ---- assembly of the lower triangle; the n(n-1)/2 pairs folded into rows of n-1
    const int P2 = n * (n - 1) / 2;
    for (int p = t; p < P2; p += GT) {
        const int f = p / (n - 1), e = p - f * (n - 1);
        int r, c;
        if (e < n - 1 - f) { r = f + 1 + e; c = f; } else { r = e + 1; c = n - 1 - f; }
        const double dx = cx[r] - cx[c], dy = cy[r] - cy[c], dz = cz[r] - cz[c];
        const double d2 = fma(dz, dz, fma(dy, dy, dx * dx));
        if (d2 == 0.0) st[0] = 2;  // two coincident nodes: two equal rows, singular
        double v = sqrt(d2), q = d2;  // r^p = r (r^2)^half, the power by repeated squaring
        for (int h = half; h > 0; h >>= 1) {
            if (h & 1) v *= q;
            if (h > 1) q *= q;
        }
        P[tri(r) + c] = v;
    }
    for (int j = t; j < n; j += GT) {
        P[tri(j) + j] = 0.0;
        sh_eval(ell, cx[j], cy[j], cz[j], [&](int c, double v) { P[tri(n + c) + j] = v; });
        const double dx = px - cx[j], dy = py - cy[j], dz = pz - cz[j];
        y[j] = phs_from_d2(dx * dx + dy * dy + dz * dz, half);
    }
    for (int e = t; e < tri(M); e += GT) {
        const int a = tri_row(e);
        P[tri(n + a) + n + (e - tri(a))] = 0.0;
    }
    for (int p = t; p < m; p += GT) perm[p] = p;
    if (warp == 0) sh_eval_lanes(ell, px, py, pz, lane, [&](int c, double v) { y[n + c] = v; });
    gsync();
    if (st[0]) return RBFSL_ESINGULAR;

    // ---- blocked factorisation. Per pivot step: (1) all threads form the updated column k,
    // wk[i] = a_ik - sum_q L_i,q W_k,q over the open panel's columns q (rows i >= k), with
    // per-warp maxima of |wk[i]|, i > k; (2) every thread combines them into lambda and r and takes
    // the first test; (3) when it fails, all threads form the updated column r the same way, with
    // per-warp maxima for sigma; (4) every thread takes the remaining tests, warp 0 inverts the
    // pivot block, all threads interchange, then each thread forms the multipliers of its rows
    // (into the triangle's column k), the W column(s) and the forward substitution of y. A panel
    // closes after kPanel columns (or before a 2 x 2 pivot that would overflow it) with one
    // trailing update a_ij -= sum_q L_i,q W_j,q of rows and columns >= its end. Measured at
    // m = 109 (N = 40,962): 30.3 ms against 32.7 ms for one trailing update per pivot step; panels
    // of 3, 5 and 6 columns 41.1, 32.7 and 33.7 ms (warp 0 forming the multipliers: 31.8 ms).
    const long long kAbs = 0x7fffffffffffffffLL;
    int k0 = 0, pc = 0;  // the open panel: first column, columns used
    auto trailing = [&](int k1) {
        const int Rr = m - k1, E = Rr * (Rr + 1) / 2;
        constexpr int Uu = 1;  // elements per thread per round (measured: 2 and 4 slower)
        for (int e0 = t; e0 < E; e0 += Uu * GT) {
            int addr[Uu], ii[Uu], jj[Uu];
            double v[Uu];
#pragma unroll
            for (int u = 0; u < Uu; ++u) {
                const int e = e0 + u * GT;
                const int ec = e < E ? e : E - 1;  // out-of-range slots repeat a valid element
                const int tt = tri_row(ec);
                ii[u] = k1 + tt;
                jj[u] = k1 + (ec - tri(tt));
                addr[u] = tri(ii[u]) + jj[u];
                v[u] = P[addr[u]];
            }
#pragma unroll
            for (int u = 0; u < Uu; ++u) {
                if (e0 - lane + u * GT >= E) continue;  // the whole warp past the end: no DFMA issued
                const double *Li = P + tri(ii[u]) + k0;
                for (int q = 0; q < pc; ++q) v[u] = fma(-Li[q], U[q * m + jj[u]], v[u]);
            }
#pragma unroll
            for (int u = 0; u < Uu; ++u)
                if (e0 + u * GT < E) P[addr[u]] = v[u];
        }
    };
    for (int k = 0; k < m;) {
        // (1) updated column k, per-warp maxima (smallest row on ties; rows of lanes without a
        // candidate: m)
        {
            long long best = 0;
            int r = m;
            for (int i = k + t; i < m; i += GT) {
                double v = P[tri(i) + k];
                const double *Li = P + tri(i) + k0;
                for (int q = 0; q < pc; ++q) v = fma(-Li[q], U[q * m + k], v);
                wk[i] = v;
                if (i > k) {
                    const long long b = __double_as_longlong(v) & kAbs;
                    if (b > best || r == m) { best = b; r = i; }
                }
            }
            warp_max_key_row(best, r);
            if (lane == 0) { slot[warp] = best; slot[4 + warp] = r; }
        }
        gsync();
        // (2) lambda, r and the first test, the same values in every thread
        long long best = 0;
        int r = m;
        for (int w = 0; w < NW; ++w) {
            const long long b = slot[w];
            const int rw = (int)slot[4 + w];
            if (b > best || (b == best && rw < r)) { best = b; r = rw; }
        }
        const int sx = best > 0 ? exp_of(best) : 0;  // the tests' scale 2^sx: lambda in [1, 2)
        const float lam = best > 0 ? mag_f32(best, sx) : 0.0f;
        const long long kb = __double_as_longlong(wk[k]) & kAbs;
        const float akk = mag_f32(kb, sx);
        constexpr float kAlphaF = (float)kAlpha;
        const bool need_r = !(akk >= kAlphaF * lam);
        if (need_r) {
            // (3) updated column r (rows >= k, from row / column r of the triangle), maxima of
            // |wr[c]| for c != r
            long long sb = 0;
            for (int i = k + t; i < m; i += GT) {
                double v = i < r ? P[tri(r) + i] : P[tri(i) + r];
                const double *Li = P + tri(i) + k0;
                for (int q = 0; q < pc; ++q) v = fma(-Li[q], U[q * m + r], v);
                wr[i] = v;
                if (i != r) {
                    const long long b = __double_as_longlong(v) & kAbs;
                    sb = b > sb ? b : sb;
                }
            }
            sb = warp_max_key(sb);
            if (lane == 0) slot[8 + warp] = sb;
            gsync();
        }
        // (4) the remaining tests, in every thread (the same values everywhere)
        int s = 1, piv = k;
        if (need_r) {
            long long sb = 0;
            for (int w = 0; w < NW; ++w) sb = slot[8 + w] > sb ? slot[8 + w] : sb;
            const float sg = mag_f32(sb, sx);
            if (akk * sg >= kAlphaF * lam * lam) {
                s = 1;
            } else if (mag_f32(__double_as_longlong(wr[r]) & kAbs, sx) >= kAlphaF * sg) {
                piv = r;
            } else {
                s = 2;
                piv = r;
            }
        }
        if (s == 2 && pc + 2 > kPanel) {  // a 2 x 2 pivot that does not fit: close the panel first
            trailing(k);
            gsync();
            k0 = k;
            pc = 0;
            continue;
        }
        if (best <= 0 && kb == 0) return RBFSL_ESINGULAR;  // a zero column
        const int a = s == 1 ? k : k + 1, b = piv;
        // (4a) warp 0: the pivot block's inverse, from the updated columns before the interchange
        // (they are scratch: the interchange is applied to them by index below, never moved).
        // All threads: the symmetric interchange of positions a < b in the triangle (L rows
        // included), the panel's W rows, y and the row map.
        double *scal = reinterpret_cast<double *>(slot + 12);
        if (warp == 0) {
            auto bad_bits = [](double v) {  // zero or non-finite
                const long long bb = __double_as_longlong(v) & 0x7fffffffffffffffLL;
                return bb == 0 || bb >= 0x7ff0000000000000LL;
            };
            if (s == 1) {
                const double d = piv == k ? wk[k] : wr[r];
                const double dinv = recip_nr(d);  // every lane, same bits
                if (lane == 0) { scal[0] = dinv; if (bad_bits(d)) st[0] = 2; }
            } else {
                const double a11 = wk[k], a21 = wk[r], a22 = wr[r];
                const double det = fma(a11, a22, -(a21 * a21));
                const double idet = recip_nr(det);
                if (lane == 0) {  // D^-1 = [[e22, -e21], [-e21, e11]]
                    scal[0] = a11 * idet; scal[1] = a21 * idet; scal[2] = a22 * idet;
                    if (bad_bits(det)) st[0] = 2;
                }
            }
        }
        if (b != a) {
            for (int c = t; c < m; c += GT) {
                double *p1, *p2;
                if (c < a) { p1 = &P[tri(a) + c]; p2 = &P[tri(b) + c]; }
                else if (c == a) { p1 = &P[tri(a) + a]; p2 = &P[tri(b) + b]; }
                else if (c < b) { p1 = &P[tri(c) + a]; p2 = &P[tri(b) + c]; }
                else if (c == b) continue;
                else { p1 = &P[tri(c) + a]; p2 = &P[tri(c) + b]; }
                const double v = *p1;
                *p1 = *p2;
                *p2 = v;
            }
            const int o = GT - 1 - t;  // the last threads: the vectors
            if (o < pc) {
                const double v = U[o * m + a]; U[o * m + a] = U[o * m + b]; U[o * m + b] = v;
            } else if (o == kPanel) {
                const double v = y[a]; y[a] = y[b]; y[b] = v;
            } else if (o == kPanel + 1) {
                const int q = perm[a]; perm[a] = perm[b]; perm[b] = q;
            }
        }
        gsync();
        if (st[0]) return RBFSL_ESINGULAR;
        // (4b) multipliers, one row per thread: the column(s) after the interchange are the
        // updated columns read through the transposition (a b)
        if (s == 1) {
            const double *col = piv == k ? wk : wr;
            const double dinv = scal[0], yk = y[k];
            for (int i = k + 1 + t; i < m; i += GT) {
                const int si = i == a ? b : (i == b ? a : i);
                const double c = col[si];
                U[pc * m + i] = c;
                const double l = c * dinv;
                P[tri(i) + k] = l;
                y[i] = fma(-l, yk, y[i]);
            }
            if (t == 0) { P[tri(k) + k] = dinv; ptype[k] = 1; }
        } else {
            const double e11 = scal[0], e21 = scal[1], e22 = scal[2];
            const double yk0 = y[k], yk1 = y[k + 1];
            for (int i = k + 2 + t; i < m; i += GT) {
                const int si = i == a ? b : (i == b ? a : i);
                const double c0 = wk[si], c1 = wr[si];
                U[pc * m + i] = c0;
                U[(pc + 1) * m + i] = c1;
                const double L0 = fma(c0, e22, -(c1 * e21)), L1 = fma(c1, e11, -(c0 * e21));
                P[tri(i) + k] = L0;
                P[tri(i) + k + 1] = L1;
                y[i] = fma(-L1, yk1, fma(-L0, yk0, y[i]));
            }
            if (t == 0) {
                P[tri(k) + k] = e22;
                P[tri(k + 1) + k] = -e21;
                P[tri(k + 1) + k + 1] = e11;
                ptype[k] = 2; ptype[k + 1] = 0;
            }
        }
        gsync();
        pc += s;
        k += s;
        if (pc == kPanel || k >= m) {
            if (k < m) {
                trailing(k);
                gsync();
            }
            k0 = k;
            pc = 0;
        }
    }
    if (warp != 0) return RBFSL_OK;
    // ---- D z = y (blocks independent), then L^T x = z column by column
    for (int p = lane; p < m; p += kWarp) {  // the diagonal blocks hold their inverses
        if (ptype[p] == 1) {
            y[p] = y[p] * P[tri(p) + p];
        } else if (ptype[p] == 2) {
            const double f11 = P[tri(p) + p], f21 = P[tri(p + 1) + p], f22 = P[tri(p + 1) + p + 1];
            const double y0 = y[p], y1 = y[p + 1];
            y[p] = fma(f11, y0, f21 * y1);
            y[p + 1] = fma(f22, y1, f21 * y0);
        }
    }
    __syncwarp();
    for (int j = m - 1; j > 0; --j) {
        const double xj = y[j];
        const int skip = ptype[j] == 0 ? j - 1 : -1;  // (j-1, j) is a 2 x 2 block: no L entry
        for (int i = lane; i < j; i += kWarp)
            if (i != skip) y[i] = fma(-P[tri(j) + i], xj, y[i]);
        __syncwarp();
    }
    for (int p = lane; p < m; p += kWarp)
        if (perm[p] < n) out[perm[p]] = y[p];
    __syncwarp();
    return RBFSL_OK;
}

// Centre-stencil weights of one point by one warp (Sec. 3.3): the point uses the stencil
// S = Ik[k] of its nearest node k, whose m x m saddle-point matrix was factorised once. Ft is
// that factor stored column-major, the upper columns scaled by the reciprocal diagonal
// (Ft[c m + r] = L_rc below the diagonal, U_rc / U_cc above it, 1 / U_cc on it), pr its row order. b = [phi(|p - x_Sj|); Y(p)], then
// L U w~ = P b by column-oriented substitution: lane l keeps rows l, l+32, ... of the
// right-hand side in registers; after row c is final it is broadcast by a shuffle and every lane
// updates its later (earlier) rows with one coalesced column of the factor. b: m shared
// doubles of the warp. On return y_out[0..n) (shared, m doubles) holds the weights.
template <int NU>
__device__ __forceinline__ void center_point_nu(const double *__restrict__ X, const int32_t *__restrict__ S,
                                                const double *__restrict__ Ft, const int32_t *__restrict__ pr,
                                                int n, int m, int ell, int half, double px, double py,
                                                double pz, double *b, double *y_out, int lane) {
    for (int j = lane; j < n; j += 32) {
        const int64_t s = S[j];
        const double dx = px - X[3 * s], dy = py - X[3 * s + 1], dz = pz - X[3 * s + 2];
        b[j] = phs_from_d2(dx * dx + dy * dy + dz * dz, half);
    }
    sh_eval_lanes(ell, px, py, pz, lane, [&](int c, double v) { b[n + c] = v; });
    __syncwarp();
    double y[NU];
#pragma unroll
    for (int u = 0; u < NU; ++u) {
        const int r = lane + 32 * u;
        y[u] = r < m ? b[pr[r]] : 0.0;
    }
    // Column c's live entries (rows > c forward, rows < c backward) are loaded two columns
    // ahead into registers, so HBM latency overlaps the substitution.
    auto load_lower = [&](int c, double *v) {
#pragma unroll
        for (int u = 0; u < NU; ++u) {
            const int r = lane + 32 * u;
            v[u] = (c < m - 1 && u >= ((c + 1) >> 5) && r > c && r < m) ? Ft[(size_t)c * m + r] : 0.0;
        }
    };
    auto load_upper = [&](int c, double *v) {
#pragma unroll
        for (int u = 0; u < NU; ++u) {
            const int r = lane + 32 * u;
            v[u] = (c >= 0 && u <= (c >> 5) && r <= c) ? Ft[(size_t)c * m + r] : 0.0;
        }
    };
    double c0[NU], c1[NU], c2[NU];
    // forward: unit lower
    load_lower(0, c0);
    load_lower(1, c1);
    for (int c = 0; c < m - 1; ++c) {
        load_lower(c + 2, c2);
        const int uc = c >> 5;
        double own = 0.0;
#pragma unroll
        for (int u = 0; u < NU; ++u)
            if (u == uc) own = y[u];
        const double yc = __shfl_sync(0xffffffffu, own, c & 31);
#pragma unroll
        for (int u = 0; u < NU; ++u) {
            if (u >= ((c + 1) >> 5)) {  // warp-uniform: no FP64 issue for finished chunks
                const int r = lane + 32 * u;
                if (r > c && r < m) y[u] = fma(-c0[u], yc, y[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < NU; ++u) { c0[u] = c1[u]; c1[u] = c2[u]; }
    }
    // backward: upper with columns pre-scaled by the reciprocal diagonal (Ft[c m + r] = U_rc / U_cc
    // above the diagonal, 1 / U_cc on it): y_r -= Ft[c m + r] y_c for r < c, and at the end
    // x_r = y_r / U_rr, one multiply per row (kept aside as row r's diagonal entry passes by)
    double dg[NU];
#pragma unroll
    for (int u = 0; u < NU; ++u) dg[u] = 0.0;
    load_upper(m - 1, c0);
    load_upper(m - 2, c1);
    for (int c = m - 1; c >= 0; --c) {
        load_upper(c - 2, c2);
        const int uc = c >> 5;
        double own = 0.0;
#pragma unroll
        for (int u = 0; u < NU; ++u)
            if (u == uc) {
                own = y[u];
                if (lane == (c & 31)) dg[u] = c0[u];
            }
        const double yc = __shfl_sync(0xffffffffu, own, c & 31);
#pragma unroll
        for (int u = 0; u < NU; ++u) {
            if (u <= ((c - 1) >> 5) && c > 0) {
                const int r = lane + 32 * u;
                if (r < c) y[u] = fma(-c0[u], yc, y[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < NU; ++u) { c0[u] = c1[u]; c1[u] = c2[u]; }
    }
#pragma unroll
    for (int u = 0; u < NU; ++u) y[u] *= dg[u];
#pragma unroll
    for (int u = 0; u < NU; ++u) {
        const int r = lane + 32 * u;
        if (r < m) y_out[r] = y[u];
    }
    __syncwarp();
}

__device__ __forceinline__ void center_point(const double *__restrict__ X, const int32_t *__restrict__ S,
                                             const double *__restrict__ Ft, const int32_t *__restrict__ pr,
                                             int n, int m, int ell, int half, double px, double py,
                                             double pz, double *b, double *y, int lane) {
    if (m <= 64) center_point_nu<2>(X, S, Ft, pr, n, m, ell, half, px, py, pz, b, y, lane);
    else if (m <= 96) center_point_nu<3>(X, S, Ft, pr, n, m, ell, half, px, py, pz, b, y, lane);
    else if (m <= 128) center_point_nu<4>(X, S, Ft, pr, n, m, ell, half, px, py, pz, b, y, lane);
    else center_point_nu<5>(X, S, Ft, pr, n, m, ell, half, px, py, pz, b, y, lane);
}

// One output row of the gather-dot for tracer lanes t = lane, lane + 32, ... < T, with the
// weights w[0..n) and stencil S[0..n) of the row (shared or global memory). FP64:
// sum_j w_j q[S_j][t]; FP32: difference form q_c + sum_j w_j (q_j - q_c), c = S[0]. The
// summation runs over j in stencil order (the same order as gather_dot_kernel).
template <typename R, typename W>
__device__ __forceinline__ void gather_row(const W *__restrict__ w, const int32_t *__restrict__ S, int n,
                                           const R *__restrict__ q, int T, R *__restrict__ out, int lane) {
    for (int t = lane; t < T; t += 32) {
        R acc = R(0);
        if (sizeof(R) == 8) {
            for (int j = 0; j < n; ++j) acc = fma((R)w[j], q[(int64_t)S[j] * T + t], acc);
            out[t] = acc;
        } else {
            const R qc = q[(int64_t)S[0] * T + t];
            for (int j = 0; j < n; ++j) acc = fma((R)w[j], q[(int64_t)S[j] * T + t] - qc, acc);
            out[t] = qc + acc;
        }
    }
}


}  // namespace rbfsl
