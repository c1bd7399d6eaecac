"""FP64 CPU oracle for RBF semi-Lagrangian transport on S^2 -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously-correct restatement of the paper's method (Shankar & Wright,
"Mesh-free semi-Lagrangian methods for transport on a sphere using RBFs"), used to check
the CUDA library. Only the tests, ``__graft_entry__.smoke()`` and the bench's CPU-baseline
leg may import it. It shares no code with the CUDA path: the arithmetic lives in
``oracle.c`` (plain C, FP64, no FMA contraction) plus the closed forms below.

Parity status of each function (what pins it, see tests/test_oracle_*.py):
  trace_rk4          Rodrigues closed form (rigid rotation), exact y-axis rotation
                     (deformation), fifth-order local error, return after a period
  velocity (kind 2)  the paper's deformational flow in spherical form: x cross grad(psi) for
                     its stream function (central differences), tangency, pure rotation at
                     t = T/2, hand-evaluated values, return of the flow map at t = T
  knn                numpy lexsort of all distances (library sort), scipy cKDTree distances
  sh_eval            scipy.special.sph_harm_y, quadrature orthonormality
  gepp_solve         numpy.linalg.solve (LAPACK dgesv), pivot-order invariance
  stencil_weights    sum w = 1, exact reproduction of every spherical harmonic of degree
                     <= ell, w = e_k at a node, agreement with an mpmath 50-digit solve
  stencil_weights_ld the same system in long double: agreement with an mpmath 50-digit
                     solve (to the long double's precision times the condition number),
                     sum w = 1 and harmonic reproduction, w = e_k at a node
  local_step         return of a smooth field after a full revolution within method error
  global_*           interpolation at the nodes, LAPACK solve, Cholesky vs numpy
  global_cardinal    identity at the nodes (cardinal property), E q equal to solve-then-evaluate,
                     LAPACK solve of the transposed system, smooth fields between the nodes
  pu_*               partition of unity, interpolation at nodes, reproduction of SH <= ell,
                     B-spline / Wendland closed-form values
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (gcc, FP64, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I = ctypes.c_int
_D = ctypes.c_double


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            sig = {
                "orc_num_threads": (_I, []),
                "orc_set_threads": (None, [_I]),
                "orc_velocity": (None, [_I, _P, _P, _D, _P]),
                "orc_trace_rk4": (None, [_I, _P, _P, _I64, _D, _D, _P]),
                "orc_trace_rk5": (None, [_I, _P, _P, _I64, _D, _D, _P]),
                "orc_knn": (None, [_P, _I64, _P, _I64, _I, _P, _P]),
                "orc_sh_eval": (None, [_I, _P, _P]),
                "orc_gepp_solve": (_I, [_P, _I, _P, _I]),
                "orc_lu_factor": (_I, [_P, _I64, _P]),
                "orc_lu_solve": (None, [_P, _P, _I64, _P, _I]),
                "orc_cholesky": (_I, [_P, _I64]),
                "orc_kernel": (_D, [_I, _D, _D]),
                "orc_stencil_weights": (_I, [_P, _P, _I, _I, _I, _D, _P, _P]),
                "orc_long_double_digits": (_I, []),
                "orc_stencil_weights_ld": (_I64, [_P, _P, _I64, _I, _I, _I, _P, _P]),
                "orc_local_apply": (_I64, [_P, _I64, _I, _I, _I, _D, _I, _P, _I64, _P, _I, _P, _P, _P]),
                "orc_global_matrix": (None, [_P, _I64, _I, _D, _P]),
                "orc_global_eval": (None, [_P, _I64, _P, _I64, _I, _D, _P, _I, _P]),
                "orc_kernel_matrix": (None, [_P, _I64, _P, _I64, _I, _D, _P]),
                "orc_pu_phi": (_D, [_I, _D]),
                "orc_pu_eval": (_I64, [_P, _I64, _P, _P, _I64, _D, _P, _P, _P, _P, _I, _I, _D, _I, _I, _P]),
                "orc_pu_coefficients": (_I64, [_P, _I64, _P, _P, _P, _I, _I, _D, _P, _I, _P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return lib().orc_num_threads()


# Kernel kinds (same numbering as the library's public header, restated here).
PHS, GAUSS, IMQ = 0, 1, 2
DIRECT, CENTER = 0, 1
WENDLAND, BSPLINE = 0, 1


# ----------------------------------------------------------------------------- tracing
def set_threads(n):
    """OpenMP threads of the oracle's parallel loops (n <= 0: all processors)."""
    lib().orc_set_threads(int(n))


def velocity(kind, prm, x, t):
    x = _f64(x); prm = _f64(prm); u = np.empty(3)
    lib().orc_velocity(kind, _ptr(prm), _ptr(x), t, _ptr(u))
    return u


def trace_rk4(X, kind, prm, t1, dt):
    """Departure points of every node for the step (t1 - dt, t1] (Eq. sl_ode, RK4)."""
    X = _f64(X); prm = _f64(prm); Xi = np.empty_like(X)
    lib().orc_trace_rk4(kind, _ptr(prm), _ptr(X), X.shape[0], t1, dt, _ptr(Xi))
    return Xi


def trace_rk5(X, kind, prm, t1, dt):
    """Departure points of every node for the step (t1 - dt, t1] (Eq. sl_ode, Fehlberg's
    fifth-order formula, every stage projected)."""
    X = _f64(X); prm = _f64(prm); Xi = np.empty_like(X)
    lib().orc_trace_rk5(kind, _ptr(prm), _ptr(X), X.shape[0], t1, dt, _ptr(Xi))
    return Xi


def rotate(P, axis, angle):
    """Rodrigues rotation of points P about the unit axis by `angle` (right-handed)."""
    P = _f64(P); a = _f64(axis) / np.linalg.norm(axis)
    c, s = math.cos(angle), math.sin(angle)
    return P * c + np.cross(a[None, :], P) * s + (P @ a)[:, None] * a[None, :] * (1 - c)


def exact_departure(P, kind, prm, t0, t1):
    """Closed-form flow map from time t1 back to time t0 for both velocity kinds.

    Rigid rotation: rotate about a by -omega (t1 - t0). Deformation: y is invariant and
    (z, x) rotates about the y axis with rate g = 2 kappa y cos(pi t / T), so the map is a
    rotation about y by angle 2 kappa y (T/pi) (sin(pi t0/T) - sin(pi t1/T)) (applied with
    u = g (-z, 0, x): d(x,z)/dt = g (-z, x), i.e. positive rotation in the (z,x) plane).
    """
    P = _f64(P)
    if kind == 0:
        return rotate(P, prm[:3], -prm[3] * (t1 - t0))
    if kind != 1:
        raise ValueError("no closed-form flow map for this velocity kind")
    kappa, T = prm[0], prm[1]
    y = P[:, 1]
    beta = 2 * kappa * y * (T / math.pi) * (math.sin(math.pi * t0 / T) - math.sin(math.pi * t1 / T))
    c, s = np.cos(beta), np.sin(beta)
    x, z = P[:, 0], P[:, 2]
    # d/dt (x, z) = g (-z, x): (x, z) rotates by +G where G = int g dt; from t1 to t0, G = beta.
    return np.stack([x * c - z * s, y, z * c + x * s], axis=1)


# ----------------------------------------------------------------------------- kNN
def knn(X, Q, k, return_d2=False):
    """Brute-force k nearest nodes of each query point, key (d^2, index) ascending."""
    X = _f64(X); Q = _f64(Q)
    idx = np.empty((Q.shape[0], k), dtype=np.int32)
    d2 = np.empty((Q.shape[0], k)) if return_d2 else None
    lib().orc_knn(_ptr(X), X.shape[0], _ptr(Q), Q.shape[0], k, _ptr(idx),
                  _ptr(d2) if return_d2 else None)
    return (idx, d2) if return_d2 else idx


# ----------------------------------------------------------------------------- SH / solves
def sh_eval(L, x):
    """Real orthonormal spherical harmonics of degree <= L at one or many unit vectors."""
    x = _f64(x)
    one = x.ndim == 1
    P = x.reshape(-1, 3)
    M = (L + 1) ** 2
    out = np.empty((P.shape[0], M))
    row = np.empty(M)
    for i in range(P.shape[0]):
        pi = _f64(P[i])
        lib().orc_sh_eval(L, _ptr(pi), _ptr(row))
        out[i] = row
    return out[0] if one else out


def gepp_solve(A, B):
    A = _f64(A).copy(); B = _f64(B).copy()
    m = A.shape[0]
    nrhs = 1 if B.ndim == 1 else B.shape[1]
    rc = lib().orc_gepp_solve(_ptr(A), m, _ptr(B), nrhs)
    if rc != 0:
        raise np.linalg.LinAlgError("zero pivot")
    return B


def kernel(kind, prm, r):
    return lib().orc_kernel(kind, prm, r)


def stencil_weights(X, I, L, kkind, kprm, xi):
    """Weights of the augmented local interpolant on stencil I at xi (Eq. rbf_poly_linsys)."""
    X = _f64(X); I = np.ascontiguousarray(I, dtype=np.int32); xi = _f64(xi)
    w = np.empty(I.shape[0])
    rc = lib().orc_stencil_weights(_ptr(X), _ptr(I), I.shape[0], L, kkind, kprm, _ptr(xi), _ptr(w))
    if rc != 0:
        raise np.linalg.LinAlgError("singular stencil")
    return w


def long_double_digits():
    """Significand bits of the C long double the referee computes in (113 = IEEE binary128)."""
    return int(lib().orc_long_double_digits())


def stencil_weights_ld(X, I, L, power, Xi):
    """Referee weights: the PHS r^power stencil systems of Eq. rbf_poly_linsys for the stencils
    I (Nq x n) at the points Xi (Nq x 3), assembled and solved by partial-pivoting elimination
    in long double (see long_double_digits), rounded to FP64. NaN rows for singular systems."""
    X = _f64(X); I = np.ascontiguousarray(I, dtype=np.int32); Xi = _f64(Xi)
    Nq, n = I.shape
    W = np.empty((Nq, n))
    lib().orc_stencil_weights_ld(_ptr(X), _ptr(I), Nq, n, L, int(power), _ptr(Xi), _ptr(W))
    return W


def local_apply(X, Xi, q, n, L, kkind, kprm, mode=DIRECT, want_IW=False):
    """Interpolate q (N x T) from the nodes to the points Xi with local stencils."""
    X = _f64(X); Xi = _f64(Xi); q = _f64(q)
    q2 = q.reshape(q.shape[0], -1)
    T = q2.shape[1]
    Nq = Xi.shape[0]
    out = np.empty((Nq, T))
    I = np.empty((Nq, n), dtype=np.int32) if want_IW else None
    W = np.empty((Nq, n)) if want_IW else None
    ns = lib().orc_local_apply(_ptr(X), X.shape[0], n, L, kkind, kprm, mode, _ptr(Xi), Nq,
                               _ptr(q2), T, _ptr(out), _ptr(I) if want_IW else None,
                               _ptr(W) if want_IW else None)
    if ns:
        raise np.linalg.LinAlgError(f"{ns} singular stencils")
    out = out.reshape((Nq,) + q.shape[1:])
    return (out, I, W) if want_IW else out


def local_run(X, q0, n, L, power, vel_kind, vel_prm, dt, steps, mode=DIRECT, t0=0.0, integrator=4):
    """Algorithm 1 with the local method: `steps` steps of size dt from t0, departure points
    by RK4 (integrator 4) or Fehlberg's fifth-order formula (integrator 5)."""
    q = _f64(q0)
    trace = trace_rk5 if integrator == 5 else trace_rk4
    for m in range(steps):
        t1 = t0 + (m + 1) * dt
        Xi = trace(X, vel_kind, vel_prm, t1, dt)
        q = local_apply(X, Xi, q, n, L, PHS, float(power), mode)
    return q


# ----------------------------------------------------------------------------- global RBF
def global_matrix(X, kkind, kprm):
    X = _f64(X); N = X.shape[0]
    A = np.empty((N, N))
    lib().orc_global_matrix(_ptr(X), N, kkind, kprm, _ptr(A))
    return A


def lu_factor(A):
    LU = _f64(A).copy()
    piv = np.empty(LU.shape[0], dtype=np.int32)
    if lib().orc_lu_factor(_ptr(LU), LU.shape[0], _ptr(piv)) != 0:
        raise np.linalg.LinAlgError("zero pivot")
    return LU, piv


def lu_solve(LU, piv, B):
    B = _f64(B).copy()
    B2 = B.reshape(B.shape[0], -1)
    lib().orc_lu_solve(_ptr(LU), _ptr(piv), LU.shape[0], _ptr(B2), B2.shape[1])
    return B2.reshape(B.shape)


def cholesky(A):
    """Lower Cholesky factor, or None on breakdown (a non-positive pivot)."""
    Lc = _f64(A).copy()
    if lib().orc_cholesky(_ptr(Lc), Lc.shape[0]) != 0:
        return None
    return np.tril(Lc)


def global_eval(P, X, C, kkind, kprm):
    P = _f64(P); X = _f64(X); C = _f64(C)
    C2 = C.reshape(C.shape[0], -1)
    out = np.empty((P.shape[0], C2.shape[1]))
    lib().orc_global_eval(_ptr(P), P.shape[0], _ptr(X), X.shape[0], kkind, kprm, _ptr(C2),
                          C2.shape[1], _ptr(out))
    return out.reshape((P.shape[0],) + C.shape[1:])


def kernel_matrix(P, X, kkind, kprm):
    """Phi(P, X)[i][j] = phi(|p_i - x_j|), the evaluation matrix of Eq. srbfinterp."""
    P = _f64(P); X = _f64(X)
    Phi = np.empty((P.shape[0], X.shape[0]))
    lib().orc_kernel_matrix(_ptr(P), P.shape[0], _ptr(X), X.shape[0], kkind, kprm, _ptr(Phi))
    return Phi


def global_cardinal(P, X, kkind, kprm):
    """Cardinal (Lagrange) matrix of the global interpolant at the points P (Sec. 2.1): the
    interpolant of q at p is phi(p, X) c with A_X c = q (Eqs. srbfinterp, rbf_linsys), so the
    interpolant at all of P is E q with E = Phi(P, X) A_X^-1 (Nq x N) for every field q. Computed
    from that definition: E^T = A_X^-T Phi(P, X)^T, with the pivoted LU of A_X^T."""
    A = global_matrix(X, kkind, kprm)
    LU, piv = lu_factor(A.T)
    return lu_solve(LU, piv, kernel_matrix(P, X, kkind, kprm).T).T.copy()


class GlobalInterpolator:
    """Global RBF interpolation (Eqs. srbfinterp, rbf_linsys): A_X factorised once
    (Cholesky; pivoted LU when Cholesky breaks down), then per step c = A_X^-1 q and
    evaluation at the departure points (Sec. 3.3)."""

    def __init__(self, X, kkind=GAUSS, kprm=6.0):
        self.X = _f64(X); self.kkind = kkind; self.kprm = kprm
        A = global_matrix(self.X, kkind, kprm)
        self.LU, self.piv = lu_factor(A)
        self.factor = "lu"

    def coefficients(self, q):
        return lu_solve(self.LU, self.piv, q)

    def apply(self, Xi, q):
        return global_eval(Xi, self.X, self.coefficients(q), self.kkind, self.kprm)


# ----------------------------------------------------------------------------- RBF-PU
def pu_phi(kind, r):
    return lib().orc_pu_phi(kind, r)


class PUInterpolator:
    """RBF-PU interpolation (Eqs. wght_func, pu_func, PU_interp; Sec. 3.3): patches of radius
    R = 2 sqrt(n/N) (Eq. rad_patches) around Mp = ceil(a N / n) centres (Eq. num_patches),
    members |x - omega| < R, augmented PHS interpolant per patch."""

    def __init__(self, X, centers, n, L, power, weight_kind=WENDLAND, R=None):
        self.X = _f64(X); self.Om = _f64(centers)
        N = self.X.shape[0]
        self.R = 2.0 * math.sqrt(n / N) if R is None else float(R)
        self.L = L; self.kprm = float(power); self.wkind = weight_kind
        d2 = ((self.Om[:, None, :] - self.X[None, :, :]) ** 2).sum(-1)
        mem = [np.nonzero(np.sqrt(row) < self.R)[0].astype(np.int32) for row in d2]
        if any(len(m) == 0 for m in mem):
            raise ValueError("a patch contains no node")
        self.mstart = np.zeros(len(mem) + 1, dtype=np.int64)
        self.mstart[1:] = np.cumsum([len(m) for m in mem])
        self.members = np.ascontiguousarray(np.concatenate(mem), dtype=np.int32)

    def _coff(self, T):
        M = (self.L + 1) ** 2
        sizes = (np.diff(self.mstart) + M) * T
        coff = np.zeros(len(sizes), dtype=np.int64)
        coff[1:] = np.cumsum(sizes)[:-1]
        return coff, int(sizes.sum())

    def coefficients(self, q):
        q2 = _f64(q).reshape(self.X.shape[0], -1)
        T = q2.shape[1]
        coff, tot = self._coff(T)
        coef = np.empty(tot)
        ns = lib().orc_pu_coefficients(_ptr(self.X), self.Om.shape[0], _ptr(self.mstart),
                                       _ptr(self.members), _ptr(coff), self.L, PHS, self.kprm,
                                       _ptr(q2), T, _ptr(coef))
        if ns:
            raise np.linalg.LinAlgError(f"{ns} singular patches")
        return coef, coff, T

    def apply(self, P, q):
        P = _f64(P)
        coef, coff, T = self.coefficients(q)
        out = np.empty((P.shape[0], T))
        unc = lib().orc_pu_eval(_ptr(P), P.shape[0], _ptr(self.X), _ptr(self.Om),
                                self.Om.shape[0], self.R, _ptr(self.mstart), _ptr(self.members),
                                _ptr(coff), _ptr(coef), self.L, PHS, self.kprm, self.wkind, T,
                                _ptr(out))
        if unc:
            raise ValueError(f"{unc} points covered by no patch")
        return out.reshape((P.shape[0],) + np.shape(q)[1:])


# ----------------------------------------------------------------------------- errors
def rel_l2(approx, exact):
    return float(np.linalg.norm(approx - exact) / np.linalg.norm(exact))


def rel_linf(approx, exact):
    return float(np.max(np.abs(approx - exact)) / np.max(np.abs(exact)))
