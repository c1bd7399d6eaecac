"""Pins for the oracle's local stencil weights (Eqs. rbf_poly, rbf_poly_linsys).

The weights w of a point xi on a stencil must (i) sum to one and reproduce every spherical
harmonic of degree <= ell exactly (the moment rows of the saddle-point system), (ii) equal
the unit vector e_k when xi is the k-th stencil node (interpolation, Eq. rbf_poly_linsys),
(iii) give the same value as building the interpolant's coefficients and evaluating it
(numpy solve), and (iv) agree with a 40-digit mpmath solve of the same system.
"""
import math

import mpmath
import numpy as np
import pytest
from scipy.special import sph_harm_y

from paper_1804_01609_gb300 import inputs

import _mp_referee

PHS = 0


def _real_sh_scipy(L, P):
    P = np.atleast_2d(P)
    theta = np.arccos(np.clip(P[:, 2], -1, 1))
    phi = np.arctan2(P[:, 1], P[:, 0])
    cols = []
    for l in range(L + 1):
        for m in range(-l, l + 1):
            Y = sph_harm_y(l, abs(m), theta, phi)
            cols.append(Y.real if m == 0 else math.sqrt(2) * (Y.real if m > 0 else Y.imag))
    return np.stack(cols, axis=1)


CASES = [(2562, 31, 2, 3), (10242, 55, 3, 5), (40962, 84, 4, 5)]


def _setup(N, n, seed=3, npts=12):
    X = inputs.nodes(N, seed)
    rng = np.random.default_rng(seed)
    # departure-like points: nodes displaced by a fraction of the node spacing
    P = X[rng.integers(0, N, npts)] + rng.normal(scale=0.5 / math.sqrt(N), size=(npts, 3))
    P /= np.linalg.norm(P, axis=1, keepdims=True)
    return X, P


@pytest.mark.parametrize("N,n,ell,power", CASES)
def test_weights_reproduce_spherical_harmonics(orc, N, n, ell, power):
    X, P = _setup(N, n)
    I = orc.knn(X, P, n)
    for i, xi in enumerate(P):
        w = orc.stencil_weights(X, I[i], ell, PHS, float(power), xi)
        assert abs(w.sum() - 1.0) < 1e-12
        Ys = _real_sh_scipy(ell, X[I[i]])     # independent SH evaluation (scipy)
        Yxi = _real_sh_scipy(ell, xi)[0]
        scale = np.abs(w).sum() * np.abs(Ys).max()
        np.testing.assert_allclose(w @ Ys, Yxi, atol=1e-12 * scale)


@pytest.mark.parametrize("N,n,ell,power,tol", [(2562, 31, 2, 3, 1e-12), (10242, 55, 3, 5, 1e-7)])
def test_weights_at_a_node_are_a_unit_vector(orc, N, n, ell, power, tol):
    """Interpolation at the nodes; the bound follows the conditioning of each size (the FP64
    weights themselves are only determined to ~1e-13 and ~1e-9 there)."""
    X, _ = _setup(N, n)
    for k in (0, 7, n - 1):
        I = orc.knn(X, X[100:101], n)[0]
        w = orc.stencil_weights(X, I, ell, PHS, float(power), X[I[k]])
        e = np.zeros(n); e[k] = 1.0
        np.testing.assert_allclose(w, e, atol=tol)


def test_weights_equal_the_interpolant_value(orc):
    """sum_j w_j f_j equals s(xi) from the coefficients of Eq. rbf_poly_linsys (numpy solve)."""
    N, n, ell, p = 2562, 31, 2, 3
    X, P = _setup(N, n)
    I = orc.knn(X, P, n)
    rng = np.random.default_rng(8)
    for i, xi in enumerate(P):
        S = X[I[i]]
        r = np.linalg.norm(S[:, None] - S[None], axis=-1)
        Ps = _real_sh_scipy(ell, S)
        M = Ps.shape[1]
        A = np.block([[r ** p, Ps], [Ps.T, np.zeros((M, M))]])
        f = rng.standard_normal(n)
        c = np.linalg.solve(A, np.concatenate([f, np.zeros(M)]))
        s = np.linalg.norm(xi - S, axis=1) ** p @ c[:n] + _real_sh_scipy(ell, xi)[0] @ c[n:]
        w = orc.stencil_weights(X, I[i], ell, PHS, float(p), xi)
        assert abs(w @ f - s) < 1e-11 * np.abs(f).max()


def test_weights_vs_40_digit_solve(orc):
    """FP64 GEPP weights agree with an mpmath solve of the same FP64 system to 1e-11."""
    N, n, ell, p = 2562, 31, 2, 3
    X, P = _setup(N, n, npts=3)
    I = orc.knn(X, P, n)
    mpmath.mp.dps = 40
    for i, xi in enumerate(P):
        S = X[I[i]]
        Ys = orc.sh_eval(ell, S)
        M = Ys.shape[1]
        m = n + M
        A = mpmath.matrix(m, m)
        b = mpmath.matrix(m, 1)
        for a in range(n):
            for c in range(n):
                d = [mpmath.mpf(float(S[a, t])) - mpmath.mpf(float(S[c, t])) for t in range(3)]
                A[a, c] = mpmath.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2) ** p
            for c in range(M):
                A[a, n + c] = A[n + c, a] = mpmath.mpf(float(Ys[a, c]))
            d = [mpmath.mpf(float(xi[t])) - mpmath.mpf(float(S[a, t])) for t in range(3)]
            b[a] = mpmath.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2) ** p
        Yx = orc.sh_eval(ell, xi)
        for c in range(M):
            b[n + c] = mpmath.mpf(float(Yx[c]))
        ref = np.array([float(v) for v in mpmath.lu_solve(A, b)[:n]])
        w = orc.stencil_weights(X, I[i], ell, PHS, float(p), xi)
        assert np.abs(w - ref).max() < 1e-11 * np.abs(ref).max()


def test_long_double_referee_vs_50_digit_solve(orc):
    """The long-double referee (stencil_weights_ld) against a 50-digit solve of the same
    polynomial system with its harmonics from mpmath's Legendre functions (tests/_mp_referee.py):
    within the long double's precision times the system's conditioning (1e7 allowed here); with
    IEEE binary128 that is the final rounding to FP64."""
    N, n, ell, p = 2562, 31, 2, 3
    X, P = _setup(N, n, npts=3)
    I = orc.knn(X, P, n)
    W = orc.stencil_weights_ld(X, I, ell, p, P)
    for i, xi in enumerate(P):
        ref = _mp_referee.mp_weights(X[I[i]], xi, ell, p)
        tol = max(2.0 ** -52, 1e7 * 2.0 ** -orc.long_double_digits())
        assert np.abs(W[i] - ref).max() <= tol * np.abs(ref).max()
        assert abs(W[i].sum() - 1.0) < 1e-15


def test_long_double_referee_at_a_node_and_invariants(orc):
    """w = e_k at the k-th stencil node; sum w = 1 and reproduction of every harmonic of
    degree <= ell (scipy's harmonics) at the m = 71 size, to the long double's precision."""
    N, n, ell, p = 10242, 55, 3, 7
    X, P = _setup(N, n, npts=4)
    I = orc.knn(X, P, n)
    W = orc.stencil_weights_ld(X, I, ell, p, P)
    for i, xi in enumerate(P):
        assert abs(W[i].sum() - 1.0) < 1e-12
        Ys = _real_sh_scipy(ell, X[I[i]])
        np.testing.assert_allclose(W[i] @ Ys, _real_sh_scipy(ell, xi)[0], atol=1e-12 * np.abs(W[i]).sum())
    Ik = I[:1]
    Wk = orc.stencil_weights_ld(X, Ik, ell, p, X[Ik[0, 5]][None])
    e = np.zeros(n); e[5] = 1.0
    np.testing.assert_allclose(Wk[0], e, atol=1e-9)
