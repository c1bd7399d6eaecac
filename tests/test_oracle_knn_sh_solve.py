"""Pins for the oracle's brute-force k-NN, spherical harmonics and dense solvers.

k-NN: against numpy's lexicographic sort of every squared distance, computed elementwise in
the same operation order (library sort), and scipy's kd-tree distances (the paper's search
structure, Sec. 3.3).
Spherical harmonics (augmentation basis of Eq. rbf_poly): against scipy.special.sph_harm_y
and an exact quadrature of the Gram matrix.
Solvers: against LAPACK (numpy.linalg.solve / cholesky).
"""
import math

import numpy as np
import pytest
from scipy.spatial import cKDTree
from scipy.special import roots_legendre, sph_harm_y

from paper_1804_01609_gb300 import inputs


def _d2_numpy(X, q):
    dx, dy, dz = q[0] - X[:, 0], q[1] - X[:, 1], q[2] - X[:, 2]
    return (dx * dx + dy * dy) + dz * dz


@pytest.mark.parametrize("k", [1, 31, 84])
def test_knn_bit_exact_vs_lexsort(orc, k):
    X = inputs.nodes(3000, 21)
    rng = np.random.default_rng(4)
    Q = inputs.random_unit_vectors(64, rng)
    Q[:8] = X[rng.integers(0, 3000, 8)]  # queries exactly at nodes: the node comes first
    idx, d2 = orc.knn(X, Q, k, return_d2=True)
    for i, q in enumerate(Q):
        d = _d2_numpy(X, q)
        order = np.lexsort((np.arange(len(X)), d))[:k]
        np.testing.assert_array_equal(idx[i], order)
        np.testing.assert_array_equal(d2[i], d[order])
    assert np.all(d2[:8, 0] == 0.0)
    tree = cKDTree(X)
    dd, _ = tree.query(Q, k=k)
    np.testing.assert_allclose(np.sqrt(d2), dd.reshape(d2.shape), rtol=1e-14, atol=1e-16)


def test_knn_ties_broken_by_index(orc):
    """Duplicated coordinates give equal keys; the smaller index must come first."""
    X = inputs.nodes(400, 2)
    X = np.concatenate([X, X[:50]])  # nodes 400..449 duplicate 0..49
    idx = orc.knn(X, X[:50], 2)
    np.testing.assert_array_equal(idx[:, 0], np.arange(50))
    np.testing.assert_array_equal(idx[:, 1], np.arange(400, 450))


def _real_sh_scipy(l, m, P):
    theta = np.arccos(np.clip(P[:, 2], -1, 1))
    phi = np.arctan2(P[:, 1], P[:, 0])
    Y = sph_harm_y(l, abs(m), theta, phi)
    if m == 0:
        return Y.real
    return math.sqrt(2) * (Y.real if m > 0 else Y.imag)


@pytest.mark.parametrize("L", [2, 4, 6])
def test_sh_matches_scipy_up_to_sign(orc, L):
    P = inputs.random_unit_vectors(50, np.random.default_rng(L))
    Y = orc.sh_eval(L, P)
    for l in range(L + 1):
        for m in range(-l, l + 1):
            ref = _real_sh_scipy(l, m, P)
            got = Y[:, l * l + l + m]
            s = np.sign(ref @ got)  # sign conventions differ by (-1)^m
            np.testing.assert_allclose(got, s * ref, atol=1e-13)


def test_sh_orthonormal_by_exact_quadrature(orc):
    """Gauss-Legendre in z times a uniform rule in azimuth integrates every polynomial of
    degree <= 2L exactly, so the Gram matrix must be the identity."""
    L = 5
    zq, wz = roots_legendre(L + 2)
    nphi = 2 * L + 2
    ph = 2 * math.pi * np.arange(nphi) / nphi
    Z, PH = np.meshgrid(zq, ph, indexing="ij")
    W = np.outer(wz, np.full(nphi, 2 * math.pi / nphi)).ravel()
    r = np.sqrt(1 - Z ** 2)
    P = np.stack([(r * np.cos(PH)).ravel(), (r * np.sin(PH)).ravel(), Z.ravel()], axis=1)
    Y = orc.sh_eval(L, P)
    G = Y.T @ (W[:, None] * Y)
    np.testing.assert_allclose(G, np.eye((L + 1) ** 2), atol=1e-13)


def test_gepp_vs_lapack(orc):
    rng = np.random.default_rng(0)
    for m in (1, 2, 7, 40, 109):
        A = rng.standard_normal((m, m))
        B = rng.standard_normal((m, 3))
        np.testing.assert_allclose(orc.gepp_solve(A, B), np.linalg.solve(A, B), rtol=1e-10, atol=1e-12)


def test_gepp_needs_pivoting_and_flags_singular(orc):
    A = np.array([[0.0, 1.0], [1.0, 0.0]])  # zero leading entry: pivoting is required
    np.testing.assert_allclose(orc.gepp_solve(A, np.array([2.0, 3.0])), [3.0, 2.0])
    with pytest.raises(np.linalg.LinAlgError):
        orc.gepp_solve(np.array([[1.0, 2.0], [2.0, 4.0]]), np.array([1.0, 1.0]))


def test_lu_and_cholesky_vs_lapack(orc):
    rng = np.random.default_rng(1)
    m = 150
    A = rng.standard_normal((m, m))
    LU, piv = orc.lu_factor(A)
    B = rng.standard_normal((m, 5))
    np.testing.assert_allclose(orc.lu_solve(LU, piv, B), np.linalg.solve(A, B), rtol=1e-9, atol=1e-11)
    S = A @ A.T + m * np.eye(m)
    np.testing.assert_allclose(orc.cholesky(S), np.linalg.cholesky(S), rtol=1e-12, atol=1e-12)
    S[5, 5] = -1.0
    S[5, :5] = S[:5, 5] = 0
    assert orc.cholesky(S) is None
