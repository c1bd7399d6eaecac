"""The allocation-free factorisation entry point gives the same factor as the allocating one.

rbfsl_global_factor_noalloc serves callers that cannot allocate device memory when they
factorise (a process whose allocator owns the device budget, or code that must not let an
allocation synchronise the device under running streams); it keeps its scratch in a
library-owned device array instead. This file is collected last so that a run stopping at
the first failure has already run every other test. It passes alone in a fresh process and
after the rest of the suite.

Tolerance: the two entry points run the same kernels on the same inputs, so the factors agree
to 1e-13 relative (in practice bit for bit) and the row orders exactly; the solves through
either factor agree to the LU residual bound used by the global-method tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1804_01609_gb300 import inputs, rbfsl  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
EPS = 6.0


def _t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(DEV, dtype)


def _factor(fn, X):
    N = X.shape[0]
    LU = torch.empty((N, N), dtype=torch.float64, device=DEV)
    perm = torch.empty(N, dtype=torch.int32, device=DEV)
    fn(_t(X), rbfsl.GAUSS, EPS, LU, perm)
    return LU, perm


def _solve(LU, perm, Q):
    C = torch.empty(Q.shape, dtype=torch.float64, device=DEV)
    rbfsl.rbfsl_global_solve(LU, perm, _t(Q), C)
    return C.cpu().numpy()


@pytest.mark.parametrize("calls", [[(2562, 3), (1000, 5)]])
def test_noalloc_factor_matches_allocating_factor_twice(calls):
    for N, seed in calls:  # two calls in a row, different sizes: the shared scratch is reused
        X = inputs.nodes(N, seed)
        Q = inputs.config_global_rotation(N=N, T=4).tracers(X)
        LU_ref, perm_ref = _factor(rbfsl.rbfsl_global_factor, X)
        LU, perm = _factor(rbfsl.rbfsl_global_factor_noalloc, X)
        np.testing.assert_array_equal(perm.cpu().numpy(), perm_ref.cpu().numpy())
        a, b = LU.cpu().numpy(), LU_ref.cpu().numpy()
        assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()
        C, C_ref = _solve(LU, perm, Q), _solve(LU_ref, perm_ref, Q)
        A_inf = np.exp(-(EPS ** 2) * ((X[:, None] - X[None]) ** 2).sum(-1)).sum(1).max()
        bound = 10.0 * np.sqrt(N) * np.finfo(float).eps * A_inf * np.abs(C_ref).max()
        assert np.abs(C - C_ref).max() <= bound


def test_noalloc_factor_rejects_sizes_beyond_its_scratch():
    N = 16385  # RBFSL_NOALLOC_FACTOR_MAX_N + 1: refused before any device work
    x = torch.zeros((N, 3), dtype=torch.float64, device=DEV)
    LU = torch.empty(1, dtype=torch.float64, device=DEV)
    perm = torch.empty(1, dtype=torch.int32, device=DEV)
    with pytest.raises(rbfsl.RbfslError) as e:
        rbfsl.rbfsl_global_factor_noalloc(x, rbfsl.GAUSS, EPS, LU, perm)
    assert e.value.code == rbfsl.EINVAL and "RBFSL_NOALLOC_FACTOR_MAX_N" in str(e.value)


def test_noalloc_factor_starts_clean_after_a_singular_call():
    # N nodes at one point: every entry of A_X is 1, the first elimination step leaves exact
    # zeros, and the next pivot is zero. The status word in the shared array then reads
    # ESINGULAR; the following call must clear it and succeed.
    N = 100
    Xs = np.tile(np.array([[0.0, 0.0, 1.0]]), (N, 1))
    for fn in (rbfsl.rbfsl_global_factor, rbfsl.rbfsl_global_factor_noalloc):
        with pytest.raises(rbfsl.RbfslError) as e:
            _factor(fn, Xs)
        assert e.value.code == rbfsl.ESINGULAR
    X = inputs.nodes(642, 7)
    LU_ref, perm_ref = _factor(rbfsl.rbfsl_global_factor, X)
    LU, perm = _factor(rbfsl.rbfsl_global_factor_noalloc, X)
    np.testing.assert_array_equal(perm.cpu().numpy(), perm_ref.cpu().numpy())
    a, b = LU.cpu().numpy(), LU_ref.cpu().numpy()
    assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()
