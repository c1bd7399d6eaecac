"""GPU parity of the RBF-PU path (Sec. 2.3, 3.3) against the FP64 oracle, through the C ABI.

Tolerances: interpolated values within 5x the oracle's own FP64 noise floor (its change when
every node coordinate moves by one ulp) plus 1e-12 of max|q|; the invariants the method fixes
exactly -- partition of unity, interpolation at the nodes, reproduction of spherical harmonics
of degree <= ell -- to 1e-10; the FP32 evaluation (FP32 kernel values and
accumulation): the PHS coefficients of a patch cancel strongly (sum |c_j phi_j| is ~3e3 times
|s| at N = 2,562 with r^7), so FP32 evaluation keeps ~3-4 digits; the bound is 2e-3 of max|q|.
"""
import math

import numpy as np
import pytest
from scipy.special import sph_harm_y

torch = pytest.importorskip("torch")

from paper_1804_01609_gb300 import inputs, rbfsl  # noqa: E402

import _parity  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(DEV, dtype)


def _setup(N, n, ell=3, power=7, a=2.5, seed=4):
    X = inputs.nodes(N, seed)
    Mp = math.ceil(a * N / n)
    Om = inputs.fibonacci_nodes(Mp)
    R = 2.0 * math.sqrt(n / N)
    return X, Om, R


def _gpu_apply(X, Om, R, q, P, ell=3, power=7, wkind=0, dtype=torch.float64, pairs=False):
    pu = rbfsl.rbfsl_pu_create(_t(X), _t(Om), R, ell, rbfsl.PHS, power)
    q2 = q.reshape(len(X), -1)
    shape = (len(P), q2.shape[1], 2) if pairs else (len(P), q2.shape[1])
    out = torch.empty(shape, dtype=torch.float32 if pairs else dtype, device=DEV)
    st = torch.full((len(P),), 99, dtype=torch.int32, device=DEV)
    rbfsl.rbfsl_pu_apply(pu, _t(q2), _t(P), wkind, out, st, pairs=pairs)
    o = out.cpu().numpy().astype(np.float64)
    res = (o[..., 0] + o[..., 1] if pairs else o), st.cpu().numpy()
    pu.close()
    return res


@pytest.mark.parametrize("wkind", [0, 1])
def test_pu_parity_small(orc, wkind):
    N, n = 2562, 60
    X, Om, R = _setup(N, n)
    P = inputs.random_unit_vectors(1000, np.random.default_rng(1))
    q = inputs.config_local_deformation(N=N, n_random=3).tracers(X)
    got, st = _gpu_apply(X, Om, R, q, P, wkind=wkind)
    assert (st == 0).all()
    ref = orc.PUInterpolator(X, Om, n, 3, 7, weight_kind=wkind, R=R).apply(P, q)
    s = np.random.default_rng(0).choice([-1.0, 1.0], size=X.shape)
    alt = orc.PUInterpolator(np.nextafter(X, X + s), Om, n, 3, 7, weight_kind=wkind, R=R).apply(P, q)
    floor = np.abs(alt - ref).max()
    _parity.record(test=f"PU noise floor N={N} n={n} weight={wkind}", oracle_floor=float(floor),
                   gpu_diff=float(np.abs(got - ref).max()), scale=float(np.abs(q).max()))
    assert np.abs(got - ref).max() <= 5 * floor + 1e-12 * np.abs(q).max()


def test_pu_invariants():
    N, n = 2562, 60
    X, Om, R = _setup(N, n)
    P = inputs.random_unit_vectors(500, np.random.default_rng(2))
    one, _ = _gpu_apply(X, Om, R, np.ones(N), P)
    np.testing.assert_allclose(one, 1.0, atol=1e-10)
    f = inputs.cosine_bell(X, [0, 0, 1], 0.8)
    at_nodes, _ = _gpu_apply(X, Om, R, f, X)
    np.testing.assert_allclose(at_nodes[:, 0], f, atol=1e-10)
    th = lambda Q: np.arccos(np.clip(Q[:, 2], -1, 1))
    ph = lambda Q: np.arctan2(Q[:, 1], Q[:, 0])
    for (l, m) in [(1, 0), (2, 1), (3, -2), (3, 3)]:
        Y = lambda Q: (sph_harm_y(l, abs(m), th(Q), ph(Q)).real if m >= 0 else sph_harm_y(l, abs(m), th(Q), ph(Q)).imag)
        got, _ = _gpu_apply(X, Om, R, Y(X), P)
        np.testing.assert_allclose(got[:, 0], Y(P), atol=1e-10)


def test_pu_fp32_eval_and_uncovered():
    N, n = 2562, 60
    X, Om, R = _setup(N, n)
    P = inputs.random_unit_vectors(500, np.random.default_rng(3))
    q = inputs.config_local_deformation(N=N, n_random=2).tracers(X)
    g64, _ = _gpu_apply(X, Om, R, q, P)
    g32, st = _gpu_apply(X, Om, R, q, P, dtype=torch.float32)
    assert (st == 0).all()
    assert np.abs(g32 - g64).max() <= 2e-3 * np.abs(q).max()
    # patches only on the northern hemisphere: southern points are uncovered
    keep = Om[:, 2] > 0.2
    P2 = np.array([[0.0, 0.0, -1.0], [0.0, 0.0, 1.0]])
    out, st = _gpu_apply(X, Om[keep], R, q, P2)
    assert st[0] == rbfsl.EUNCOVERED and np.isnan(out[0]).all()
    assert st[1] == 0 and np.isfinite(out[1]).all()


def test_pu_ctx_steps_match_oracle(orc):
    """Whole SL steps of RBF-PU through the context vs the oracle (N=2562, 60 per patch)."""
    N, n, S = 2562, 60, 6
    X, Om, R = _setup(N, n)
    prm = inputs.rigid_rotation_params(inputs.tilted_axis(0.3), 1.0)
    q0 = inputs.gaussian_hills(X, [[0, 0.6, 0.8]], 5.0, 0.95)
    ctx = rbfsl.Context(0)
    ctx.set_nodes(X)
    ctx.set_velocity(0, prm)
    ctx.set_method(rbfsl.PU)
    ctx.set_stencil_size(n)
    ctx.set_sh_degree(3)
    ctx.set_kernel(rbfsl.PHS, 7)
    ctx.set_pu(Om, R)
    ctx.set_dt(1.0 / 24)
    ctx.set_tracers(q0)
    ctx.step(S)
    q = ctx.get_q()[:, 0]
    st = ctx.get_stats()
    ctx.close()
    assert st.uncovered_points == 0
    pu = orc.PUInterpolator(X, Om, n, 3, 7, R=R)
    ref = q0.copy()
    for m in range(S):
        ref = pu.apply(orc.trace_rk4(X, 0, prm, (m + 1) / 24, 1 / 24), ref)
    assert orc.rel_l2(q, ref) < 1e-9


def test_pu_full_size_sampled(orc):
    """N=40962 nodes, ~100 per patch (1025 patches): sampled departure points vs the oracle."""
    N, n = 40962, 100
    X, Om, R = _setup(N, n)
    rng = np.random.default_rng(5)
    P = X[rng.choice(N, 400, replace=False)] + rng.normal(scale=0.5 / math.sqrt(N), size=(400, 3))
    P /= np.linalg.norm(P, axis=1, keepdims=True)
    q = inputs.config_local_deformation(N=N, n_random=1).tracers(X)
    got, st = _gpu_apply(X, Om, R, q, P)
    assert (st == 0).all()
    ref = orc.PUInterpolator(X, Om, n, 3, 7, R=R).apply(P, q)
    assert np.abs(got - ref).max() <= 1e-8 * np.abs(q).max()


@pytest.mark.parametrize("wkind", [0, 1])
def test_pu_pair_eval(orc, wkind):
    """The mixed step's blend (RBFSL_F32X2: FP64 factors, FP32-pair sums) against the FP64
    evaluation to 1e-10 of max|q| (pair rounding ~n 2^-48 times the patch sums' cancellation
    of ~3e3), and against the oracle within 5 times its one-ulp noise floor plus that bound;
    uncovered points give NaN pairs and EUNCOVERED."""
    N, n = 2562, 60
    X, Om, R = _setup(N, n)
    P = inputs.random_unit_vectors(1000, np.random.default_rng(2))
    q = inputs.config_local_deformation(N=N, n_random=3).tracers(X)
    g64, _ = _gpu_apply(X, Om, R, q, P, wkind=wkind)
    gp, st = _gpu_apply(X, Om, R, q, P, wkind=wkind, pairs=True)
    assert (st == 0).all()
    scale = np.abs(q).max()
    assert np.abs(gp - g64).max() <= 1e-10 * scale
    ref = orc.PUInterpolator(X, Om, n, 3, 7, weight_kind=wkind, R=R).apply(P, q)
    s = np.random.default_rng(0).choice([-1.0, 1.0], size=X.shape)
    alt = orc.PUInterpolator(np.nextafter(X, X + s), Om, n, 3, 7, weight_kind=wkind, R=R).apply(P, q)
    floor = np.abs(alt - ref).max()
    _parity.record(test=f"PU pairs noise floor N={N} n={n} weight={wkind}", oracle_floor=float(floor),
                   gpu_diff=float(np.abs(gp - ref).max()), scale=float(scale))
    assert np.abs(gp - ref).max() <= 5 * floor + 1e-10 * scale
    keep = Om[:, 2] > 0.2
    out, st = _gpu_apply(X, Om[keep], R, q, np.array([[0.0, 0.0, -1.0]]), wkind=wkind, pairs=True)
    assert st[0] == rbfsl.EUNCOVERED and np.isnan(out[0]).all()
