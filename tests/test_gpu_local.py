"""GPU parity of the local RBF-SL hot path against the FP64 oracle, through the C ABI.

Tolerances (FP64 unless stated):
  departure points        1e-14 absolute (RK4 with the same stage order; rounding only)
  mixed departure points  1e-10 absolute (increment form: FP32 rounding scales with the stage
                          increments ~ |grad u| |u| dt^2, the node's own velocity is FP64)
  k-NN                    bit-exact indices vs brute force on the same points
  weights, n=31 ell=2     1e-10 relative to max|w| (the workload's stated bound; FP64 weights are
                          determined to ~3e-13 at this size)
  weights, n=84 ell=4     the saddle-point systems have cond ~1e18: moving the nodes by one
                          ulp changes the weights by ~1e-6..1e-3, so two FP64 solvers cannot
                          agree beyond that. Parity is checked on what FP64 does fix: sum w = 1
                          and spherical-harmonic reproduction to 1e-11 of the weights' scale,
                          and interpolated fields within 5x the oracle's own FP64 noise floor
                          (the largest change of the oracle's interpolated values when every
                          node coordinate moves by one ulp), plus 1e-12 of max|q|
  fields after S steps    1e-10 relative l2 at n=31 (cfg 1 literal bound)
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1804_01609_gb300 import inputs, rbfsl  # noqa: E402

import _parity  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(DEV, dtype)


@pytest.fixture(scope="module")
def cfg1():
    return inputs.config_local_rotation()


@pytest.fixture(scope="module")
def cfg2():
    return inputs.config_local_deformation()


@pytest.mark.parametrize("kind", [0, 1])
def test_trace_parity(orc, kind):
    X = inputs.nodes(40962, 12)
    prm = (inputs.rigid_rotation_params(inputs.tilted_axis(0.3)) if kind == 0
           else inputs.deformation_params(2.4, 1.0))
    dt, t1 = 1.0 / 600, 0.3
    ref = orc.trace_rk4(X, kind, prm, t1, dt)
    x = _t(X)
    xi = torch.empty_like(x)
    rbfsl.rbfsl_trace_rk4(x, kind, prm, t1, dt, rbfsl.FP64, xi)
    torch.cuda.synchronize()
    assert np.abs(xi.cpu().numpy() - ref).max() < 1e-14
    rbfsl.rbfsl_trace_rk4(x, kind, prm, t1, dt, rbfsl.MIXED, xi)
    got = xi.cpu().numpy()
    assert np.abs(got - ref).max() < 1e-10
    np.testing.assert_allclose(np.linalg.norm(got, axis=1), 1.0, atol=1e-15)


@pytest.mark.parametrize("N,k", [(2562, 31), (2562, 1), (40962, 84), (10242, 55), (642, 200)])
def test_knn_bit_exact(orc, N, k):
    X = inputs.nodes(N, 3)
    rng = np.random.default_rng(N + k)
    Q = X + rng.normal(scale=1.0 / math.sqrt(N), size=X.shape)
    Q /= np.linalg.norm(Q, axis=1, keepdims=True)
    Q[:16] = X[rng.integers(0, N, 16)]           # queries on nodes (d2 = 0)
    sample = np.arange(N) if N <= 2562 else rng.choice(N, 3000, replace=False)
    x = _t(X)
    ix = rbfsl.rbfsl_knn_index_create(x, k)
    q = _t(Q)
    idx = torch.empty((N, k), dtype=torch.int32, device=DEV)
    st = torch.full((N,), 99, dtype=torch.int32, device=DEV)
    rbfsl.rbfsl_knn_query(ix, q, k, idx, st)
    ref = orc.knn(X, Q[sample], k)
    np.testing.assert_array_equal(idx.cpu().numpy()[sample], ref)
    assert (st.cpu().numpy() == 0).all()
    ix.close()


def test_knn_ties_broken_by_index(orc):
    X = inputs.nodes(2000, 5)
    X = np.concatenate([X, X[:300]])             # exact duplicates: equal keys
    x = _t(X)
    ix = rbfsl.rbfsl_knn_index_create(x, 8)
    Q = X[:300]
    idx = torch.empty((300, 8), dtype=torch.int32, device=DEV)
    rbfsl.rbfsl_knn_query(ix, _t(Q), 8, idx)
    np.testing.assert_array_equal(idx.cpu().numpy(), orc.knn(X, Q, 8))


def test_knn_empty_and_bad_k():
    X = inputs.nodes(100, 1)
    ix = rbfsl.rbfsl_knn_index_create(_t(X), 4)
    idx = torch.empty((0, 4), dtype=torch.int32, device=DEV)
    rbfsl.rbfsl_knn_query(ix, torch.empty((0, 3), dtype=torch.float64, device=DEV), 4, idx)
    with pytest.raises(rbfsl.RbfslError):
        rbfsl.rbfsl_knn_query(ix, _t(X), 101, torch.empty((100, 101), dtype=torch.int32, device=DEV))


@pytest.mark.parametrize("kind", [0, 1])
def test_trace_rk5_parity(orc, kind):
    """Fehlberg's fifth-order tracer (Sec. 3.2) against the oracle's: FP64 to rounding; mixed
    (FP32 stage increments) to 1e-10 at dt = 1/600 as the RK4 tracer, and 16 times that at four
    times the step (the increments' FP32 rounding grows like |grad u| |u| dt^2)."""
    X = inputs.nodes(40962, 12)
    prm = (inputs.rigid_rotation_params(inputs.tilted_axis(0.3)) if kind == 0
           else inputs.deformation_params(2.4, 1.0))
    x = _t(X)
    xi = torch.empty_like(x)
    for dt, bound in ((1.0 / 600, 1e-10), (1.0 / 150, 1.6e-9)):
        t1 = 0.3
        ref = orc.trace_rk5(X, kind, prm, t1, dt)
        rbfsl.rbfsl_trace_rk5(x, kind, prm, t1, dt, rbfsl.FP64, xi)
        torch.cuda.synchronize()
        assert np.abs(xi.cpu().numpy() - ref).max() < 1e-14
        rbfsl.rbfsl_trace_rk5(x, kind, prm, t1, dt, rbfsl.MIXED, xi)
        got = xi.cpu().numpy()
        assert np.abs(got - ref).max() < bound
        np.testing.assert_allclose(np.linalg.norm(got, axis=1), 1.0, atol=1e-15)


def perturb_one_ulp(X, seed=0):
    """Every coordinate moved by one ulp in a random direction."""
    s = np.random.default_rng(seed).choice([-1.0, 1.0], size=X.shape)
    return np.nextafter(X, X + s)


def assert_within_noise_floor(orc, X, I, P, q, got, ell, p, factor=5.0, nrows=300):
    """got[r] (interpolated values at P[r] on stencil I[r]) must match the oracle within
    `factor` times the oracle's own sensitivity to a one-ulp move of the node coordinates."""
    rows = np.arange(min(nrows, len(P)))
    Xp = perturb_one_ulp(X)
    ref = np.stack([orc.stencil_weights(X, I[r], ell, orc.PHS, float(p), P[r]) @ q[I[r]] for r in rows])
    alt = np.stack([orc.stencil_weights(Xp, I[r], ell, orc.PHS, float(p), P[r]) @ q[I[r]] for r in rows])
    floor = np.abs(alt - ref).max()
    diff = np.abs(got[rows] - ref).max()
    _parity.record(test=f"noise floor N={X.shape[0]} n={I.shape[1]} ell={ell} r^{p}", rows=len(rows),
                   oracle_floor=float(floor), gpu_diff=float(diff), scale=float(np.abs(q).max()))
    assert diff <= factor * floor + 1e-12 * np.abs(q).max(), (diff, floor)


def _departures(X, seed, scale=0.6):
    rng = np.random.default_rng(seed)
    P = X + rng.normal(scale=scale / math.sqrt(X.shape[0]), size=X.shape)
    return P / np.linalg.norm(P, axis=1, keepdims=True)


def test_weights_parity_n31(orc):
    """cfg-1 stencils: FP64 weights within 1e-10 of the oracle's, every point."""
    N, n, ell, p = 2562, 31, 2, 3
    X = inputs.nodes(N, 1)
    P = _departures(X, 2)
    I = orc.knn(X, P, n)
    _, _, Wref = orc.local_apply(X, P, np.zeros(N), n, ell, orc.PHS, float(p), want_IW=True)
    w = torch.empty((N, n), dtype=torch.float64, device=DEV)
    st = torch.empty(N, dtype=torch.int32, device=DEV)
    rbfsl.rbfsl_stencil_weights(_t(X), _t(I, torch.int32), n, ell, rbfsl.PHS, p, _t(P), w, st)
    W = w.cpu().numpy()
    assert (st.cpu().numpy() == 0).all()
    assert np.abs(W - Wref).max() < 1e-10 * np.abs(Wref).max()


@pytest.mark.parametrize("N,n,ell,p", [(40962, 84, 4, 5), (10242, 55, 3, 5), (642, 84, 4, 5)])
def test_weights_invariants_and_interpolation(orc, N, n, ell, p):
    X = inputs.nodes(N, 7)
    P = _departures(X, 8)
    rng = np.random.default_rng(9)
    rows = np.sort(rng.choice(N, min(N, 1500), replace=False))
    I = orc.knn(X, P, n)
    w = torch.empty((N, n), dtype=torch.float64, device=DEV)
    st = torch.empty(N, dtype=torch.int32, device=DEV)
    rbfsl.rbfsl_stencil_weights(_t(X), _t(I, torch.int32), n, ell, rbfsl.PHS, p, _t(P), w, st)
    W = w.cpu().numpy()
    assert (st.cpu().numpy() == 0).all()
    for i in rows[:300]:
        scale = np.abs(W[i]).sum()
        assert abs(W[i].sum() - 1.0) < 1e-11 * scale
        Ys = orc.sh_eval(ell, X[I[i]])
        np.testing.assert_allclose(W[i] @ Ys, orc.sh_eval(ell, P[i]), atol=1e-11 * scale * np.abs(Ys).max())
    # interpolation of smooth fields agrees with the oracle within its FP64 noise floor
    wl = inputs.config_local_deformation(N=N, n_random=4)
    q = wl.tracers(X)
    got = np.einsum("ij,ijt->it", W[rows], q[I[rows]])
    assert_within_noise_floor(orc, X, I[rows], P[rows], q, got, ell, p)


@pytest.mark.parametrize("T", [1, 5, 33, 64])
def test_gather_dot_parity(T):
    N, n = 20000, 55
    rng = np.random.default_rng(T)
    I = rng.integers(0, N, (N, n)).astype(np.int32)
    W = rng.standard_normal((N, n))
    W /= W.sum(1, keepdims=True)
    q = rng.standard_normal((N, T))
    out = torch.empty((N, T), dtype=torch.float64, device=DEV)
    rbfsl.rbfsl_gather_dot(_t(I, torch.int32), _t(W), _t(q), out)
    ref = np.einsum("ij,ijt->it", W, q[I])
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    out32 = torch.empty((N, T), dtype=torch.float32, device=DEV)
    rbfsl.rbfsl_gather_dot(_t(I, torch.int32), _t(W, torch.float32), _t(q, torch.float32), out32)
    err = np.abs(out32.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < 1e-5


def _to_pairs(q):
    hi = q.astype(np.float32)
    return np.stack([hi, (q - hi.astype(np.float64)).astype(np.float32)], axis=-1)


@pytest.mark.parametrize("T", [1, 5, 33, 64])
def test_gather_dot_pairs(T):
    """FP32 pairs (the mixed-precision storage of w and q): the result equals the exact
    sum_j w_j q_j of the pairs' values within the pair arithmetic's rounding,
    2 (n + 8) 2^-48 sum_j |w_j| |q_j|, plus the output pair's own 2^-46 |result|; pairs come back
    normalised; small-integer data, whose sums are exact in FP32, come back bit for bit."""
    N, n = 20000, 55
    rng = np.random.default_rng(100 + T)
    I = rng.integers(0, N, (N, n)).astype(np.int32)
    W = rng.standard_normal((N, n))
    W /= W.sum(1, keepdims=True)
    q = rng.standard_normal((N, T)) + 3.0
    Wp, qp = _to_pairs(W), _to_pairs(q)
    wv = Wp[..., 0].astype(np.float64) + Wp[..., 1].astype(np.float64)
    qv = qp[..., 0].astype(np.float64) + qp[..., 1].astype(np.float64)
    out = torch.empty((N, T, 2), dtype=torch.float32, device=DEV)
    rbfsl.rbfsl_gather_dot(_t(I, torch.int32), _t(Wp, torch.float32), _t(qp, torch.float32), out, pairs=True)
    got = out.cpu().numpy()
    gv = got[..., 0].astype(np.float64) + got[..., 1].astype(np.float64)
    ref = np.einsum("ij,ijt->it", wv, qv[I])
    bound = 2 * (n + 8) * 2.0 ** -48 * np.einsum("ij,ijt->it", np.abs(wv), np.abs(qv[I])) + 2.0 ** -46 * np.abs(ref)
    assert np.all(np.abs(gv - ref) <= bound)
    # the pair storage is ~2^24 times more accurate than FP32: the error is far below FP32 rounding
    assert np.abs(gv - ref).max() < 1e-3 * 2.0 ** -24 * np.abs(ref).max()
    hi, lo = got[..., 0], got[..., 1]
    assert np.all(np.abs(lo) <= np.spacing(np.abs(hi)) / 2)
    Wi = rng.integers(-3, 4, (N, n)).astype(np.float64)
    qi = rng.integers(-1000, 1001, (N, T)).astype(np.float64)
    rbfsl.rbfsl_gather_dot(_t(I, torch.int32), _t(_to_pairs(Wi), torch.float32), _t(_to_pairs(qi), torch.float32),
                           out, pairs=True)
    got = out.cpu().numpy()
    np.testing.assert_array_equal(got[..., 0].astype(np.float64), np.einsum("ij,ijt->it", Wi, qi[I]))
    np.testing.assert_array_equal(got[..., 1], 0.0)


def _run_ctx(w, precision=rbfsl.FP64, mode=rbfsl.DIRECT, steps=None):
    ctx = rbfsl.Context(0)
    ctx.set_nodes(w.X)
    ctx.set_velocity(w.vel_kind, w.vel_params)
    ctx.set_method(rbfsl.LOCAL, mode)
    ctx.set_stencil_size(w.n)
    ctx.set_sh_degree(w.ell)
    ctx.set_kernel(rbfsl.PHS, w.power)
    ctx.set_precision(precision)
    ctx.set_dt(w.dt)
    ctx.set_time(0.0)
    ctx.set_tracers(w.q0())
    ctx.step(w.steps if steps is None else steps)
    q = ctx.get_q()
    st = ctx.get_stats()
    ctx.close()
    return q, st


@pytest.mark.parametrize("mode", [rbfsl.DIRECT, rbfsl.CENTER])
def test_cfg1_full_run_matches_oracle(orc, cfg1, mode):
    """The rotation workload at full size: N=2562, n=31, r^3, ell=2, one revolution in 120 steps."""
    q, st = _run_ctx(cfg1, mode=mode)
    assert st.singular_points == 0 and st.knn_failures == 0
    ref = orc.local_run(cfg1.X, cfg1.q0(), cfg1.n, cfg1.ell, cfg1.power, cfg1.vel_kind,
                        cfg1.vel_params, cfg1.dt, cfg1.steps, mode=mode)
    assert orc.rel_l2(q, ref) < 1e-10
    q0 = cfg1.q0()
    assert orc.rel_l2(q, q0) < 0.1                # returns after one revolution (method error)


def test_cfg1_rk5_run_matches_oracle(orc, cfg1):
    """The rotation workload through the context with the Fehlberg tracer (rbfsl_set_integrator)
    against the oracle's run with the same tracer; the field returns after one revolution."""
    w = cfg1
    ctx = rbfsl.Context(0)
    ctx.set_nodes(w.X)
    ctx.set_velocity(w.vel_kind, w.vel_params)
    ctx.set_method(rbfsl.LOCAL, rbfsl.DIRECT)
    ctx.set_stencil_size(w.n)
    ctx.set_sh_degree(w.ell)
    ctx.set_kernel(rbfsl.PHS, w.power)
    ctx.set_integrator(rbfsl.RK5)
    ctx.set_dt(w.dt)
    ctx.set_tracers(w.q0())
    ctx.step(w.steps)
    q = ctx.get_q()
    with pytest.raises(rbfsl.RbfslError):
        ctx.set_integrator(3)
    ctx.close()
    ref = orc.local_run(w.X, w.q0(), w.n, w.ell, w.power, w.vel_kind, w.vel_params, w.dt, w.steps,
                        integrator=5)
    assert orc.rel_l2(q, ref) < 1e-10
    assert orc.rel_l2(q, w.q0()) < 0.1


def test_cfg1_mixed_precision_error(orc, cfg1):
    q64, _ = _run_ctx(cfg1)
    qmx, _ = _run_ctx(cfg1, precision=rbfsl.MIXED)
    q0 = cfg1.q0()
    e64, emx = orc.rel_l2(q64, q0), orc.rel_l2(qmx, q0)
    assert abs(emx - e64) < 0.01 * e64            # within 1% of the FP64 error vs exact
    assert orc.rel_l2(qmx, q64) < 1e-5


def test_cfg2_full_size_sampled_step(orc, cfg2):
    """The deformation workload at full size (N=40962, n=84, r^9, ell=4, 32 tracers): two FP64 steps
    through the context; the second step's stencils, weights and outputs are checked on sampled
    rows against the oracle given the same departure points and input field."""
    w = cfg2
    ctx = rbfsl.Context(0)
    ctx.set_nodes(w.X)
    ctx.set_velocity(w.vel_kind, w.vel_params)
    ctx.set_method(rbfsl.LOCAL, rbfsl.DIRECT)
    ctx.set_stencil_size(w.n)
    ctx.set_sh_degree(w.ell)
    ctx.set_kernel(rbfsl.PHS, w.power)
    ctx.set_dt(w.dt)
    ctx.set_tracers(w.q0())
    ctx.step(1)
    q1 = ctx.get_q()
    ctx.step(1)
    q2 = ctx.get_q()
    N, n = w.N, w.n
    xi, I, _ = ctx.last_step_tensors(n, torch.float64)
    Xi = xi.cpu().numpy()
    ref_xi = orc.trace_rk4(w.X, w.vel_kind, w.vel_params, 2 * w.dt, w.dt)
    assert np.abs(Xi - ref_xi).max() < 1e-14
    rows = np.sort(np.random.default_rng(0).choice(N, 1000, replace=False))
    np.testing.assert_array_equal(I.cpu().numpy()[rows], orc.knn(w.X, Xi[rows], n))
    assert_within_noise_floor(orc, w.X, I.cpu().numpy()[rows], Xi[rows], q1, q2[rows], w.ell, w.power)
    st = ctx.get_stats()
    assert st.singular_points == 0 and st.knn_failures == 0
    ctx.close()
