"""GPU parity of the cardinal form of the global interpolant, E = Phi(P, X) A_X^-1 (Sec. 2.1,
Eqs. srbfinterp and rbf_linsys), and of the product q <- E q, through the C ABI.

Tolerances:
* E against the oracle's E, entry by entry: 50 cond(A_X) eps (the forward error of a backward-
  stable solve), on well-conditioned node sets where that is tight.
* At any size, the residual of each row, |E_i A_X - Phi_i|, within the LU backward-error bound
  10 sqrt(N) eps |A_X|_inf |E_i|_inf (A_X symmetric, so rows of E solve A_X e = phi).
* FP32 pairs: hi + lo equals the FP64 value to 2^-47 of it (hi = fl32(e), lo = fl32(e - hi)).
* The product: FP64 within 1e-13 of sum_j |E_ij q_jt| (the sum's rounding scale); FP32-pair
  arithmetic within K 2^-47 of that scale, K the length of the sum (each term exact to 2^-48, the
  low-order accumulator rounded in FP32 once per term).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1804_01609_gb300 import inputs, rbfsl  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(DEV, dtype)


def _pairs(a):
    hi = a.astype(np.float32)
    lo = (a - hi.astype(np.float64)).astype(np.float32)
    return np.stack([hi, lo], -1)


def _unpair(a):
    return a[..., 0].astype(np.float64) + a[..., 1].astype(np.float64)


def _factor(x, kernel, eps):
    N = x.shape[0]
    LU = torch.empty((N, N), dtype=torch.float64, device=DEV)
    perm = torch.empty(N, dtype=torch.int32, device=DEV)
    rbfsl.rbfsl_global_factor(x, kernel, eps, LU, perm)
    return LU, perm


def _cardinal(X, P, kernel, eps, pairs=False):
    x, p = _t(X), _t(P)
    LU, perm = _factor(x, kernel, eps)
    shape = (P.shape[0], X.shape[0], 2) if pairs else (P.shape[0], X.shape[0])
    E = torch.empty(shape, dtype=torch.float32 if pairs else torch.float64, device=DEV)
    rbfsl.rbfsl_global_cardinal(LU, perm, x, kernel, eps, p, E)
    return E


@pytest.mark.parametrize("kernel,eps,Nq", [(rbfsl.GAUSS, 6.0, 1100), (rbfsl.IMQ, 4.0, 300)])
def test_cardinal_matrix_matches_oracle(orc, kernel, eps, Nq):
    """N = 642 (cond(A_X) ~ 1e2): every entry against the oracle; 1100 points span three
    512-point solve blocks, the last one ragged; pairs split the same values."""
    X = inputs.nodes(642, 1)
    P = inputs.random_unit_vectors(Nq, np.random.default_rng(7))
    ref = orc.global_cardinal(P, X, kernel, eps)
    A = orc.global_matrix(X, kernel, eps)
    tol = 50 * np.linalg.cond(A) * np.finfo(float).eps
    E = _cardinal(X, P, kernel, eps).cpu().numpy()
    assert np.abs(E - ref).max() <= tol
    Ep = _cardinal(X, P, kernel, eps, pairs=True).cpu().numpy()
    assert np.all(np.abs(_unpair(Ep) - E) <= 2.0 ** -47 * np.abs(E))
    En = _cardinal(X, X, kernel, eps).cpu().numpy()       # cardinal property at the nodes
    np.testing.assert_allclose(En, np.eye(642), atol=tol)


def test_cardinal_rows_solve_the_system_at_full_size(orc):
    """N = 10,242, Gaussian eps = 6 (the global workload; A_X numerically singular): sampled
    rows of E at the departure points satisfy E_i A_X = Phi_i to the LU backward-error bound,
    and E q agrees with the solve-then-evaluate path on the same rows."""
    w = inputs.config_global_rotation()
    X = w.X
    x = _t(X)
    xi = torch.empty_like(x)
    rbfsl.rbfsl_trace_rk4(x, w.vel_kind, w.vel_params, w.dt, w.dt, rbfsl.FP64, xi)
    LU, perm = _factor(x, rbfsl.GAUSS, w.eps)
    E = torch.empty((w.N, w.N), dtype=torch.float64, device=DEV)
    rbfsl.rbfsl_global_cardinal(LU, perm, x, rbfsl.GAUSS, w.eps, xi, E)
    Xi = xi.cpu().numpy()
    rows = np.random.default_rng(3).choice(w.N, 64, replace=False)
    Er = E[torch.as_tensor(rows, device=DEV)].cpu().numpy()
    A = orc.global_matrix(X, orc.GAUSS, w.eps)
    Phi = orc.kernel_matrix(Xi[rows], X, orc.GAUSS, w.eps)
    bound = 10.0 * np.sqrt(w.N) * np.finfo(float).eps * np.abs(A).sum(1).max()
    R = np.abs(Er @ A - Phi).max(1)
    assert np.all(R <= bound * np.abs(Er).max(1))
    # the product on the device against the definition on the sampled rows
    q = w.q0()
    out = torch.empty((w.N, w.T), dtype=torch.float64, device=DEV)
    rbfsl.rbfsl_cardinal_apply(E, _t(q), out)
    got = out.cpu().numpy()[rows]
    scale = np.abs(Er) @ np.abs(q)
    assert np.all(np.abs(got - Er @ q) <= 1e-13 * scale)
    # and pairs of the same E in pair arithmetic
    Ep = torch.empty((w.N, w.N, 2), dtype=torch.float32, device=DEV)
    rbfsl.rbfsl_global_cardinal(LU, perm, x, rbfsl.GAUSS, w.eps, xi, Ep)
    outp = torch.empty((w.N, w.T, 2), dtype=torch.float32, device=DEV)
    rbfsl.rbfsl_cardinal_apply(Ep, _t(_pairs(q), torch.float32), outp)
    assert np.all(np.abs(_unpair(outp.cpu().numpy()[rows]) - Er @ q) <= w.N * 2.0 ** -47 * scale + 1e-13 * scale)


@pytest.mark.parametrize("Nq,N,T", [(1000, 3001, 64), (37, 5000, 5), (512, 700, 100), (1, 33, 1)])
def test_cardinal_apply_matches_product(Nq, N, T):
    """out = E q for random E and q against the FP64 product: ragged row tiles (32), K chunks
    (32) and splits, one or two column tiles of 64; FP32 pairs in pair arithmetic."""
    rng = np.random.default_rng(Nq + N + T)
    E = rng.standard_normal((Nq, N)) / np.sqrt(N)
    q = rng.standard_normal((N, T))
    ref = E @ q
    scale = np.abs(E) @ np.abs(q)
    out = torch.empty((Nq, T), dtype=torch.float64, device=DEV)
    ws = rbfsl.rbfsl_cardinal_apply(_t(E), _t(q), out)
    assert np.all(np.abs(out.cpu().numpy() - ref) <= 1e-13 * scale)
    out2 = torch.empty_like(out)
    rbfsl.rbfsl_cardinal_apply(_t(E), _t(q), out2, workspace=ws)
    assert torch.equal(out, out2)                        # fixed summation order
    Ep, qp = _pairs(E), _pairs(q)
    refp = _unpair(Ep) @ _unpair(qp)
    outp = torch.empty((Nq, T, 2), dtype=torch.float32, device=DEV)
    rbfsl.rbfsl_cardinal_apply(_t(Ep, torch.float32), _t(qp, torch.float32), outp)
    got = outp.cpu().numpy()
    assert np.all(np.abs(_unpair(got) - refp) <= N * 2.0 ** -47 * scale + 1e-300)
    assert np.all(np.abs(got[..., 1]) <= np.spacing(np.abs(got[..., 0])))   # normalised pairs


def test_cardinal_apply_workspace_and_errors():
    Nq, N, T = 10242, 10242, 64
    need = rbfsl.load().rbfsl_cardinal_apply_workspace_bytes(Nq, N, T)
    assert need > 0 and need % (Nq * T * 8) == 0          # K split over the SMs at this size
    E = torch.zeros((Nq, N), dtype=torch.float64, device=DEV)
    q = torch.ones((N, T), dtype=torch.float64, device=DEV)
    out = torch.empty((Nq, T), dtype=torch.float64, device=DEV)
    with pytest.raises(rbfsl.RbfslError) as e:
        rbfsl.rbfsl_cardinal_apply(E, q, out, workspace=torch.empty(need - 8, dtype=torch.uint8, device=DEV))
    assert e.value.code == rbfsl.EINVAL
    with pytest.raises(rbfsl.RbfslError) as e:
        rbfsl.rbfsl_cardinal_apply(E, q, q[:, :T])           # q_out aliases q
    assert e.value.code == rbfsl.EINVAL
    rbfsl.rbfsl_cardinal_apply(E, q, out, workspace=torch.empty(need, dtype=torch.uint8, device=DEV))
    assert out.abs().max().item() == 0.0
    e0 = torch.empty((0, N), dtype=torch.float64, device=DEV)
    rbfsl.rbfsl_cardinal_apply(e0, q, torch.empty((0, T), dtype=torch.float64, device=DEV))


def _ctx(w, precision, form, steps, dt=None):
    ctx = rbfsl.Context(0)
    ctx.set_nodes(w.X)
    ctx.set_velocity(w.vel_kind, w.vel_params)
    ctx.set_method(rbfsl.GLOBAL, rbfsl.DIRECT)
    ctx.set_kernel(rbfsl.GAUSS, w.eps)
    ctx.set_precision(precision)
    ctx.set_global_form(form)
    ctx.set_dt(dt or w.dt)
    ctx.set_tracers(w.q0())
    ctx.step(steps)
    return ctx


@pytest.mark.parametrize("precision", [rbfsl.FP64, rbfsl.MIXED])
def test_cardinal_run_matches_oracle(orc, precision):
    """A revolution of the rotation workload at N = 642 with the cardinal form (FP64, and FP32
    pairs) against the oracle's E applied step by step; then set_dt rebuilds E for the new
    departure points; a time-dependent flow is refused."""
    w = inputs.config_global_rotation(N=642, T=4, steps=120)
    Xi = orc.trace_rk4(w.X, w.vel_kind, w.vel_params, w.dt, w.dt)
    E = orc.global_cardinal(Xi, w.X, orc.GAUSS, w.eps)
    ref = w.q0()
    for _ in range(w.steps):
        ref = E @ ref
    ctx = _ctx(w, precision, rbfsl.GLOBAL_CARDINAL, w.steps)
    assert orc.rel_l2(ctx.get_q(), ref) < 1e-10
    assert ctx.get_stats().steps_done == w.steps
    ctx.set_dt(2 * w.dt)
    ctx.step(10)
    E2 = orc.global_cardinal(orc.trace_rk4(w.X, w.vel_kind, w.vel_params, 2 * w.dt, 2 * w.dt), w.X,
                             orc.GAUSS, w.eps)
    for _ in range(10):
        ref = E2 @ ref
    assert orc.rel_l2(ctx.get_q(), ref) < 1e-10
    ctx.close()
    wd = inputs.config_local_deformation(N=642, steps=4)
    c2 = rbfsl.Context(0)
    c2.set_nodes(wd.X)
    c2.set_velocity(wd.vel_kind, wd.vel_params)
    c2.set_method(rbfsl.GLOBAL, rbfsl.DIRECT)
    c2.set_kernel(rbfsl.GAUSS, 6.0)
    c2.set_global_form(rbfsl.GLOBAL_CARDINAL)
    c2.set_dt(wd.dt)
    c2.set_tracers(wd.q0())
    with pytest.raises(rbfsl.RbfslError) as e:
        c2.step(1)
    assert e.value.code == rbfsl.EINVAL
    c2.close()
