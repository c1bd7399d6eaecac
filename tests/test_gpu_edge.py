"""Edge cases of the C ABI on the GPU: empty inputs, degenerate stencils, the largest systems the
library accepts and the first it refuses, departure points that coincide with a node, and the
error codes a mis-configured context returns. Expected values come from the definitions
(Eq. rbf_poly_linsys: interpolation at a node reproduces the datum; a stencil with two equal
nodes has two equal rows) and from the oracle where a number is compared."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1804_01609_gb300 import inputs, rbfsl  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(DEV, dtype)


def test_empty_inputs_are_no_ops():
    """Nq = 0 (or N = 0 for the tracer) launches nothing and leaves outputs untouched."""
    X = inputs.nodes(642, 3)
    x = _t(X)
    e3 = torch.empty((0, 3), dtype=torch.float64, device=DEV)
    rbfsl.rbfsl_trace_rk4(e3, rbfsl.VEL_RIGID, inputs.rigid_rotation_params(inputs.tilted_axis(0.3)), 0.1,
                          0.01, rbfsl.MIXED, torch.empty_like(e3))
    idx0 = torch.empty((0, 31), dtype=torch.int32, device=DEV)
    w0 = torch.empty((0, 31), dtype=torch.float64, device=DEV)
    rbfsl.rbfsl_stencil_weights(x, idx0, 31, 2, rbfsl.PHS, 3, e3, w0)
    q = _t(np.ones((642, 4)))
    out0 = torch.empty((0, 4), dtype=torch.float64, device=DEV)
    rbfsl.rbfsl_gather_dot(idx0, w0, q, out0)
    C = _t(np.ones((642, 4)))
    rbfsl.rbfsl_global_eval(e3, x, rbfsl.GAUSS, 6.0, C, out0)
    o32 = torch.empty((0, 4), dtype=torch.float32, device=DEV)
    rbfsl.rbfsl_global_eval_tc(e3, x, rbfsl.GAUSS, 6.0, C, o32)
    pu = rbfsl.rbfsl_pu_create(x, _t(inputs.fibonacci_nodes(17)), 2.0 * np.sqrt(100 / 642), 3, rbfsl.PHS, 7)
    rbfsl.rbfsl_pu_apply(pu, q, e3, rbfsl.PU_WENDLAND, out0)
    pu.close()
    torch.cuda.synchronize()


def test_duplicate_nodes_give_a_singular_stencil():
    """Two equal nodes in one stencil make two equal rows of the saddle-point matrix: the point
    is flagged RBFSL_ESINGULAR and its weights are NaN; other points are unaffected."""
    n, ell, p = 31, 2, 3
    X = inputs.nodes(2562, 5)
    X[1] = X[0]
    I = np.stack([np.arange(n), np.arange(100, 100 + n)]).astype(np.int32)
    P = np.stack([X[2] + 1e-3, X[110] + 1e-3])
    P /= np.linalg.norm(P, axis=1, keepdims=True)
    w = torch.empty((2, n), dtype=torch.float64, device=DEV)
    st = torch.zeros(2, dtype=torch.int32, device=DEV)
    rbfsl.rbfsl_stencil_weights(_t(X), _t(I, torch.int32), n, ell, rbfsl.PHS, p, _t(P), w, status=st)
    s = st.cpu().numpy()
    W = w.cpu().numpy()
    assert s[0] == rbfsl.ESINGULAR and np.isnan(W[0]).all()
    assert s[1] == rbfsl.OK and np.isfinite(W[1]).all() and abs(W[1].sum() - 1.0) < 1e-12


@pytest.mark.parametrize("prec_dtype", [torch.float64, torch.float32])
def test_departure_point_on_a_node_reproduces_its_value(orc, prec_dtype):
    """xi = x_k: the weights are the k-th unit vector (interpolation at a node), to rounding;
    float32 here means the FP32-pair weights of the mixed step (value = hi + lo)."""
    n, ell, p = 31, 2, 3
    X = inputs.nodes(2562, 6)
    rows = np.arange(0, 2562, 97)
    P = X[rows]
    I = orc.knn(X, P, n).astype(np.int32)
    assert (I[:, 0] == rows).all()
    shape = (len(rows), n) if prec_dtype == torch.float64 else (len(rows), n, 2)
    w = torch.empty(shape, dtype=prec_dtype, device=DEV)
    rbfsl.rbfsl_stencil_weights(_t(X), _t(I, torch.int32), n, ell, rbfsl.PHS, p, _t(P), w)
    W = w.cpu().numpy().astype(np.float64)
    if W.ndim == 3:
        W = W[..., 0] + W[..., 1]
    E = np.zeros_like(W)
    E[:, 0] = 1.0
    assert np.abs(W - E).max() < 1e-11


def test_largest_accepted_system_and_first_refused():
    """n + (ell+1)^2 = RBFSL_MAX_SYSTEM = 160 (n = 124, ell = 5) runs and its weights sum to 1;
    161 and ell = RBFSL_MAX_SH_DEGREE + 1 are refused with EINVAL."""
    X = inputs.nodes(10242, 7)
    rng = np.random.default_rng(0)
    P = X[rng.choice(10242, 64, replace=False)] + 2e-3 * rng.standard_normal((64, 3))
    P /= np.linalg.norm(P, axis=1, keepdims=True)
    x = _t(X)
    ix = rbfsl.rbfsl_knn_index_create(x, 125)
    for n, ell, ok in [(124, 5, True), (125, 5, False), (31, 9, False)]:
        I = torch.empty((64, n), dtype=torch.int32, device=DEV)
        rbfsl.rbfsl_knn_query(ix, _t(P), n, I)
        w = torch.empty((64, n), dtype=torch.float64, device=DEV)
        st = torch.zeros(64, dtype=torch.int32, device=DEV)
        if ok:
            rbfsl.rbfsl_stencil_weights(x, I, n, ell, rbfsl.PHS, 2 * ell + 1, _t(P), w, status=st)
            W = w.cpu().numpy()
            assert (st.cpu().numpy() == rbfsl.OK).all()
            assert np.abs(W.sum(1) - 1.0).max() < 1e-8
        else:
            with pytest.raises(rbfsl.RbfslError) as e:
                rbfsl.rbfsl_stencil_weights(x, I, n, ell, rbfsl.PHS, 2 * ell + 1, _t(P), w, status=st)
            assert e.value.code == rbfsl.EINVAL
    ix.close()


def test_context_reports_misconfiguration():
    """ENOTCONF for a step before the problem is complete, EINVAL for bad arguments and for a
    kernel the method cannot use; the context stays usable after each error."""
    w = inputs.config_local_rotation(N=642, steps=2)
    c = rbfsl.Context(0)
    with pytest.raises(rbfsl.RbfslError) as e:
        c.step(1)
    assert e.value.code == rbfsl.ENOTCONF
    c.set_nodes(w.X)
    with pytest.raises(rbfsl.RbfslError) as e:
        c.set_tracers(np.ones((100, 2)))            # wrong N
    assert e.value.code == rbfsl.EINVAL
    with pytest.raises(rbfsl.RbfslError) as e:
        c.set_precision(7)
    assert e.value.code == rbfsl.EINVAL
    c.set_velocity(w.vel_kind, w.vel_params)
    c.set_method(rbfsl.LOCAL, rbfsl.DIRECT)
    c.set_stencil_size(w.n)
    c.set_sh_degree(w.ell)
    c.set_kernel(rbfsl.GAUSS, 6.0)                  # local stencils need the PHS kernel
    c.set_dt(w.dt)
    c.set_tracers(w.q0())
    with pytest.raises(rbfsl.RbfslError) as e:
        c.step(1)
    assert e.value.code == rbfsl.EINVAL
    c.set_kernel(rbfsl.PHS, w.power)
    c.step(w.steps)                                 # recovers once configured
    assert np.isfinite(c.get_q()).all() and c.get_stats().steps_done == w.steps
    c.set_method(rbfsl.PU)
    with pytest.raises(rbfsl.RbfslError) as e:      # RBF-PU without patches
        c.step(1)
    assert e.value.code == rbfsl.ENOTCONF
    c.close()
