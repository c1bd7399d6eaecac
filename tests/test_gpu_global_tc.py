"""Tensor-core (tcgen05, split TF32) evaluation of the global interpolant against the FP64
oracle. Tolerance: split TF32 keeps ~21 bits of each factor and the three products accumulate
in FP32 (a few 1e-7 of the sum's scale sum_j |phi_ij c_j|); the kernel values come from FP32
squared distances, whose rounding (~1e-7 of d^2 <= 4) is amplified by eps^2 = 36 in the
exponent. Bound: 1e-5 of the scale."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1804_01609_gb300 import inputs, rbfsl  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
EPS = 6.0


def _t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(DEV, dtype)


def _phi(P, X, kind, eps):
    d2 = ((P[:, None, :] - X[None]) ** 2).sum(-1)
    return np.exp(-(eps ** 2) * d2) if kind == rbfsl.GAUSS else 1.0 / np.sqrt(1.0 + eps ** 2 * d2)


# sizes: one tile; ragged points and nodes (partial 128-point tile, partial 32-node chunk);
# split node ranges; Tn = 112 (one CTA per SM); two tracer tiles (T = 300 -> 2 x 160); one point
@pytest.mark.parametrize("Nq,N,T,kind", [(128, 32, 32, rbfsl.GAUSS), (300, 1000, 5, rbfsl.GAUSS),
                                         (777, 2562, 64, rbfsl.GAUSS), (1, 40, 1, rbfsl.GAUSS),
                                         (200, 3001, 100, rbfsl.GAUSS), (130, 700, 300, rbfsl.GAUSS),
                                         (513, 1500, 17, rbfsl.IMQ)])
def test_tc_eval_parity(orc, Nq, N, T, kind):
    X = inputs.nodes(N, 9)
    rng = np.random.default_rng(N + T)
    C = rng.standard_normal((N, T))
    P = inputs.random_unit_vectors(Nq, rng)
    ref = orc.global_eval(P, X, C, orc.GAUSS if kind == rbfsl.GAUSS else orc.IMQ, EPS)
    scale = _phi(P, X, kind, EPS) @ np.abs(C)
    out = torch.full((Nq, T), float("nan"), dtype=torch.float32, device=DEV)
    st = torch.zeros(1, dtype=torch.int32, device=DEV)
    rbfsl.rbfsl_global_eval_tc(_t(P), _t(X), kind, EPS, _t(C), out, status=st)
    got = out.cpu().numpy().astype(np.float64)
    assert int(st.item()) == 0
    assert np.isfinite(got).all()
    assert np.all(np.abs(got - ref) <= 1e-5 * scale + 1e-30)


def test_tc_eval_deterministic_and_workspace_checked():
    """Split-K partial sums are added in a fixed order: two calls agree bit for bit. A workspace
    below the stated size is refused (EINVAL) before any launch."""
    N, T, Nq = 4000, 64, 2000
    X = inputs.nodes(N, 5)
    rng = np.random.default_rng(1)
    P, C = _t(inputs.random_unit_vectors(Nq, rng)), _t(rng.standard_normal((N, T)))
    x = _t(X)
    o1 = torch.empty((Nq, T), dtype=torch.float32, device=DEV)
    o2 = torch.empty_like(o1)
    ws = rbfsl.rbfsl_global_eval_tc(P, x, rbfsl.GAUSS, EPS, C, o1)
    rbfsl.rbfsl_global_eval_tc(P, x, rbfsl.GAUSS, EPS, C, o2, workspace=ws)
    torch.cuda.synchronize()
    assert torch.equal(o1, o2)
    small = torch.empty(ws.numel() - 16, dtype=torch.uint8, device=DEV)
    with pytest.raises(rbfsl.RbfslError) as e:
        rbfsl.rbfsl_global_eval_tc(P, x, rbfsl.GAUSS, EPS, C, o1, workspace=small)
    assert e.value.code == rbfsl.EINVAL


def test_tc_eval_full_size_sampled(orc):
    """The global workload's size: N = 10,242 nodes, 64 tracers, departure points of a step."""
    w = inputs.config_global_rotation()
    rng = np.random.default_rng(3)
    C = rng.standard_normal((w.N, w.T))
    x = _t(w.X)
    xi = torch.empty_like(x)
    rbfsl.rbfsl_trace_rk4(x, w.vel_kind, w.vel_params, w.dt, w.dt, rbfsl.FP64, xi)
    out = torch.empty((w.N, w.T), dtype=torch.float32, device=DEV)
    rbfsl.rbfsl_global_eval_tc(xi, x, rbfsl.GAUSS, EPS, _t(C, torch.float32), out)
    rows = rng.choice(w.N, 200, replace=False)
    Xi = xi.cpu().numpy()
    C32 = C.astype(np.float32).astype(np.float64)
    ref = orc.global_eval(Xi[rows], w.X, C32, orc.GAUSS, EPS)
    scale = np.exp(-(EPS ** 2) * ((Xi[rows][:, None, :] - w.X[None]) ** 2).sum(-1)) @ np.abs(C32)
    assert np.all(np.abs(out.cpu().numpy()[rows] - ref) <= 1e-5 * scale)
