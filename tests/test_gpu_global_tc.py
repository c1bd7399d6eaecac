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


@pytest.mark.parametrize("Nq,N,T", [(128, 32, 32), (300, 1000, 5), (777, 2562, 64), (1, 40, 1)])
def test_tc_eval_parity(orc, Nq, N, T):
    X = inputs.nodes(N, 9)
    rng = np.random.default_rng(N + T)
    C = rng.standard_normal((N, T))
    P = inputs.random_unit_vectors(Nq, rng)
    ref = orc.global_eval(P, X, C, orc.GAUSS, EPS)
    scale = np.exp(-(EPS ** 2) * ((P[:, None, :] - X[None]) ** 2).sum(-1)) @ np.abs(C)
    out = torch.full((Nq, T), float("nan"), dtype=torch.float32, device=DEV)
    rbfsl.rbfsl_global_eval_tc(_t(P), _t(X), rbfsl.GAUSS, EPS, _t(C), out)
    got = out.cpu().numpy().astype(np.float64)
    assert np.isfinite(got).all()
    assert np.all(np.abs(got - ref) <= 1e-5 * scale + 1e-30)


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
