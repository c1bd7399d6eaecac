"""GPU parity on the paper's own test cases (Sec. 4) against the oracle, through the C ABI:
the deformational flow of Sec. 4.2 (velocity kind RBFSL_VEL_NL: the CUDA path evaluates it as
x cross grad(psi), the oracle in the paper's spherical form, so the two share no formula),
and the solid-body rotation of Sec. 4.1 at alpha = pi/2 with the paper's time step pi/10.

Tolerances: departure points to 1e-13 (two evaluations of the same field, trigonometric
rounding only; the mixed tracer evaluates this field in FP64, so it equals the FP64 one
bitwise); whole runs to 1e-10 relative l2 as the other local runs; the mixed run within 1% of
the FP64 error against the exact solution.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1804_01609_gb300 import inputs, rbfsl  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(DEV, dtype)


@pytest.mark.parametrize("t1", [0.1, 2.3, 5.0])
def test_nl_departure_points(orc, t1):
    X = inputs.nodes(10242, 11)
    prm = inputs.nl_deformation_params(5.0)
    x = _t(X)
    xi = torch.empty_like(x)
    xm = torch.empty_like(x)
    for trace, ref_fn in ((rbfsl.rbfsl_trace_rk4, orc.trace_rk4), (rbfsl.rbfsl_trace_rk5, orc.trace_rk5)):
        ref = ref_fn(X, rbfsl.VEL_NL, prm, t1, 0.1)
        trace(x, rbfsl.VEL_NL, prm, t1, 0.1, rbfsl.FP64, xi)
        trace(x, rbfsl.VEL_NL, prm, t1, 0.1, rbfsl.MIXED, xm)
        assert np.abs(xi.cpu().numpy() - ref).max() < 1e-13
        assert torch.equal(xi, xm)


def _run(w, mode, precision=rbfsl.FP64, method=rbfsl.LOCAL):
    ctx = rbfsl.Context(0)
    ctx.set_nodes(w.X)
    ctx.set_velocity(w.vel_kind, w.vel_params)
    ctx.set_method(method, mode)
    ctx.set_stencil_size(w.n)
    ctx.set_sh_degree(w.ell)
    ctx.set_kernel(rbfsl.PHS, w.power)
    ctx.set_precision(precision)
    ctx.set_dt(w.dt)
    ctx.set_tracers(w.q0())
    ctx.step(w.steps)
    q = ctx.get_q()
    st = ctx.get_stats()
    ctx.close()
    assert st.singular_points == 0 and st.knn_failures == 0
    return q


@pytest.mark.parametrize("ic,mode", [("cosine", rbfsl.CENTER), ("gaussian", rbfsl.DIRECT)])
def test_nl_deformation_run_matches_oracle(orc, ic, mode):
    """Two cosine bells / two Gaussian bells through the deformational flow to T = 5 in 50
    steps (dt = 1/10 as in the paper), N = 2562, n = 31 (ell = 2, r^5 by the paper's rules)."""
    w = inputs.config_nl(2562, ic=ic, n=31)
    q = _run(w, mode)
    ref = orc.local_run(w.X, w.q0(), w.n, w.ell, w.power, w.vel_kind, w.vel_params, w.dt, w.steps, mode=mode)
    assert orc.rel_l2(q, ref) < 1e-10
    q0 = w.q0()
    e64 = orc.rel_l2(q, q0)
    assert e64 < 0.5                                      # returns at T = 5 (method error)
    emx = orc.rel_l2(_run(w, mode, rbfsl.MIXED), q0)
    assert abs(emx - e64) < 0.01 * e64


def test_sbr_run_matches_oracle(orc):
    """One revolution of the cosine bell of radius 1/3 over the poles (alpha = pi/2) in 20 steps
    of pi/10, N = 2562, n = 31, direct stencils."""
    w = inputs.config_sbr(2562, n=31)
    assert w.steps == 20 and abs(w.dt - np.pi / 10) < 1e-15
    q = _run(w, rbfsl.DIRECT)
    ref = orc.local_run(w.X, w.q0(), w.n, w.ell, w.power, w.vel_kind, w.vel_params, w.dt, w.steps)
    assert orc.rel_l2(q, ref) < 1e-10
    assert orc.rel_l2(q, w.q0()) < 0.5
