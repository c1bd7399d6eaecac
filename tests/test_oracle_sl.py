"""End-to-end pins of the oracle's SL loop (Algorithm 1): after a full revolution of a rigid
rotation, or at the reversal time of the deformational flow, the exact solution is the
initial field, and the error must shrink as N grows (Sec. 4: the methods converge)."""
import math

import numpy as np
import pytest

from paper_1804_01609_gb300 import inputs


def _hills(P):
    return inputs.gaussian_hills(P, [[0.0, 0.6, 0.8], [0.8, -0.6, 0.0]], 5.0, 0.95)


@pytest.mark.parametrize("mode", [0, 1])
def test_local_rotation_converges(orc, mode):
    prm = inputs.rigid_rotation_params(inputs.tilted_axis(0.3), 1.0)
    errs = []
    for N in (642, 2562):
        X = inputs.nodes(N, 1)
        q0 = _hills(X)
        q = orc.local_run(X, q0, 31, 2, 3, 0, prm, 1.0 / 24, 24, mode=mode)
        errs.append(orc.rel_l2(q, q0))
    assert errs[1] < errs[0] / 3, errs
    assert errs[1] < 5e-3, errs


def test_local_deformation_returns(orc):
    prm = inputs.deformation_params(2.4, 1.0)
    X = inputs.nodes(2562, 2)
    q0 = _hills(X)
    q = orc.local_run(X, q0, 31, 2, 3, 1, prm, 1.0 / 30, 30)
    assert orc.rel_l2(q, q0) < 2e-2


def test_global_rotation_returns(orc):
    prm = inputs.rigid_rotation_params(inputs.tilted_axis(0.3), 1.0)
    X = inputs.nodes(642, 3)
    q0 = _hills(X)
    G = orc.GlobalInterpolator(X, orc.GAUSS, 6.0)
    q = q0.copy()
    S = 12
    for m in range(S):
        q = G.apply(orc.trace_rk4(X, 0, prm, (m + 1) / S, 1.0 / S), q)
    assert orc.rel_l2(q, q0) < 5e-3


def test_pu_rotation_returns(orc):
    prm = inputs.rigid_rotation_params(inputs.tilted_axis(0.3), 1.0)
    N, n = 2562, 60
    X = inputs.nodes(N, 3)
    pu = orc.PUInterpolator(X, inputs.fibonacci_nodes(math.ceil(2.5 * N / n)), n, 3, 7)
    q0 = _hills(X)
    q = q0.copy()
    S = 12
    for m in range(S):
        q = pu.apply(orc.trace_rk4(X, 0, prm, (m + 1) / S, 1.0 / S), q)
    assert orc.rel_l2(q, q0) < 5e-3
