"""Pins for the oracle's velocity fields of the paper's test cases (Sec. 4).

Solid-body rotation (Sec. 4.1): the paper's spherical (u, v) at angle alpha, converted to
Cartesian here, equals the rigid rotation of inputs.sbr_params.
Deformational flow (Sec. 4.2, velocity kind 2): the oracle evaluates the paper's spherical
formula; it is pinned by (a) x cross grad(psi) for the stream function
psi = kappa cos(pi t/T) (y cos c - x sin c)^2 - (2 pi / T) z, c = 2 pi t / T, with grad(psi) by
central differences, (b) tangency, (c) pure rotation about z at t = T/2 where the deformation
vanishes, (d) hand-evaluated values (tests/golden/nl_velocity.txt), (e) the flow map over [0, T]
returning to the identity at fourth order in dt.
"""
import math
import os

import numpy as np

from paper_1804_01609_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
NL = 2


def _paper_sbr_velocity(P, alpha):
    lam = np.arctan2(P[:, 1], P[:, 0])
    th = np.arcsin(np.clip(P[:, 2], -1, 1))
    u = np.sin(th) * np.sin(lam) * np.sin(alpha) - np.cos(th) * np.cos(alpha)
    v = np.cos(lam) * np.sin(alpha)
    el = np.stack([-np.sin(lam), np.cos(lam), np.zeros_like(lam)], 1)
    et = np.stack([-np.sin(th) * np.cos(lam), -np.sin(th) * np.sin(lam), np.cos(th)], 1)
    return u[:, None] * el + v[:, None] * et


def test_sbr_rotation_is_the_papers_field(orc):
    P = inputs.random_unit_vectors(50, np.random.default_rng(4))
    for alpha in (math.pi / 2, 0.0, 0.7):
        prm = inputs.sbr_params(alpha)
        U = np.array([orc.velocity(0, prm, p, 0.0) for p in P])
        np.testing.assert_allclose(U, _paper_sbr_velocity(P, alpha), atol=1e-14)
    assert np.allclose(orc.velocity(0, inputs.sbr_params(), [1.0, 0.0, 0.0], 0.0), [0, 0, 1], atol=1e-15)


def _psi(P, kappa, T, t):
    c = 2 * math.pi * t / T
    b = P[..., 1] * math.cos(c) - P[..., 0] * math.sin(c)
    return kappa * math.cos(math.pi * t / T) * b * b - 2 * math.pi / T * P[..., 2]


def test_nl_field_is_x_cross_grad_psi(orc):
    kappa, T = inputs.nl_deformation_params(5.0)
    P = inputs.random_unit_vectors(40, np.random.default_rng(5))
    h = 1e-5
    for t in (0.0, 0.7, 2.5, 3.9):
        for p in P:
            g = np.array([(_psi(p + h * e, kappa, T, t) - _psi(p - h * e, kappa, T, t)) / (2 * h)
                          for e in np.eye(3)])
            u = orc.velocity(NL, [kappa, T], p, t)
            np.testing.assert_allclose(u, np.cross(p, g), atol=1e-8)
            assert abs(u @ p) < 1e-14


def test_nl_field_at_half_period_is_a_rotation(orc):
    kappa, T = inputs.nl_deformation_params(5.0)
    for p in inputs.random_unit_vectors(20, np.random.default_rng(6)):
        u = orc.velocity(NL, [kappa, T], p, T / 2)
        np.testing.assert_allclose(u, 2 * math.pi / T * np.array([-p[1], p[0], 0.0]), atol=1e-14)


def test_nl_field_golden_values(orc):
    kappa, T = inputs.nl_deformation_params(5.0)
    rows = [l.split() for l in open(os.path.join(GOLDEN, "nl_velocity.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 4
    for lam_s, th_s, t_s, *U in rows:
        lam, th, t = (eval(s, {"pi": math.pi}) for s in (lam_s, th_s, t_s))
        p = [math.cos(th) * math.cos(lam), math.cos(th) * math.sin(lam), math.sin(th)]
        np.testing.assert_allclose(orc.velocity(NL, [kappa, T], p, t), [float(v) for v in U], atol=1e-14)


def test_nl_flow_returns_at_the_final_time(orc):
    """Tracing every node back from t = T to 0 lands on the node (the flow reverses at T/2 while
    the background makes one revolution); the error falls ~16x when dt halves (RK4)."""
    X = inputs.nodes(642, 3)
    prm = inputs.nl_deformation_params(5.0)
    errs = []
    for S in (50, 100):
        dt = 5.0 / S
        P = X.copy()
        for m in range(S, 0, -1):
            P = orc.trace_rk4(P, NL, prm, m * dt, dt)
        errs.append(np.abs(P - X).max())
    assert errs[1] < 1e-4
    assert 10 < errs[0] / errs[1] < 24


def test_error_measures_decompose_the_mean_square_error():
    """Eqs. dissipation + dispersion add up to the mean-square error (with equal weights);
    a shifted copy is pure dissipation, a scaled copy about the mean keeps the correlation."""
    from paper_1804_01609_gb300 import diagnostics
    rng = np.random.default_rng(8)
    q = rng.standard_normal(1000)
    qX = q + 0.1 * rng.standard_normal(1000)
    m = diagnostics.error_measures(qX, q)
    assert abs(m["dissipation"] + m["dispersion"] - 1.0) < 1e-12
    m = diagnostics.error_measures(q + 0.25, q)
    assert abs(m["dissipation"] - 1.0) < 1e-12 and abs(m["dispersion"]) < 1e-12
    assert abs(m["mass"] - 0.25) < 1e-15
    m = diagnostics.error_measures(q.mean() + 1.5 * (q - q.mean()), q)
    assert abs(m["dispersion"]) < 1e-12 and abs(m["mass"]) < 1e-13
    assert diagnostics.error_measures(q, q)["l2"] == 0.0
    Ns = [2562, 10242, 40962]
    assert abs(diagnostics.convergence_order(Ns, [3.0 * N ** -2.0 for N in Ns]) - 4.0) < 1e-12
