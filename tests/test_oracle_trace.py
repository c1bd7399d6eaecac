"""Pins for the oracle's velocity fields and RK4 departure-point tracer (Sec. 3.2, Eq. sl_ode).

Independent checks: the velocity fields against their definitions (numpy cross products,
finite-difference gradient of the stream function), the closed-form flow maps against the
ODE itself (finite differences), and the RK4 tracer against the closed forms with its
fifth-order local error.
"""
import math

import numpy as np
import pytest

from paper_1804_01609_gb300 import inputs


def _rigid():
    return inputs.rigid_rotation_params(inputs.tilted_axis(0.3), 1.0)


def _deform():
    return inputs.deformation_params(2.4, 1.0)


def test_rigid_velocity_is_omega_cross_x(orc):
    X = inputs.nodes(200, 7)
    prm = _rigid()
    for x in X[:20]:
        u = orc.velocity(0, prm, x, 0.3)
        np.testing.assert_allclose(u, prm[3] * np.cross(prm[:3], x), atol=1e-15)
        assert abs(u @ x) < 1e-14


def test_deformation_velocity_is_x_cross_grad_psi(orc):
    """u = x cross grad(psi), psi = kappa y^2 cos(pi t / T): gradient by central differences."""
    kappa, T = 2.4, 1.0
    prm = _deform()
    psi = lambda p, t: kappa * p[1] ** 2 * math.cos(math.pi * t / T)
    X = inputs.nodes(100, 3)
    h = 1e-6
    for x in X[:15]:
        for t in (0.0, 0.37, 0.8):
            g = np.array([(psi(x + h * e, t) - psi(x - h * e, t)) / (2 * h) for e in np.eye(3)])
            u = orc.velocity(1, prm, x, t)
            np.testing.assert_allclose(u, np.cross(x, g), atol=1e-8)
            assert abs(u @ x) < 1e-14


@pytest.mark.parametrize("kind", [0, 1])
def test_exact_flow_map_solves_the_ode(orc, kind):
    """d/dt0 of the closed-form departure map at t0 = t1 equals u(x, t1); and the map
    composes: (t2 -> t1) then (t1 -> t0) equals (t2 -> t0)."""
    prm = _rigid() if kind == 0 else _deform()
    X = inputs.nodes(300, 11)
    t1, h = 0.41, 1e-5
    fd = (orc.exact_departure(X, kind, prm, t1 + h, t1) - orc.exact_departure(X, kind, prm, t1 - h, t1)) / (2 * h)
    u = np.stack([orc.velocity(kind, prm, x, t1) for x in X])
    np.testing.assert_allclose(fd, u, atol=1e-8)
    a = orc.exact_departure(orc.exact_departure(X, kind, prm, 0.3, 0.55), kind, prm, 0.1, 0.3)
    b = orc.exact_departure(X, kind, prm, 0.1, 0.55)
    np.testing.assert_allclose(a, b, atol=1e-14)
    np.testing.assert_allclose(np.linalg.norm(b, axis=1), 1.0, atol=1e-15)


@pytest.mark.parametrize("kind", [0, 1])
def test_rk4_matches_closed_form_with_fifth_order_local_error(orc, kind):
    prm = _rigid() if kind == 0 else _deform()
    X = inputs.nodes(2562, 5)
    errs = []
    for S in (30, 60, 120):
        dt = 1.0 / S
        t1 = 0.2 + dt  # away from t = 0.5, where the deformation field vanishes
        Xi = orc.trace_rk4(X, kind, prm, t1, dt)
        ex = orc.exact_departure(X, kind, prm, t1 - dt, t1)
        errs.append(np.abs(Xi - ex).max())
        np.testing.assert_allclose(np.linalg.norm(Xi, axis=1), 1.0, atol=2e-16 * 4)
    # local error O(dt^5): halving dt divides it by ~32
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 20 < r1 < 45 and 20 < r2 < 45, errs
    if kind == 0:
        theta = prm[3] / 120
        assert errs[2] < theta ** 5 / 60


@pytest.mark.parametrize("kind", [0, 1])
def test_tracer_returns_after_one_period(orc, kind):
    """Composing S backward steps over [0, 1] returns every node to itself: a full
    revolution for the rotation, the reversal at t = T for the deformation."""
    prm = _rigid() if kind == 0 else _deform()
    X = inputs.nodes(500, 9)
    S = 120
    dt = 1.0 / S
    P = X.copy()
    for m in range(S, 0, -1):  # follow the parcel at X back from t = 1 to t = 0
        P = orc.trace_rk4(P, kind, prm, m * dt, dt)
    bound = 5e-7 if kind == 0 else 1e-5
    assert np.abs(P - X).max() < bound


@pytest.mark.parametrize("kind", [0, 1])
def test_rk5_matches_closed_form_with_sixth_order_local_error(orc, kind):
    """Fehlberg's fifth-order formula (Sec. 3.2): local error O(dt^6) against the closed-form
    flow maps (halving dt divides it by ~64), and well below the RK4 step's error. A wrong
    tableau entry breaks the order."""
    prm = _rigid() if kind == 0 else _deform()
    X = inputs.nodes(2562, 5)
    errs = []
    for S in (30, 60, 120):
        dt = 1.0 / S
        t1 = 0.2 + dt
        ex = orc.exact_departure(X, kind, prm, t1 - dt, t1)
        Xi = orc.trace_rk5(X, kind, prm, t1, dt)
        errs.append(np.abs(Xi - ex).max())
        assert errs[-1] < np.abs(orc.trace_rk4(X, kind, prm, t1, dt) - ex).max() / 10
        np.testing.assert_allclose(np.linalg.norm(Xi, axis=1), 1.0, atol=2e-16 * 4)
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 45 < r1 < 85 and 45 < r2 < 85, errs


@pytest.mark.parametrize("kind", [0, 1])
def test_rk5_tracer_returns_after_one_period(orc, kind):
    prm = _rigid() if kind == 0 else _deform()
    X = inputs.nodes(500, 9)
    S = 120
    dt = 1.0 / S
    P = X.copy()
    for m in range(S, 0, -1):
        P = orc.trace_rk5(P, kind, prm, m * dt, dt)
    bound = 1e-8 if kind == 0 else 1e-7
    assert np.abs(P - X).max() < bound
