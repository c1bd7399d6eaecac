"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module generates data only: node sets, velocity-field parameters and initial tracer
fields. It holds none of the transport method's arithmetic (no departure-point tracing, no
neighbour search, no RBF or spherical-harmonic evaluation), so that the CUDA path and the
CPU oracle can both read the same arrays without sharing method code.

Workloads follow the shapes of the paper's experiments (Sec. 4: quasi-uniform nodes with
h ~ 1/sqrt(N), C^1 cosine bells, Gaussian bells, smooth fields, solid-body rotation and a
reversing deformational flow). The paper's own node files (icosahedral / maximum-
determinant, Sec. 3.1) are replaced by Fibonacci-spiral nodes with a seeded tangential
jitter; the paper's smooth test fields are complemented by random plane-wave fields.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Velocity kinds (must match RBFSL_VEL_* in include/rbfsl.h).
VEL_RIGID = 0      # u = omega * (a x x): solid-body rotation about unit axis a
VEL_DEFORM_Y2 = 1  # u = x cross grad(psi), psi = kappa * y^2 * cos(pi t / T)
VEL_NL = 2         # the paper's deformational flow (Sec. 4.2), params {kappa, T}

SEED_BASE = 1804 * 100


def fibonacci_nodes(N: int) -> np.ndarray:
    """Fibonacci-spiral points on S^2 (N x 3, float64, row-major).

    z_i = 1 - (2i+1)/N, azimuth i * pi * (3 - sqrt 5): a quasi-uniform set with spacing
    h ~ 1/sqrt(N), standing in for the quasi-uniform node sets of Sec. 3.1.
    """
    i = np.arange(N, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / N
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    X = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
    return X / np.linalg.norm(X, axis=1, keepdims=True)


def jitter_nodes(X: np.ndarray, angle: float, rng: np.random.Generator) -> np.ndarray:
    """Move every node by exactly `angle` radians of arc along a random tangent direction."""
    g = rng.standard_normal(X.shape)
    t = g - np.sum(g * X, axis=1, keepdims=True) * X
    t /= np.linalg.norm(t, axis=1, keepdims=True)
    Y = math.cos(angle) * X + math.sin(angle) * t
    return np.ascontiguousarray(Y / np.linalg.norm(Y, axis=1, keepdims=True))


def nodes(N: int, seed: int, jitter: float = 1e-3) -> np.ndarray:
    """Seeded node set: Fibonacci spiral plus a tangential jitter of `jitter` rad."""
    X = fibonacci_nodes(N)
    if jitter > 0:
        X = jitter_nodes(X, jitter, np.random.default_rng(seed))
    return np.ascontiguousarray(X, dtype=np.float64)


def random_unit_vectors(k: int, rng: np.random.Generator) -> np.ndarray:
    v = rng.standard_normal((k, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


# ----------------------------------------------------------------------------- velocity
def rigid_rotation_params(axis, period: float = 1.0) -> np.ndarray:
    """[a_x, a_y, a_z, omega]: rotation about unit axis a with angular speed 2*pi/period."""
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    return np.array([a[0], a[1], a[2], 2.0 * math.pi / period], dtype=np.float64)


def tilted_axis(tilt: float) -> np.ndarray:
    """Unit axis tilted `tilt` rad from +z towards +x (azimuth 0)."""
    return np.array([math.sin(tilt), 0.0, math.cos(tilt)])


def deformation_params(kappa: float = 2.4, T: float = 1.0) -> np.ndarray:
    """[kappa, T] for psi = kappa * y^2 * cos(pi t / T)."""
    return np.array([kappa, T], dtype=np.float64)


def nl_deformation_params(T: float = 5.0) -> np.ndarray:
    """[kappa, T] of the paper's deformational flow (Sec. 4.2): kappa = 10 / T, T = 5."""
    return np.array([10.0 / T, T], dtype=np.float64)


def sbr_params(alpha: float = math.pi / 2) -> np.ndarray:
    """Solid-body rotation of the paper's first test (Sec. 4.1), one revolution per 2 pi, at
    angle alpha to the equator: rotation vector -(0, sin alpha, cos alpha) (at (1, 0, 0) the
    flow is northward for alpha = pi / 2)."""
    return rigid_rotation_params([0.0, -math.sin(alpha), -math.cos(alpha)], 2.0 * math.pi)


# ----------------------------------------------------------------------------- tracers
def cosine_bell(P: np.ndarray, center, radius: float, base: float = 0.0, amp: float = 1.0):
    """C^1 cosine bell 0.5*(1 + cos(pi r / R)) for great-circle distance r < R (Sec. 4.1)."""
    c = np.asarray(center, dtype=np.float64)
    r = np.arccos(np.clip(P @ c, -1.0, 1.0))
    q = np.where(r < radius, 0.5 * (1.0 + np.cos(math.pi * r / radius)), 0.0)
    return base + amp * q


def gaussian_hills(P: np.ndarray, centers, width: float = 5.0, amp: float = 0.95):
    """Sum of Gaussian bells amp * exp(-width * |x - p|^2) (Sec. 4.2, Gaussian bells)."""
    q = np.zeros(P.shape[0])
    for p in np.asarray(centers, dtype=np.float64).reshape(-1, 3):
        d = P - p
        q += amp * np.exp(-width * np.sum(d * d, axis=1))
    return q


@dataclass
class PlaneWaveField:
    """q(x) = scale * sum_k a_k cos(k . x + phase_k), |k| <= kmax: a smooth random field."""
    wavevectors: np.ndarray  # (K, 3)
    amplitudes: np.ndarray   # (K,)
    phases: np.ndarray       # (K,)
    scale: float = 1.0

    def __call__(self, P: np.ndarray) -> np.ndarray:
        arg = P @ self.wavevectors.T + self.phases[None, :]
        return self.scale * (np.cos(arg) @ self.amplitudes)


def plane_wave_field(rng: np.random.Generator, kmax: float, nwaves: int = 8) -> PlaneWaveField:
    dirs = random_unit_vectors(nwaves, rng)
    mags = kmax * rng.random(nwaves) ** (1.0 / 3.0)
    return PlaneWaveField(dirs * mags[:, None], rng.standard_normal(nwaves),
                          rng.uniform(0, 2 * math.pi, nwaves))


@dataclass
class TracerSet:
    """Initial tracer fields, evaluable at any points (for exact solutions)."""
    fns: list = field(default_factory=list)

    def __call__(self, P: np.ndarray) -> np.ndarray:
        """(len(P), T) float64, tracer-minor."""
        return np.ascontiguousarray(np.stack([f(P) for f in self.fns], axis=1))

    @property
    def T(self) -> int:
        return len(self.fns)


def _normalised(fn, X):
    """Scale a field so that max|q| over the nodes is 1."""
    s = 1.0 / np.max(np.abs(fn(X)))
    if isinstance(fn, PlaneWaveField):
        fn.scale = s
        return fn
    return lambda P, fn=fn, s=s: s * fn(P)


# ----------------------------------------------------------------------------- configs
@dataclass
class Workload:
    name: str
    N: int
    X: np.ndarray
    method: str            # "local" | "global" | "pu"
    n: int = 0             # stencil size (local) or nodes per patch (PU)
    ell: int = 0           # spherical-harmonic degree
    power: int = 3         # PHS exponent 2k+1 (local / PU)
    eps: float = 0.0       # Gaussian shape (global)
    vel_kind: int = VEL_RIGID
    vel_params: np.ndarray = None
    steps: int = 1
    dt: float = 1.0
    tracers: TracerSet = None
    seed: int = 0
    pu_overlap: float = 2.5

    @property
    def T(self) -> int:
        return self.tracers.T

    def q0(self) -> np.ndarray:
        return self.tracers(self.X)


def config_local_rotation(N: int = 2562, n: int = 31, ell: int = 2, power: int = 3,
                          steps: int = 120, seed: int = SEED_BASE + 1) -> Workload:
    """Solid-body rotation of a cosine bell (radius 0.5 rad) about an axis tilted 0.3 rad from z,
    period 1, one revolution in `steps` RK4 steps; local stencils n=31, r^3, SH degree 2."""
    rng = np.random.default_rng(seed)
    X = nodes(N, seed)
    c = random_unit_vectors(1, rng)[0]
    tr = TracerSet([lambda P, c=c: cosine_bell(P, c, 0.5)])
    return Workload(f"local-rotation N={N} n={n} ell={ell} r^{power}", N, X, "local", n=n, ell=ell,
                    power=power, vel_kind=VEL_RIGID,
                    vel_params=rigid_rotation_params(tilted_axis(0.3), 1.0),
                    steps=steps, dt=1.0 / steps, tracers=tr, seed=seed)


def config_local_deformation(N: int = 40962, n: int = 84, ell: int = 4, power: int = 9,
                             steps: int = 600, n_random: int = 31, kmax: float = 8.0,
                             seed: int = SEED_BASE + 2) -> Workload:
    """Reversing deformational flow psi = 2.4 y^2 cos(pi t), T = 1 over `steps` steps;
    tracers: two seeded Gaussian hills (width 5) plus `n_random` smooth random fields.

    The PHS exponent follows the paper's rule k = L (Sec. 2.4): r^(2L+1) = r^9 for L = 4.
    With r^5 at N = 40962, n = 84 the FP64 iteration diverges within tens of steps (both the
    CPU oracle and the GPU path), while r^9 returns the field to ~2e-7."""
    rng = np.random.default_rng(seed)
    X = nodes(N, seed)
    hills = random_unit_vectors(2, rng)
    fns = [lambda P, h=hills: gaussian_hills(P, h, 5.0, 0.95)]
    for _ in range(n_random):
        fns.append(_normalised(plane_wave_field(rng, kmax), X))
    return Workload(f"local-deformation N={N} n={n} ell={ell} r^{power} T={1 + n_random}", N, X,
                    "local", n=n, ell=ell, power=power, vel_kind=VEL_DEFORM_Y2,
                    vel_params=deformation_params(2.4, 1.0), steps=steps, dt=1.0 / steps,
                    tracers=TracerSet(fns), seed=seed)


def config_global_rotation(N: int = 10242, eps: float = 6.0, steps: int = 200, T: int = 64,
                           kmax: float = 16.0, seed: int = SEED_BASE + 3) -> Workload:
    """Global Gaussian RBF, shape eps = 6, same tilted rotation over `steps` steps, T smooth
    random fields."""
    rng = np.random.default_rng(seed)
    X = nodes(N, seed)
    fns = [_normalised(plane_wave_field(rng, kmax), X) for _ in range(T)]
    return Workload(f"global-rotation N={N} eps={eps} T={T}", N, X, "global", eps=eps,
                    vel_kind=VEL_RIGID, vel_params=rigid_rotation_params(tilted_axis(0.3), 1.0),
                    steps=steps, dt=1.0 / steps, tracers=TracerSet(fns), seed=seed)


def config_pu_rotation(N: int = 10242, n: int = 100, ell: int = 3, power: int = 7,
                       steps: int = 100, seed: int = SEED_BASE + 5) -> Workload:
    """RBF-PU on a tilted rotation: patches of ~n nodes, overlap a = 2.5, SH degree 3."""
    rng = np.random.default_rng(seed)
    X = nodes(N, seed)
    c = random_unit_vectors(2, rng)
    tr = TracerSet([lambda P, c=c[0]: cosine_bell(P, c, 0.5),
                    lambda P, h=c[1:]: gaussian_hills(P, h, 5.0, 0.95)])
    return Workload(f"pu-rotation N={N} n={n} ell={ell} r^{power}", N, X, "pu", n=n, ell=ell,
                    power=power, vel_kind=VEL_RIGID,
                    vel_params=rigid_rotation_params(tilted_axis(0.3), 1.0),
                    steps=steps, dt=1.0 / steps, tracers=tr, seed=seed)


# The paper's test cases (Sec. 4) on the Fibonacci node sets that stand in for its node files.
PAPER_P1 = (math.sqrt(3.0) / 2.0, 0.5, 0.0)
PAPER_P2 = (math.sqrt(3.0) / 2.0, -0.5, 0.0)


def config_sbr(N: int, method: str = "local", n: int = 31, ell: int = -1, power: int = -1,
               steps: int = 20, revolutions: int = 1, eps: float = 0.0,
               seed: int = SEED_BASE + 6) -> Workload:
    """Solid-body rotation of the cosine bell of Sec. 4.1: alpha = pi / 2, bell of radius 1/3 at
    (1, 0, 0), final time 2 pi per revolution, dt = pi / 10 (20 steps per revolution). ell and
    power default to the paper's rules (ell = floor((sqrt(n) - 1) / 2), r^(2 ell + 1))."""
    X = nodes(N, seed)
    if ell < 0:
        ell = int(math.floor(0.5 * (math.sqrt(n) - 1.0)))
    if power < 0:
        power = 2 * ell + 1
    tr = TracerSet([lambda P: cosine_bell(P, (1.0, 0.0, 0.0), 1.0 / 3.0)])
    total = steps * revolutions
    return Workload(f"sbr-cosine-bell N={N} {method} n={n}", N, X, method, n=n, ell=ell, power=power,
                    eps=eps, vel_kind=VEL_RIGID, vel_params=sbr_params(), steps=total,
                    dt=2.0 * math.pi / steps, tracers=tr, seed=seed)


def config_nl(N: int, ic: str = "cosine", method: str = "local", n: int = 31, ell: int = -1,
              power: int = -1, steps: int = 50, eps: float = 0.0, seed: int = SEED_BASE + 7) -> Workload:
    """Deformational flow of Sec. 4.2 (T = 5, dt = 1/10 by default) with the paper's two cosine
    bells (0.1 + 0.9 (q1 + q2), radius 1/2) or two Gaussian bells (0.95 exp(-5 |x - p|^2)) at
    p1, p2 = (sqrt(3)/2, +-1/2, 0); the exact solution at t = T is the initial field."""
    X = nodes(N, seed)
    if ell < 0:
        ell = int(math.floor(0.5 * (math.sqrt(n) - 1.0)))
    if power < 0:
        power = 2 * ell + 1
    if ic == "cosine":
        fn = lambda P: 0.1 + 0.9 * (cosine_bell(P, PAPER_P1, 0.5) + cosine_bell(P, PAPER_P2, 0.5))
    else:
        fn = lambda P: gaussian_hills(P, [PAPER_P1, PAPER_P2], 5.0, 0.95)
    return Workload(f"nl-deformation-{ic} N={N} {method} n={n}", N, X, method, n=n, ell=ell,
                    power=power, eps=eps, vel_kind=VEL_NL, vel_params=nl_deformation_params(5.0),
                    steps=steps, dt=5.0 / steps, tracers=TracerSet([fn]), seed=seed)


def batched_problems(P: int = 64, seed: int = SEED_BASE + 4, Ns=(2562, 10242, 40962, 163842)):
    """Descriptors of P independent local problems: N from Ns, (n, ell) from
    {(31,2),(55,3),(84,4)}, 1..16 tracers, each with its own tilted rotation or deformation
    field (seeded parameters)."""
    rng = np.random.default_rng(seed)
    out = []
    for p in range(P):
        N = int(rng.choice(list(Ns)))
        n, ell = [(31, 2), (55, 3), (84, 4)][int(rng.integers(0, 3))]
        T = int(rng.integers(1, 17))
        if rng.random() < 0.5:
            vk, vp = VEL_RIGID, rigid_rotation_params(random_unit_vectors(1, rng)[0],
                                                      float(rng.uniform(0.5, 2.0)))
        else:
            vk, vp = VEL_DEFORM_Y2, deformation_params(float(rng.uniform(1.5, 2.5)), 1.0)
        # PHS exponent by the paper's rule k = L (Sec. 2.4): r^(2 ell + 1)
        out.append(dict(N=N, n=n, ell=ell, power=2 * ell + 1, T=T, vel_kind=vk,
                        vel_params=vp, seed=int(seed * 1000 + p)))
    return out
