"""Error measures of the paper's experiments (Sec. 4), computed on the host from node values.

Relative l2 and l_inf errors; the dissipation and dispersion errors of Eqs. dissipation and
dispersion (a decomposition of the mean-square error into a part from the mean and the spread
of the field and a part from its correlation with the exact solution), divided by the
mean-square error as in the paper; and the mass error |(1/4pi) int (q - q_X) dS|. Surface
means use equal quadrature weights 4 pi / N over the quasi-uniform nodes (the paper uses a
kernel-based quadrature); with equal weights, dissipation + dispersion equals the mean-square
error exactly.
"""
from __future__ import annotations

import math

import numpy as np


def error_measures(qX: np.ndarray, q: np.ndarray) -> dict:
    """qX: numerical solution at the nodes; q: exact solution there (1-D arrays)."""
    qX = np.asarray(qX, dtype=np.float64).ravel()
    q = np.asarray(q, dtype=np.float64).ravel()
    d = qX - q
    mq, mx = q.mean(), qX.mean()
    sq = math.sqrt(np.mean((q - mq) ** 2))
    sx = math.sqrt(np.mean((qX - mx) ** 2))
    cov = float(np.mean((q - mq) * (qX - mx)))
    mse = float(np.mean(d * d))
    diss = (sq - sx) ** 2 + (mq - mx) ** 2
    disp = 2.0 * (sq * sx - cov)
    return {
        "l2": float(np.linalg.norm(d) / np.linalg.norm(q)),
        "linf": float(np.abs(d).max() / np.abs(q).max()),
        "dissipation": diss / mse if mse > 0 else 0.0,
        "dispersion": disp / mse if mse > 0 else 0.0,
        "mass": abs(float(d.mean())),
    }


def convergence_order(Ns, errs) -> float:
    """p in err ~ C N^(-p/2) (the paper plots against sqrt(N)), least squares over the points
    given, as in the paper's fits."""
    x = np.log(np.sqrt(np.asarray(Ns, dtype=np.float64)))
    y = np.log(np.asarray(errs, dtype=np.float64))
    return float(-np.polyfit(x, y, 1)[0])
