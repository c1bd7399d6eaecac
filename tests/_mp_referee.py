"""50-digit mpmath solve of a local stencil system (Eq. rbf_poly_linsys), the pin of the
long-double referee.

The augmentation functions are the spherical harmonics of degree <= ell written as polynomials
in (x, y, z) (Sec. 2.2; the form the oracle and the CUDA path both evaluate): up to a constant
factor per function, Q_l^m(z) Re (x + iy)^m and Q_l^m(z) Im (x + iy)^m with the polynomial
Q_l^m(z) = P_l^m(z) / (1 - z^2)^(m/2). Here P_l^m is mpmath's associated Legendre function
(legenp), an independent evaluation route; the per-function constants do not change the span,
so they leave the weights unchanged. Node coordinates are unit vectors only to FP64 rounding,
and at condition numbers near 1e18 the weights of this polynomial form and of the angular form
Y(theta(x), phi(x)) differ visibly, so the referee must use the same form.
"""
import mpmath
import numpy as np


def poly_harmonics(pt, ell):
    x, y, z = pt
    out = []
    w = 1 - z * z
    for l in range(ell + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            q = mpmath.legenp(l, am, z) / (w ** (mpmath.mpf(am) / 2)) if am else mpmath.legenp(l, 0, z)
            c = mpmath.mpc(x, y) ** am
            out.append(q * (mpmath.re(c) if m >= 0 else mpmath.im(c)))
    return out


def mp_weights(S, xi, ell, p, dps=50):
    """Weights of the stencil S (n x 3 FP64 nodes) at xi for the PHS r^p with harmonics of
    degree <= ell, from an mpmath LU solve at `dps` digits of the exact system."""
    mpmath.mp.dps = dps
    n = len(S)
    M = (ell + 1) ** 2
    m = n + M
    Sm = [[mpmath.mpf(float(v)) for v in row] for row in S]
    xm = [mpmath.mpf(float(v)) for v in xi]

    def phs(a, b):
        return mpmath.sqrt(sum((a[t] - b[t]) ** 2 for t in range(3))) ** p

    A = mpmath.matrix(m, m)
    b = mpmath.matrix(m, 1)
    for a in range(n):
        for c in range(n):
            A[a, c] = phs(Sm[a], Sm[c]) if a != c else 0
        Ya = poly_harmonics(Sm[a], ell)
        for c in range(M):
            A[a, n + c] = A[n + c, a] = Ya[c]
        b[a] = phs(xm, Sm[a])
    Yx = poly_harmonics(xm, ell)
    for c in range(M):
        b[n + c] = Yx[c]
    return np.array([float(v) for v in mpmath.lu_solve(A, b)[:n]])
