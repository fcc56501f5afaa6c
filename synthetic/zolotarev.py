"""Zolotarev-type 5th-dimension coefficients b_i, c_i (inputs, not the method).

The paper's Sec. 3 runs the operator with "Zolotarev coefficients": the
per-slice Mobius coefficients are chosen so that the 4D operator of App. A
(Eq. polar with Eq. argument) carries an optimal rational approximation of
the sign function.  With b_i - c_i = 1 every a_i X_i of Eq. argument shares
the kernel X = gamma5 D_w (2 + D_w)^-1 and the approximation reads

    R(x) = [prod_i (1 + a_i x) - prod_i (1 - a_i x)]
         / [prod_i (1 + a_i x) + prod_i (1 - a_i x)],    a_i = b_i + c_i,

an odd rational function of x with zeros of R(x) - 1 at x = 1/a_i.  The
coefficients below minimise max |R(x) - 1| over x in [xmin, xmax]; the
optimum is characterised by Ls + 1 alternating extrema of R - 1 of equal
size, endpoints included (Chebyshev equioscillation).  It is found with the
Remez exchange method (E. Ya. Remez, 1934): locate the extrema, then take a
Newton step on the equioscillation equations, repeat.

The paper used A. Kennedy's code for these numbers (Acknowledgment), which is
not available; any set of b_i, c_i is a valid input to both the CUDA path and
the oracle, so the exact values cannot affect parity.
"""
from __future__ import annotations

import numpy as np


def _err(x, z):
    """R(x) - 1 for zeros z_i = 1/a_i (vectorised in x)."""
    x = np.asarray(x, dtype=np.float64)
    rho = np.ones_like(x)
    for zi in z:
        a = 1.0 / zi
        rho = rho * (1.0 - a * x) / (1.0 + a * x)
    return -2.0 * rho / (1.0 + rho)


def _interval_extremum(lo, hi, z):
    """Point of largest |R - 1| on [lo, hi] (golden section in log x, plus ends)."""
    la, lb = np.log(lo), np.log(hi)
    grid = np.exp(np.linspace(la, lb, 65))
    v = np.abs(_err(grid, z))
    k = int(np.argmax(v))
    a = np.log(grid[max(k - 1, 0)])
    b = np.log(grid[min(k + 1, len(grid) - 1)])
    g = (np.sqrt(5.0) - 1.0) / 2.0
    c = b - g * (b - a)
    d = a + g * (b - a)
    fc = abs(_err(np.exp(c), z))
    fd = abs(_err(np.exp(d), z))
    for _ in range(80):
        if fc > fd:
            b, d, fd = d, c, fc
            c = b - g * (b - a)
            fc = abs(_err(np.exp(c), z))
        else:
            a, c, fc = c, d, fd
            d = a + g * (b - a)
            fd = abs(_err(np.exp(d), z))
    xm = np.exp(0.5 * (a + b))
    cands = [lo, hi, xm]
    vals = [abs(_err(p, z)) for p in cands]
    return cands[int(np.argmax(vals))]


def _extrema(z, xmin, xmax):
    edges = [xmin] + list(np.sort(z)) + [xmax]
    pts = []
    for j in range(len(edges) - 1):
        if j == 0:
            pts.append(xmin)
        elif j == len(edges) - 2:
            pts.append(xmax)
        else:
            pts.append(_interval_extremum(edges[j], edges[j + 1], z))
    return np.array(pts)


def zolotarev_sign_coefficients(Ls: int, xmin: float = 0.05, xmax: float = 6.0,
                                tol: float = 1e-13, max_iter: int = 200):
    """Return (a, delta): a_i > 0 (ascending) minimising max |R - 1| on [xmin, xmax].

    delta is the equal ripple max |R(x) - 1| of the optimum.
    """
    if Ls < 1 or not (0 < xmin < xmax):
        raise ValueError("need Ls >= 1 and 0 < xmin < xmax")
    u = (np.arange(Ls) + 0.5) / Ls
    logz = np.log(xmin) * (1.0 - u) + np.log(xmax) * u
    sgn = np.array([(-1.0) ** (j + 1) for j in range(Ls + 1)])  # e(xmin) < 0
    delta = None
    for _ in range(max_iter):
        z = np.exp(logz)
        pts = _extrema(z, xmin, xmax)
        e = _err(pts, z)
        delta = float(np.mean(np.abs(e)))
        spread = float(np.max(np.abs(e)) - np.min(np.abs(e)))
        if spread <= tol * delta:
            break
        # Newton on F(theta) = e(pts; z(theta)) - sgn * delta = 0, theta = (log z, delta)
        theta = np.concatenate([logz, [delta]])

        def F(th):
            return _err(pts, np.exp(th[:Ls])) - sgn * th[Ls]

        f0 = F(theta)
        J = np.empty((Ls + 1, Ls + 1))
        for k in range(Ls + 1):
            h = 1e-7 * max(1.0, abs(theta[k]))
            tp = theta.copy()
            tp[k] += h
            tm = theta.copy()
            tm[k] -= h
            J[:, k] = (F(tp) - F(tm)) / (2 * h)
        step = np.linalg.solve(J, -f0)
        lam = 1.0
        for _ls in range(30):
            cand = theta + lam * step
            zc = np.sort(np.exp(cand[:Ls]))
            if np.all(np.diff(np.log(zc)) > 0) and zc[0] > xmin and zc[-1] < xmax:
                break
            lam *= 0.5
        logz = np.sort(cand[:Ls])
    a = np.sort(1.0 / np.exp(logz))
    return a, delta


def concave_order(values):
    """Order ascending values so the smallest sit at s=1 and s=Ls, the largest at Ls/2.

    Sorted ascending, the values are placed alternately at positions
    1, Ls, 2, Ls-1, ... (paper Sec. 3: concave ordering of the coefficients).
    """
    v = np.sort(np.asarray(values, dtype=np.float64))
    n = len(v)
    out = np.empty(n)
    lo, hi = 0, n - 1
    for k in range(n):
        if k % 2 == 0:
            out[lo] = v[k]
            lo += 1
        else:
            out[hi] = v[k]
            hi -= 1
    return out


def zolotarev_mobius(Ls: int, xmin: float = 0.05, xmax: float = 6.0):
    """Per-slice Mobius coefficients b_i, c_i with b_i + c_i = a_i = 1/omega_i, b_i - c_i = 1.

    The a_i come from zolotarev_sign_coefficients and are concavely ordered.
    Returns (b, c, a_ordered, delta).
    """
    a, delta = zolotarev_sign_coefficients(Ls, xmin, xmax)
    a = concave_order(a)
    b = 0.5 * (a + 1.0)
    c = 0.5 * (a - 1.0)
    return b, c, a, delta
