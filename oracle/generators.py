"""1D Toeplitz generators of the Kronecker factors (oracle; test infrastructure only).

Eq. sep_integrands defines, for a node tau and axis p with cell size h_p,

    p != q:  int_{I_j} exp(-tau^2 (xi_i - y)^2) dy
    p == q:  int_{I_j} (xi_i - y) exp(-tau^2 (xi_i - y)^2) dy,

and Sec. 4.2 (the display before Eq. conv_op) shows that on a uniform grid
with midpoint collocation they depend on d = i - j only, with
x = xi_i - y running over [a_d, b_d] = [d h - h/2, d h + h/2].  The closed
forms are the ones of Eq. f_anal:

    E[d] = int_{a_d}^{b_d} exp(-tau^2 x^2) dx
         = sqrt(pi)/(2 tau) (erf(tau b_d) - erf(tau a_d))
    F[d] = int_{a_d}^{b_d} x exp(-tau^2 x^2) dx
         = (exp(-tau^2 a_d^2) - exp(-tau^2 b_d^2)) / (2 tau^2).

E is even and F odd in d, F[0] = 0.  The erf difference cancels when both
arguments are in the tail (large tau; Lemma 2 discusses this tail), so it is
evaluated there through erfc, which is the same number.  The F difference is
written e^{-tau^2 a^2} (1 - e^{-tau^2 (b^2 - a^2)}) with b^2 - a^2 = 2|d|h^2,
evaluated with expm1.  Arrays are indexed by d + n - 1, d = -(n-1)..n-1.
"""
from __future__ import annotations

import numpy as np
from scipy import special


def scaled_spacing(n, h):
    """Scale the domain so that its longest edge is 1 (Sec. 3.4, rho_max = 3).

    Returns (s, hh) with s = max_p n_p h_p and hh_p = h_p / s.  The collocation
    matrix entries of Eq. matrix_op scale linearly with length, so
    phi(original) = s * phi(scaled).
    """
    n = np.asarray(n, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    s = float(np.max(n * h))
    return s, h / s


def gen_E(tau: float, hh: float, n: int) -> np.ndarray:
    """E[d], d = -(n-1)..n-1, for one node tau and scaled cell size hh."""
    d = np.abs(np.arange(-(n - 1), n, dtype=np.float64))
    a = (d - 0.5) * hh
    b = (d + 0.5) * hh
    out = np.empty_like(d)
    centre = d == 0
    # d = 0: the interval is symmetric, [-hh/2, hh/2].
    out[centre] = np.sqrt(np.pi) / tau * special.erf(0.5 * tau * hh)
    far = ~centre
    ta, tb = tau * a[far], tau * b[far]
    tail = ta > 1.0
    diff = np.where(tail, special.erfc(ta) - special.erfc(tb), special.erf(tb) - special.erf(ta))
    out[far] = 0.5 * np.sqrt(np.pi) / tau * diff
    return out


def gen_F(tau: float, hh: float, n: int) -> np.ndarray:
    """F[d], d = -(n-1)..n-1, for one node tau and scaled cell size hh."""
    dd = np.arange(-(n - 1), n, dtype=np.float64)
    d = np.abs(dd)
    a = (d - 0.5) * hh
    t2 = tau * tau
    mag = np.exp(-t2 * a * a) * (-np.expm1(-2.0 * d * t2 * hh * hh)) / (2.0 * t2)
    return np.sign(dd) * mag


def toeplitz(gen: np.ndarray, n: int) -> np.ndarray:
    """Dense n x n matrix T[i, j] = gen[i - j] from a generator indexed by d + n - 1."""
    i = np.arange(n)
    return gen[(i[:, None] - i[None, :]) + n - 1]
