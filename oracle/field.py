"""Stray field from analytic derivative factors (oracle; test infrastructure only).

h_d = -grad phi at the collocation points, without finite differences.  In
the Kronecker form of phi (Cor. 3, Eq. kron_operator) the collocation point
xi enters each 1D factor only through the limits of its cell integral,
T[d] = int_{xi - y_hi}^{xi - y_lo} f(x) dx, so d/dxi_p acts on the axis-p
factor alone and replaces it by f(b_d) - f(a_d) (a_d, b_d as in generators):

    f(x) = exp(-tau^2 x^2)       ->  dE[d] = exp(-tau^2 b^2) - exp(-tau^2 a^2) = -2 tau^2 F[d]
    f(x) = x exp(-tau^2 x^2)     ->  dF[d] = b exp(-tau^2 b^2) - a exp(-tau^2 a^2)

(the derivative relations of the cell integrals behind the analytic stray
field).  dE is odd and dF even in d.  With the domain scaled by s (Sec. 3.4),
d/dxi_phys = (1/s) d/dxi_scaled, so the field carries c omega_k without the
factor s of phi.  dF is evaluated as exp(-tau^2 a^2) (h + b expm1(-2 |d| tau^2 h^2))
for |d| >= 1, which avoids the cancellation of the two exponentials.
"""
from __future__ import annotations

import numpy as np

from .full import mode_product, C_POT, factor_kind
from .generators import gen_E, gen_F, scaled_spacing, toeplitz
from .quadrature import sinc_nodes


def gen_dE(tau: float, hh: float, n: int) -> np.ndarray:
    """d/dxi of E[d] (scaled coordinates), d = -(n-1)..n-1."""
    return -2.0 * tau * tau * gen_F(tau, hh, n)


def gen_dF(tau: float, hh: float, n: int) -> np.ndarray:
    """d/dxi of F[d] (scaled coordinates), d = -(n-1)..n-1 (even in d)."""
    d = np.abs(np.arange(-(n - 1), n, dtype=np.float64))
    a = (d - 0.5) * hh
    b = (d + 0.5) * hh
    t2 = tau * tau
    out = np.exp(-t2 * a * a) * (hh + b * np.expm1(-2.0 * d * t2 * hh * hh))
    centre = d == 0
    out[centre] = hh * np.exp(-t2 * hh * hh / 4.0)
    return out


def apply_field(m: np.ndarray, n, h, R: int, c0: float = 2.15) -> np.ndarray:
    """h_d[p] = -d phi / d xi_p at the cell centres, p = 1..3: float64 [3, n3, n2, n1].

    For each direction p the Kronecker sum of apply_full with the axis-p factor
    of every term replaced by its derivative (dE for E, dF for F).
    """
    n = tuple(int(v) for v in n)
    m = np.asarray(m, dtype=np.float64)
    if R < 5 or R % 2 == 0:
        raise ValueError("R must be odd and >= 5")
    M = (R - 1) // 2
    _, hh = scaled_spacing(n, h)
    _, _, tau, omega = sinc_nodes(M, c0)
    hd = np.zeros((3, n[2], n[1], n[0]))
    for k in range(M):
        T = {}
        for p in range(3):
            T[(p, "E")] = toeplitz(gen_E(tau[k], hh[p], n[p]), n[p])
            T[(p, "F")] = toeplitz(gen_F(tau[k], hh[p], n[p]), n[p])
            T[(p, "dE")] = toeplitz(gen_dE(tau[k], hh[p], n[p]), n[p])
            T[(p, "dF")] = toeplitz(gen_dF(tau[k], hh[p], n[p]), n[p])
        for direction in range(3):
            acc = np.zeros((n[2], n[1], n[0]))
            for q in range(3):
                X = m[q]
                for p in range(3):
                    kind = factor_kind(p, q)
                    if p == direction:
                        kind = "d" + kind
                    X = mode_product(X, T[(p, kind)], p + 1)
                acc += X
            hd[direction] -= omega[k] * acc
    return C_POT * hd
