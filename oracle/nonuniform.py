"""The Kronecker operator on a non-uniform tensor grid (oracle; test infrastructure only).

Sec. 3.1 (Notation) lets each axis be partitioned into arbitrary sub-intervals
I_j = [y_j, y_{j+1}] with collocation at the midpoints xi_i; Eq. sep_integrands
and Cor. 3 (Eq. kron_operator) then give, per node tau_k, dense (no longer
Toeplitz) factor matrices

    E[i, j] = int_{I_j} exp(-tau^2 (xi_i - y)^2) dy = int_a^b exp(-tau^2 x^2) dx
    F[i, j] = int_{I_j} (xi_i - y) exp(-tau^2 (xi_i - y)^2) dy = int_a^b x exp(-tau^2 x^2) dx

with a = xi_i - y_{j+1} < b = xi_i - y_j, and phi = c s sum_k omega_k
sum_q U3 (x) U2 (x) U1 m^(q) exactly as in oracle.full.  The domain is scaled
by s = the longest edge (beta_p - alpha_p), as on uniform grids.

Closed forms (the same integrals as the uniform generators, general limits):
  E = sqrt(pi)/(2 tau) (erf(tau b) - erf(tau a)), through erfc when both
      limits lie in the same tail; E(a, b) = E(-b, -a).
  F = (exp(-tau^2 a^2) - exp(-tau^2 b^2)) / (2 tau^2), written
      exp(-tau^2 a^2) (-expm1(-tau^2 (b - a)(b + a))) / (2 tau^2) for 0 <= a;
      F(a, b) = -F(-b, -a).
The transposes are no longer -F and E (the cell widths differ), so the adjoint
is formed with explicit transposes.
"""
from __future__ import annotations

import numpy as np
from scipy import special

from .full import C_POT, factor_kind, mode_product
from .quadrature import sinc_nodes


def _E(tau, a, b):
    """int_a^b exp(-tau^2 x^2) dx for arrays a < b."""
    a, b = np.broadcast_arrays(np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64))
    neg = b <= 0  # both limits <= 0: mirror
    lo = np.where(neg, -b, a)
    hi = np.where(neg, -a, b)
    tl, th = tau * lo, tau * hi
    tail = tl > 1.0
    diff = np.where(tail, special.erfc(tl) - special.erfc(th), special.erf(th) - special.erf(tl))
    return 0.5 * np.sqrt(np.pi) / tau * diff


def _F(tau, a, b):
    """int_a^b x exp(-tau^2 x^2) dx for arrays a < b."""
    a, b = np.broadcast_arrays(np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64))
    t2 = tau * tau
    neg = b <= 0
    lo = np.where(neg, -b, a)
    hi = np.where(neg, -a, b)
    straddle = lo < 0
    lc = np.maximum(lo, 0.0)  # (the same-sign form is used only where lo >= 0)
    same = np.exp(-t2 * lc * lc) * (-np.expm1(-t2 * (hi - lc) * (hi + lc))) / (2.0 * t2)
    cross = (np.exp(-t2 * lo * lo) - np.exp(-t2 * hi * hi)) / (2.0 * t2)
    val = np.where(straddle, cross, same)
    return np.where(neg, -val, val)


def scale_of(edges):
    """s = the longest domain edge; edges[p] are the n_p + 1 cell edges of axis p (i1 first)."""
    return float(max(e[-1] - e[0] for e in edges))


def factor_matrices(edges_p, s: float, tau: float):
    """(E, F) n_p x n_p for one axis: rows = collocation points, columns = cells (scaled by 1/s)."""
    y = np.asarray(edges_p, dtype=np.float64) / s
    xi = 0.5 * (y[:-1] + y[1:])
    a = xi[:, None] - y[None, 1:]
    b = xi[:, None] - y[None, :-1]
    return _E(tau, a, b), _F(tau, a, b)


def _check(edges, R):
    if R < 5 or R % 2 == 0:
        raise ValueError("R must be odd and >= 5")
    for e in edges:
        if np.any(np.diff(e) <= 0):
            raise ValueError("cell edges must increase")


def apply_full(m: np.ndarray, edges, R: int, c0: float = 2.15, transpose: bool = False) -> np.ndarray:
    """phi = sum_q P^(q) m^(q) on the grid `edges` (float64 [n3, n2, n1]).

    With transpose=True, m is one field y [n3, n2, n1] and the result is the
    adjoint g[q] = (P^(q))^T y, [3, n3, n2, n1], from the transposed matrices.
    """
    _check(edges, R)
    M = (R - 1) // 2
    s = scale_of(edges)
    _, _, tau, omega = sinc_nodes(M, c0)
    n = tuple(len(e) - 1 for e in edges)
    m = np.asarray(m, dtype=np.float64)
    out = np.zeros((3, n[2], n[1], n[0])) if transpose else np.zeros((n[2], n[1], n[0]))
    for k in range(M):
        mats = {}
        for p in range(3):
            E, F = factor_matrices(edges[p], s, tau[k])
            mats[(p, "E")], mats[(p, "F")] = (E.T, F.T) if transpose else (E, F)
        for q in range(3):
            X = m if transpose else m[q]
            for p in range(3):
                X = mode_product(X, mats[(p, factor_kind(p, q))], p + 1)
            if transpose:
                out[q] += omega[k] * X
            else:
                out += omega[k] * X
    return (C_POT * s) * out


def apply_full_lines(m: np.ndarray, edges, R: int, lines, c0: float = 2.15) -> np.ndarray:
    """phi[i3, i2, :] for a list of (i3, i2) pairs without forming all of phi (float64 [len(lines), n1]).

    The same sum as apply_full with the mode-3 and mode-2 products restricted
    to the requested output rows.
    """
    _check(edges, R)
    M = (R - 1) // 2
    s = scale_of(edges)
    _, _, tau, omega = sinc_nodes(M, c0)
    m = np.asarray(m, dtype=np.float64)
    out = np.zeros((len(lines), len(edges[0]) - 1))
    for k in range(M):
        mats = {}
        for p in range(3):
            mats[(p, "E")], mats[(p, "F")] = factor_matrices(edges[p], s, tau[k])
        for q in range(3):
            U1, U2, U3 = (mats[(p, factor_kind(p, q))] for p in range(3))
            for idx, (i3, i2) in enumerate(lines):
                w = np.tensordot(U3[i3], m[q], axes=([0], [0]))  # [n2, n1]
                out[idx] += omega[k] * (U1 @ (U2[i2] @ w))
    return (C_POT * s) * out
