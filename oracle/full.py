"""Kronecker-product potential operator on full tensors (oracle; test infrastructure only).

Cor. 3, Eq. kron_operator: for each magnetization component q,

    P^(q) = c * sum_k omega_k  U_k^(q3) (x) U_k^(q2) (x) U_k^(q1),

with (U_k^(qp))_{i j} = h^(p)_{i-j}(tau_k) the Toeplitz matrix of the
generator F (p == q) or E (p != q) from ``generators``.  The footnote of
Cor. 3 fixes the index order (i1 fastest, A^(3) (x) A^(2) (x) A^(1)), so the
action on a tensor X[i3, i2, i1] is the three mode products of Eq. modemul:

    (P^(q) X) = c * sum_k omega_k  X x_1 U^(q1) x_2 U^(q2) x_3 U^(q3).

phi = sum_q P^(q) m^(q) is Eq. pot_op.  Reading of the constant: the
collocation scheme is phi_i = (1/4pi) sum_q sum_j m_j G^(q)_ij (sign + as
argued in the package docstring), Eq. matrix_op_sep gives
G = (2/sqrt(pi)) int tau^2 prod_p h^(p) dtau, hence c = 1/(2 pi^{3/2}) times
the length scale s of ``generators.scaled_spacing``.

Arrays: a field is numpy [n3, n2, n1] (i1 fastest), a magnetization
[3, n3, n2, n1].  Mode p acts on numpy axis 3 - p.
"""
from __future__ import annotations

import numpy as np

from .quadrature import sinc_nodes
from .generators import scaled_spacing, gen_E, gen_F, toeplitz

C_POT = 1.0 / (2.0 * np.pi ** 1.5)


def mode_product(X: np.ndarray, U: np.ndarray, mode: int) -> np.ndarray:
    """Eq. modemul: (X x_mode U)[.., a, ..] = sum_b X[.., b, ..] U[a, b]; mode in 1..3."""
    ax = 3 - mode
    Y = np.tensordot(U, X, axes=([1], [ax]))  # new axis first
    return np.moveaxis(Y, 0, ax)


def terms(n, h, R: int, c0: float = 2.15):
    """Scale s, node weights omega_k and the Toeplitz matrices per node.

    Returns (s, omega, mats) where mats(k) -> dict {(p, 'E'|'F'): n_p x n_p}.
    R is the total number of symmetric nodes, R = 2M+1 (odd, >= 5).
    """
    if R < 5 or R % 2 == 0:
        raise ValueError("R must be odd and >= 5")
    M = (R - 1) // 2
    s, hh = scaled_spacing(n, h)
    _, _, tau, omega = sinc_nodes(M, c0)

    def mats(k):
        out = {}
        for p in range(3):
            # axes with the same n and spacing have the same matrices
            same = [r for r in range(p) if n[r] == n[p] and hh[r] == hh[p]]
            if same:
                out[(p, "E")], out[(p, "F")] = out[(same[0], "E")], out[(same[0], "F")]
                continue
            out[(p, "E")] = toeplitz(gen_E(tau[k], hh[p], n[p]), n[p])
            out[(p, "F")] = toeplitz(gen_F(tau[k], hh[p], n[p]), n[p])
        return out

    return s, omega, mats


def factor_kind(p: int, q: int) -> str:
    """Which generator acts on axis p for component q (Eq. sep_integrands)."""
    return "F" if p == q else "E"


def apply_full(m: np.ndarray, n, h, R: int, c0: float = 2.15, nodes=None) -> np.ndarray:
    """phi = sum_q P^(q) m^(q) for a full magnetization m[3, n3, n2, n1] (float64 result).

    `nodes` optionally restricts the node sum to a subset of k (0-based), which
    the CPU timing uses to bound its work; the default is all M nodes.
    """
    n = tuple(int(v) for v in n)
    m = np.asarray(m, dtype=np.float64)
    s, omega, mats = terms(n, h, R, c0)
    phi = np.zeros((n[2], n[1], n[0]))
    ks = range(len(omega)) if nodes is None else nodes
    for k in ks:
        T = mats(k)
        for q in range(3):
            X = m[q]
            for p in range(3):
                X = mode_product(X, T[(p, factor_kind(p, q))], p + 1)
            phi += omega[k] * X
    return (C_POT * s) * phi


def apply_full_lines(m: np.ndarray, n, h, R: int, lines, c0: float = 2.15) -> np.ndarray:
    """phi[i3, i2, :] for a list of (i3, i2) pairs, without forming all of phi.

    Same sum as apply_full (Eq. kron_operator), with the mode-3 and mode-2
    products restricted to the requested output rows:
    phi[i3, i2, :] = c s sum_k omega_k sum_q U^(q1) (sum_{j3, j2} U^(q3)[i3, j3] U^(q2)[i2, j2] m^(q)[j3, j2, :]).
    Returns float64 [len(lines), n1].
    """
    n = tuple(int(v) for v in n)
    m = np.asarray(m, dtype=np.float64)
    s, omega, mats = terms(n, h, R, c0)
    out = np.zeros((len(lines), n[0]))
    for k in range(len(omega)):
        T = mats(k)
        for q in range(3):
            U1 = T[(0, factor_kind(0, q))]
            U2 = T[(1, factor_kind(1, q))]
            U3 = T[(2, factor_kind(2, q))]
            for idx, (i3, i2) in enumerate(lines):
                w = np.tensordot(U3[i3], m[q], axes=([0], [0]))  # [n2, n1]
                w = U2[i2] @ w                                    # [n1]
                out[idx] += omega[k] * (U1 @ w)
    return (C_POT * s) * out


def apply_adjoint(y: np.ndarray, n, h, R: int, c0: float = 2.15) -> np.ndarray:
    """g^(q) = (P^(q))^T y for q = 1..3, by mode products with transposed factors.

    The transpose of a Kronecker product is the Kronecker product of the
    transposes, so (P^(q))^T = c sum_k omega_k U^(q3)T (x) U^(q2)T (x) U^(q1)T.
    """
    n = tuple(int(v) for v in n)
    y = np.asarray(y, dtype=np.float64)
    s, omega, mats = terms(n, h, R, c0)
    g = np.zeros((3, n[2], n[1], n[0]))
    for k in range(len(omega)):
        T = mats(k)
        for q in range(3):
            X = y
            for p in range(3):
                X = mode_product(X, T[(p, factor_kind(p, q))].T, p + 1)
            g[q] += omega[k] * X
    return (C_POT * s) * g


def dense_operator(n, h, R: int, c0: float = 2.15) -> np.ndarray:
    """The N x N quadrature matrices c*G~^(q), built entry by entry (tiny grids only).

    Entry (I, J) with I = i1 + n1 (i2 + n2 i3) (0-based form of the footnote of
    Cor. 3) is c * sum_k omega_k prod_p h^(p)_{i_p - j_p}(tau_k), from
    Eq. matrix_op_sep after the sinc rule.  Returns an array [3, N, N];
    phi = sum_q out[q] @ m[q].ravel().
    """
    n = tuple(int(v) for v in n)
    N = n[0] * n[1] * n[2]
    if N > 4096:
        raise ValueError("dense operator is for tiny grids only")
    M = (R - 1) // 2
    s, hh = scaled_spacing(n, h)
    _, _, tau, omega = sinc_nodes(M, c0)
    I = np.arange(N)
    idx = np.stack([I % n[0], (I // n[0]) % n[1], I // (n[0] * n[1])])  # i1, i2, i3
    out = np.zeros((3, N, N))
    for k in range(M):
        gens = {}
        for p in range(3):
            gens[(p, "E")] = gen_E(tau[k], hh[p], n[p])
            gens[(p, "F")] = gen_F(tau[k], hh[p], n[p])
        for q in range(3):
            prod = np.ones((N, N))
            for p in range(3):
                d = idx[p][:, None] - idx[p][None, :]
                prod *= gens[(p, factor_kind(p, q))][d + n[p] - 1]
            out[q] += omega[k] * prod
    return (C_POT * s) * out
