"""The operator on CP, Tucker and TT tensors (oracle; test infrastructure only).

Eq. kron_eval_cp and Eq. kron_eval_tuck (Sec. 3.4, via the Kronecker /
Khatri-Rao identities listed before them): applying P^(q) to a CP tensor
[[lambda; V1, V2, V3]] gives, for each node k, the CP tensor
[[c omega_k lambda; U^(q1) V1, U^(q2) V2, U^(q3) V3]]; a Tucker tensor keeps
its core and gets factors U^(qp) V_p.  App. C, Eq. tt_3d_2: a 3D tensor train
is the Tucker2 tensor [[G2; G1, id, G3^T]], so the operator maps G1 columns,
the mode-2 fibres of G2 and the rows of G3 through the Toeplitz factors.

The Toeplitz matvecs are done directly with the dense n x n matrices
(O(n^2) per column), deliberately not through FFTs, so that the GPU's
circulant embedding is checked against the plain product.  (Readings of
index typos: the third factor in Eq. kron_eval_cp / kron_eval_tuck is
U^(q3) V^(3), and lambda_j in Lemma DFT_cp is lambda_l.)

Layouts are the C ABI ones (index order slowest -> fastest):
  CP input:      lam [3 comp][r],  U[q][p] = [r][n_p]
  CP output:     w [M][3][r],      outU[p] = [M][3][r][n_p]
  Tucker input:  core [3][r3][r2][r1], V[q][p] = [r_p][n_p]
  Tucker output: w [M][3],         outV[p] = [M][3][r_p][n_p]
  TT input:      G1 [3][r1][n1], G2 [3][r1*r2][n2], G3 [3][r2][n3]
  TT output:     w [M][3],         oG1 [M][3][r1][n1], oG2 [M][3][r1*r2][n2], oG3 [M][3][r2][n3]
"""
from __future__ import annotations

import numpy as np

from .full import terms, factor_kind, C_POT
from .generators import gen_E, gen_F, scaled_spacing
from .quadrature import sinc_nodes


def _split_blocks(flat, n, ranks):
    """Flat (comp, mode, column, entry) buffer -> nested list [q][p] of [r_p][n_p] arrays."""
    flat = np.asarray(flat, dtype=np.float64).ravel()
    out, off = [], 0
    for q in range(3):
        row = []
        for p in range(3):
            size = ranks[p] * n[p]
            row.append(flat[off:off + size].reshape(ranks[p], n[p]))
            off += size
        out.append(row)
    if off != flat.size:
        raise ValueError("factor buffer size does not match n and ranks")
    return out


def apply_cp(lam, U, n, h, R: int, c0: float = 2.15):
    """Returns (w [M][3][r], outU list over p of [M][3][r][n_p]) in float64."""
    n = tuple(int(v) for v in n)
    lam = np.asarray(lam, dtype=np.float64)
    r = lam.shape[1]
    V = _split_blocks(U, n, (r, r, r))
    s, omega, mats = terms(n, h, R, c0)
    M = len(omega)
    w = (C_POT * s) * omega[:, None, None] * lam[None, :, :]
    outU = [np.zeros((M, 3, r, n[p])) for p in range(3)]
    for k in range(M):
        T = mats(k)
        for q in range(3):
            for p in range(3):
                outU[p][k, q] = (T[(p, factor_kind(p, q))] @ V[q][p].T).T
    return w, outU


def apply_cp_entries(lam, U, n, h, R: int, p: int, idx, c0: float = 2.15) -> np.ndarray:
    """Sampled entries outU[p][k, q, l, i] of apply_cp for i in idx (all k, q, l).

    Each needed row of the Toeplitz factor is read off its generator,
    T[i, j] = gen[i - j + n_p - 1] (Sec. 4.2), so long axes (n_p = 8192)
    are checked without forming n_p x n_p matrices.  Returns [M][3][r][len(idx)].
    """
    n = tuple(int(v) for v in n)
    lam = np.asarray(lam, dtype=np.float64)
    r = lam.shape[1]
    V = _split_blocks(U, n, (r, r, r))
    M = (R - 1) // 2
    _, hh = scaled_spacing(n, h)
    _, _, tau, _ = sinc_nodes(M, c0)
    idx = np.asarray(idx, dtype=np.int64)
    j = np.arange(n[p])
    out = np.zeros((M, 3, r, len(idx)))
    for k in range(M):
        gens = {"E": gen_E(tau[k], hh[p], n[p]), "F": gen_F(tau[k], hh[p], n[p])}
        for q in range(3):
            rows = gens[factor_kind(p, q)][(idx[:, None] - j[None, :]) + n[p] - 1]
            out[k, q] = (rows @ V[q][p].T).T
    return out


def cp_to_full(lam, factors) -> np.ndarray:
    """Form sum_l lam_l u1_l o u2_l o u3_l as [n3, n2, n1] (Eq. CP).

    factors = (U1 [r][n1], U2 [r][n2], U3 [r][n3]).
    """
    U1, U2, U3 = (np.asarray(f, dtype=np.float64) for f in factors)
    return np.einsum("l,lk,lj,li->kji", np.asarray(lam, dtype=np.float64), U3, U2, U1)


def cp_output_to_full(w, outU) -> np.ndarray:
    """The field represented by an apply_cp output: sum over (k, q, l) terms."""
    M, Q, r = w.shape
    return cp_to_full(w.reshape(-1), [outU[p].reshape(M * Q * r, -1) for p in range(3)])


def apply_tucker(core, V, n, ranks, h, R: int, c0: float = 2.15):
    """Returns (w [M][3], outV list over p of [M][3][r_p][n_p]) in float64; cores are reused."""
    n = tuple(int(v) for v in n)
    Vb = _split_blocks(V, n, ranks)
    s, omega, mats = terms(n, h, R, c0)
    M = len(omega)
    w = (C_POT * s) * np.repeat(omega[:, None], 3, axis=1)
    outV = [np.zeros((M, 3, ranks[p], n[p])) for p in range(3)]
    for k in range(M):
        T = mats(k)
        for q in range(3):
            for p in range(3):
                outV[p][k, q] = (T[(p, factor_kind(p, q))] @ Vb[q][p].T).T
    return w, outV


def tucker_to_full(core, factors) -> np.ndarray:
    """[[C; V1, V2, V3]] (Eq. tucker_rep) as [n3, n2, n1]; core [r3][r2][r1], factors [r_p][n_p]."""
    V1, V2, V3 = (np.asarray(f, dtype=np.float64) for f in factors)
    return np.einsum("cba,ai,bj,ck->kji", np.asarray(core, dtype=np.float64), V1, V2, V3)


def tucker_output_to_full(core, w, outV) -> np.ndarray:
    """Field represented by an apply_tucker output for cores core[q]."""
    M = w.shape[0]
    total = 0.0
    for k in range(M):
        for q in range(3):
            total = total + w[k, q] * tucker_to_full(core[q], [outV[p][k, q] for p in range(3)])
    return total


def apply_tt(G1, G2, G3, n, ranks, h, R: int, c0: float = 2.15):
    """Returns (w [M][3], oG1 [M][3][r1][n1], oG2 [M][3][r1 r2][n2], oG3 [M][3][r2][n3])."""
    n = tuple(int(v) for v in n)
    G1 = np.asarray(G1, dtype=np.float64)
    G2 = np.asarray(G2, dtype=np.float64)
    G3 = np.asarray(G3, dtype=np.float64)
    r1, r2 = ranks
    s, omega, mats = terms(n, h, R, c0)
    M = len(omega)
    w = (C_POT * s) * np.repeat(omega[:, None], 3, axis=1)
    o1 = np.zeros((M, 3, r1, n[0]))
    o2 = np.zeros((M, 3, r1 * r2, n[1]))
    o3 = np.zeros((M, 3, r2, n[2]))
    for k in range(M):
        T = mats(k)
        for q in range(3):
            o1[k, q] = (T[(0, factor_kind(0, q))] @ G1[q].T).T
            o2[k, q] = (T[(1, factor_kind(1, q))] @ G2[q].T).T
            o3[k, q] = (T[(2, factor_kind(2, q))] @ G3[q].T).T
    return w, o1, o2, o3


def tt_to_full(G1, G2, G3, ranks) -> np.ndarray:
    """Eq. tt_3d_1: a[i1,i2,i3] = sum G1(i1,a1) G2(a1,i2,a2) G3(a2,i3), as [n3, n2, n1].

    G1 [r1][n1], G2 [r1*r2][n2] with row index a1*r2 + a2, G3 [r2][n3].
    """
    r1, r2 = ranks
    G2r = np.asarray(G2, dtype=np.float64).reshape(r1, r2, -1)
    return np.einsum("ai,abj,bk->kji", np.asarray(G1, dtype=np.float64), G2r, np.asarray(G3, dtype=np.float64))


def tt_output_to_full(w, o1, o2, o3, ranks) -> np.ndarray:
    M = w.shape[0]
    total = 0.0
    for k in range(M):
        for q in range(3):
            total = total + w[k, q] * tt_to_full(o1[k, q], o2[k, q], o3[k, q], ranks)
    return total


def cp_inner(w1, f1, w2, f2) -> float:
    """<X, Y> of two CP tensors from weights and factor lists without forming them.

    <X, Y> = sum_{l, l'} w1_l w2_l' prod_p <u_l^(p), v_l'^(p)> (Gram matrices).
    """
    G = np.outer(np.asarray(w1, dtype=np.float64), np.asarray(w2, dtype=np.float64))
    for p in range(3):
        G = G * (np.asarray(f1[p], dtype=np.float64) @ np.asarray(f2[p], dtype=np.float64).T)
    return float(G.sum())
