"""TT rounding of the potential in tensor-train form, and the TT conversions and Hadamard
product of App. C (oracle; test infrastructure only).

App. C: a 3D tensor train a[i1,i2,i3] = sum G1(i1,a1) G2(a1,i2,a2) G3(a2,i3)
(Eq. tt_3d_1) admits recompression ("rounding", cited there): the operator
applied to a TT magnetization gives, per node k and component q, a TT with
the input ranks (Eq. tt_3d_2 with the Toeplitz factors), so the potential is a
sum of 3M trains with ranks 3M r.  Rounding to tolerance tol is the TT-SVD:
two truncated SVDs of the sequential unfoldings, each at delta = tol / sqrt(2)
of the norm (d - 1 = 2 truncations), so ||phi - phi_hat|| <= tol ||phi||.

This oracle forms the dense tensor: small grids only.  Layouts as the C ABI:
G1 [r1][n1], G2 [r1 r2][n2] with row a1 r2 + a2, G3 [r2][n3]; dense [n3, n2, n1].
"""
from __future__ import annotations

import numpy as np


def _rank(sig: np.ndarray, bound2: float) -> int:
    tail = np.concatenate([np.cumsum((sig ** 2)[::-1])[::-1], [0.0]])  # tail[r] = sum_{i >= r}
    for r in range(1, len(sig) + 1):
        if tail[r] <= bound2:
            return r
    return len(sig)


def tt_round_dense(X: np.ndarray, tol: float):
    """(G1 [r1][n1], G2 [r1 r2][n2], G3 [r2][n3], (r1, r2)) with ||X - TT|| <= tol ||X||."""
    n3, n2, n1 = X.shape
    Xt = np.asarray(X, dtype=np.float64).transpose(2, 1, 0)  # [n1, n2, n3]
    bound2 = (tol / np.sqrt(2.0)) ** 2 * float(np.sum(Xt ** 2))
    U, s, Vt = np.linalg.svd(Xt.reshape(n1, n2 * n3), full_matrices=False)
    r1 = _rank(s, bound2)
    G1 = U[:, :r1]
    C = (s[:r1, None] * Vt[:r1]).reshape(r1 * n2, n3)
    U2, s2, Vt2 = np.linalg.svd(C, full_matrices=False)
    r2 = _rank(s2, bound2)
    G2 = U2[:, :r2].reshape(r1, n2, r2)
    G3 = s2[:r2, None] * Vt2[:r2]
    return G1.T.copy(), G2.transpose(0, 2, 1).reshape(r1 * r2, n2).copy(), G3.copy(), (r1, r2)


# ---- conversions and the Hadamard product (App. C), per component, ABI layouts ----

def tucker_to_tt(core, V1, V2, V3):
    """One Tucker tensor [[C; V1, V2, V3]] (core [r3][r2][r1], V_p [r_p][n_p]) as a train of ranks
    (r1, r3): G1 = V1, G3 = V3, G2[(a1 r3 + a3)][i2] = sum_a2 C[a3][a2][a1] V2[a2][i2]."""
    C = np.asarray(core, dtype=np.float64)
    r3, r2, r1 = C.shape
    G2 = np.einsum("cba,bj->acj", C, np.asarray(V2, dtype=np.float64)).reshape(r1 * r3, -1)
    return np.asarray(V1, dtype=np.float64).copy(), G2, np.asarray(V3, dtype=np.float64).copy()


def cp_to_tt(lam, U1, U2, U3):
    """sum_l lam_l U1[l] o U2[l] o U3[l] as a train of ranks (r, r) with a diagonal middle core."""
    lam = np.asarray(lam, dtype=np.float64)
    r = lam.size
    U2 = np.asarray(U2, dtype=np.float64)
    G2 = np.zeros((r, r, U2.shape[1]))
    for a in range(r):
        G2[a, a] = lam[a] * U2[a]
    return np.asarray(U1, dtype=np.float64).copy(), G2.reshape(r * r, -1), np.asarray(U3, dtype=np.float64).copy()


def tt_hadamard(A, ra, B, rb):
    """The element-wise product of two trains (cores multiplied as Kronecker products of their rank
    indices); returns (C1, C2, C3) with ranks (ra1 rb1, ra2 rb2)."""
    A1, A2, A3 = (np.asarray(x, dtype=np.float64) for x in A)
    B1, B2, B3 = (np.asarray(x, dtype=np.float64) for x in B)
    C1 = np.einsum("ai,bi->abi", A1, B1).reshape(ra[0] * rb[0], -1)
    A2r = A2.reshape(ra[0], ra[1], -1)
    B2r = B2.reshape(rb[0], rb[1], -1)
    C2 = np.einsum("acj,bdj->abcdj", A2r, B2r).reshape(ra[0] * rb[0] * ra[1] * rb[1], -1)
    C3 = np.einsum("ak,bk->abk", A3, B3).reshape(ra[1] * rb[1], -1)
    return C1, C2, C3
