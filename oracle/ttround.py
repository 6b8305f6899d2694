"""TT rounding of the potential in tensor-train form (oracle; test infrastructure only).

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
