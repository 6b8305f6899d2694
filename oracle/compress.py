"""Alg. 2 with a compressed kernel: Tucker compression of the CP convolution
kernels (Alg. 1, HOOI) and their application to Tucker magnetizations
(oracle; test infrastructure only).

Eq. conv_pot writes the kernel of component q as the CP tensor
K^(q) = [[lam; A_1, A_2, A_3]] with lam_k = c s omega_k and columns
A_p[:, k] = generator F_k (p == q) or E_k (p != q), entries d = -(n_p-1)..n_p-1.
Alg. 2 compresses each K^(q) to a Tucker tensor [[C^(q); U_1, U_2, U_3]] with
tolerance tol (setup), and applies it to a Tucker magnetization
[[G^(q); V_1^(q), V_2^(q), V_3^(q)]] through the FFT (Lemma DFT_tucker) and the
Tucker Hadamard product (App. B, Eq. t_had2): in Fourier space the factor
columns multiply row-wise and the cores form a Kronecker product, so after the
inverse DFT the result is the Tucker tensor

    [[C^(q) (x) G^(q); W_1, W_2, W_3]],  W_p[:, (i, l)] = T(U_p[:, i]) V_p[:, l],

T(u) the Toeplitz matrix of generator u (the circular convolution cropped to
the grid; the columns are ordered i major, l minor, and the core index is
(i, l) alike).  phi is the sum of the three component results.

Compression (Alg. 1): ranks from the truncated HOSVD with the rule
r_p = min{ r : sqrt(sum_{i > r} sigma_i^2) <= tol / sqrt(3) * ||sigma|| } per
mode (the reading of the rank step of Alg. 1, whose printed inequality is
garbled), taken as the largest over the three components so that all
components share one rank per mode; then HOOI sweeps at those ranks from the
HOSVD start.  The HOSVD bound (Eq. quasi_best_tucker) gives
||K - K_tucker|| <= tol ||K|| and HOOI only increases the captured norm.

This oracle forms each kernel densely ((2n-1)^3 entries) and uses numpy SVDs
of the unfoldings: small grids only.
"""
from __future__ import annotations

import numpy as np

from .full import C_POT, factor_kind
from .generators import gen_E, gen_F, scaled_spacing, toeplitz
from .quadrature import sinc_nodes


def cp_kernel(q: int, n, h, R: int, c0: float = 2.15):
    """(A, lam): A[p] is [2 n_p - 1, M] (generator columns), lam [M] = c s omega_k."""
    n = tuple(int(v) for v in n)
    M = (R - 1) // 2
    s, hh = scaled_spacing(n, h)
    _, _, tau, omega = sinc_nodes(M, c0)
    A = []
    for p in range(3):
        gen = gen_F if factor_kind(p, q) == "F" else gen_E
        A.append(np.stack([gen(tau[k], hh[p], n[p]) for k in range(M)], axis=1))
    return A, C_POT * s * omega


def cp_to_dense(A, lam) -> np.ndarray:
    """sum_k lam_k A_3[:, k] (x) A_2[:, k] (x) A_1[:, k] as numpy [m3, m2, m1]."""
    return np.einsum("k,ck,bk,ak->cba", lam, A[2], A[1], A[0])


def unfold(X: np.ndarray, p: int) -> np.ndarray:
    """Mode-p unfolding (p = 0 is the fastest numpy axis): [m_p, prod of the others]."""
    return np.moveaxis(X, 2 - p, 0).reshape(X.shape[2 - p], -1)


def mode_mult(X: np.ndarray, U: np.ndarray, p: int) -> np.ndarray:
    """X x_p U (Eq. modemul) with U [r, m_p]; p = 0 is the fastest numpy axis."""
    ax = 2 - p
    return np.moveaxis(np.tensordot(U, X, axes=([1], [ax])), 0, ax)


def tucker_to_dense(C: np.ndarray, U) -> np.ndarray:
    X = C
    for p in range(3):
        X = mode_mult(X, U[p], p)
    return X


def truncation_rank(sigma: np.ndarray, tol: float) -> int:
    total = float(np.sum(sigma ** 2))
    tail = np.concatenate([np.cumsum((sigma ** 2)[::-1])[::-1], [0.0]])  # tail[r] = sum_{i >= r}
    bound = (tol / np.sqrt(3.0)) ** 2 * total
    for r in range(1, len(sigma) + 1):
        if tail[r] <= bound:
            return r
    return len(sigma)


def hosvd_spectra(X: np.ndarray):
    """Left singular vectors and singular values of the three unfoldings."""
    out = []
    for p in range(3):
        U, sig, _ = np.linalg.svd(unfold(X, p), full_matrices=False)
        out.append((U, sig))
    return out


def hooi(X: np.ndarray, ranks, sweeps: int = 4):
    """Alg. 1 at fixed ranks from the HOSVD start: (C, [U_1, U_2, U_3]) with U_p [m_p, r_p]."""
    U = [hosvd_spectra(X)[p][0][:, : ranks[p]] for p in range(3)]
    for _ in range(sweeps):
        for p in range(3):
            Y = X
            for j in range(3):
                if j != p:
                    Y = mode_mult(Y, U[j].T, j)
            Up, _, _ = np.linalg.svd(unfold(Y, p), full_matrices=False)
            U[p] = Up[:, : ranks[p]]
    C = X
    for p in range(3):
        C = mode_mult(C, U[p].T, p)
    return C, U


def compress_kernels(n, h, R: int, tol: float, c0: float = 2.15, sweeps: int = 4):
    """Compressed kernels of the three components: (ranks, [(C^(q), U^(q)) for q])."""
    dense = [cp_to_dense(*cp_kernel(q, n, h, R, c0)) for q in range(3)]
    ranks = [1, 1, 1]
    for X in dense:
        spec = hosvd_spectra(X)
        for p in range(3):
            ranks[p] = max(ranks[p], truncation_rank(spec[p][1], tol))
    return ranks, [hooi(X, ranks, sweeps) for X in dense]


def apply_tucker_compressed(G, V, n, compressed):
    """phi for the Tucker magnetization (G[q] [r3, r2, r1], V[q][p] [n_p, r_p]) with compressed kernels.

    Returns (parts, phi): parts[q] = (core [r3 rho3, r2 rho2, r1 rho1] numpy order, W [p] [n_p, rho_p r_p]),
    phi the dense sum (float64 [n3, n2, n1]).
    """
    n = tuple(int(v) for v in n)
    parts = []
    phi = np.zeros((n[2], n[1], n[0]))
    for q, (C, U) in enumerate(compressed):
        W = []
        for p in range(3):
            T = [toeplitz(U[p][:, i], n[p]) for i in range(U[p].shape[1])]
            # columns (i, l): i major
            W.append(np.concatenate([Ti @ V[q][p] for Ti in T], axis=1))
        # core index (i, l) per mode, i major: E[(i3 l3), (i2 l2), (i1 l1)] = C[i3 i2 i1] G[l3 l2 l1]
        E = np.einsum("abc,def->adbecf", C, G[q]).reshape(C.shape[0] * G[q].shape[0], C.shape[1] * G[q].shape[1],
                                                           C.shape[2] * G[q].shape[2])
        parts.append((E, W))
        phi += tucker_to_dense(E, W)
    return parts, phi


def tucker_hadamard(C, U, D, V):
    """App. B, Eq. t_had2: the elementwise product of [[C; U]] and [[D; V]] as a Tucker tensor.

    Factors: row-wise Kronecker products (columns (i, l), i major); core: the
    Kronecker product of the cores with the same (i, l) index.
    """
    W = [np.einsum("ni,nl->nil", U[p], V[p]).reshape(U[p].shape[0], -1) for p in range(3)]
    E = np.einsum("abc,def->adbecf", C, D).reshape(C.shape[0] * D.shape[0], C.shape[1] * D.shape[1],
                                                   C.shape[2] * D.shape[2])
    return E, W


def recompress(parts, tol: float):
    """Alg. 2's last step, approximate summation: phi = sum_q [[E_q; W_q]] recompressed to one
    Tucker tensor with ||phi - phi_hat|| <= tol ||phi|| by a truncated HOSVD of the dense sum
    (the rank rule of Alg. 1 per mode at tol / sqrt(3)); small grids only.

    Returns (C [r3, r2, r1], [U_1, U_2, U_3] with U_p [n_p, r_p] orthonormal, ranks).
    """
    phi = sum(tucker_to_dense(E, W) for E, W in parts)
    spec = hosvd_spectra(phi)
    ranks = [truncation_rank(spec[p][1], tol) for p in range(3)]
    U = [spec[p][0][:, : ranks[p]] for p in range(3)]
    C = phi
    for p in range(3):
        C = mode_mult(C, U[p].T, p)
    return C, U, ranks
