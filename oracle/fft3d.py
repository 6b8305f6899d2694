"""The potential by one 3D FFT convolution with a dense Fourier kernel
(oracle; test infrastructure only).

Sec. 4.2, Eq. conv_op, Eq. conv_pot and Eq. fft_pot: the operator P^(q) is a
convolution with the separable kernel G^(q)[J] (J = i - j, |J_p| < n_p), so

    P^(q) * X = IDFT( DFT(G^(q)) . DFT(X) )

on a grid padded so that the cyclic convolution equals the aperiodic one.
Here the padded length per axis is L_p = the next power of two >= 2 n_p - 1
(any L_p >= 2 n_p - 1 is exact; Eq. fft_pot writes 2 n_p - 1).  The node
sum of Eq. conv_pot is linear, so it is summed once into a dense Fourier
kernel

    K^(q)[w] = c s sum_k omega_k  prod_p DFT_{L_p}(g_{k,q,p})[w_p],

g_{k,q,p} the circulant embedding of the generator F (p == q) or E (p != q)
(entries d = -(n_p - 1)..n_p - 1 at index d mod L_p, zero elsewhere), and
phi = IDFT( sum_q K^(q) . DFT(m^(q)) ) cropped to the grid.  The cost is then
independent of R.  Sign and constant: c = 1/(2 pi^{3/2}) with the sign +, the
reading used for Eq. kron_operator (see oracle.full).

Arrays: a field is numpy [n3, n2, n1] (i1 fastest); a kernel [L3, L2, L1].
"""
from __future__ import annotations

import numpy as np

from .full import C_POT, factor_kind
from .generators import gen_E, gen_F, scaled_spacing
from .quadrature import sinc_nodes


def padded_lengths(n):
    """L_p = next power of two >= 2 n_p - 1 (and >= 2)."""
    out = []
    for v in n:
        L = 1
        while L < 2 * int(v) - 1:
            L *= 2
        out.append(max(L, 2))
    return tuple(out)


def circulant_column(gen: np.ndarray, n: int, L: int) -> np.ndarray:
    """Generator entries d = -(n-1)..n-1 summed into index d mod L (zeros elsewhere).

    For L >= 2n - 1 no two entries meet; a shorter L gives the periodised
    (aliased) kernel.
    """
    c = np.zeros(L)
    d = np.arange(-(n - 1), n)
    np.add.at(c, d % L, gen)
    return c


def dense_kernel(n, h, R: int, c0: float = 2.15, L=None):
    """K^(q) for q = 1..3: complex [3, L3, L2, L1], the node sum of Eq. conv_pot in Fourier space.

    L (per axis, i1 first) defaults to padded_lengths(n).
    """
    n = tuple(int(v) for v in n)
    if R < 5 or R % 2 == 0:
        raise ValueError("R must be odd and >= 5")
    M = (R - 1) // 2
    s, hh = scaled_spacing(n, h)
    _, _, tau, omega = sinc_nodes(M, c0)
    L = padded_lengths(n) if L is None else tuple(int(v) for v in L)
    K = np.zeros((3, L[2], L[1], L[0]), dtype=np.complex128)
    for k in range(M):
        spec = {}
        for p in range(3):
            for kind, gen in (("E", gen_E), ("F", gen_F)):
                spec[(p, kind)] = np.fft.fft(circulant_column(gen(tau[k], hh[p], n[p]), n[p], L[p]))
        for q in range(3):
            a1 = spec[(0, factor_kind(0, q))]
            a2 = spec[(1, factor_kind(1, q))]
            a3 = spec[(2, factor_kind(2, q))]
            K[q] += omega[k] * (a3[:, None, None] * a2[None, :, None] * a1[None, None, :])
    return (C_POT * s) * K


def apply_fft3d(m: np.ndarray, n, h, R: int, c0: float = 2.15, K=None) -> np.ndarray:
    """phi = sum_q P^(q) m^(q) by Eq. fft_pot with the summed kernel (float64 [n3, n2, n1])."""
    n = tuple(int(v) for v in n)
    m = np.asarray(m, dtype=np.float64)
    if K is None:
        K = dense_kernel(n, h, R, c0)
    L = K.shape[1:]
    acc = np.zeros(L, dtype=np.complex128)
    for q in range(3):
        acc += K[q] * np.fft.fftn(m[q], s=L, axes=(0, 1, 2))
    phi = np.fft.ifftn(acc)
    return phi.real[: n[2], : n[1], : n[0]].copy()


def dense_field_kernels(n, h, R: int, c0: float = 2.15, L=None):
    """K_pq (p, q = 1..3) of h_d[p] = sum_q IDFT(K_pq . DFT(m^(q))): complex [3, 3, L3, L2, L1].

    h_d = -grad phi with the analytic derivative factors of oracle.field: the
    axis-p factor of every term of Eq. conv_pot is replaced by its derivative
    (dE for E, dF for F), and the node sum is folded in Fourier space as for
    the potential.  The derivative generators carry 1/s, so the scale is c.
    """
    from .field import gen_dE, gen_dF
    n = tuple(int(v) for v in n)
    if R < 5 or R % 2 == 0:
        raise ValueError("R must be odd and >= 5")
    M = (R - 1) // 2
    s, hh = scaled_spacing(n, h)
    _, _, tau, omega = sinc_nodes(M, c0)
    L = padded_lengths(n) if L is None else tuple(int(v) for v in L)
    K = np.zeros((3, 3, L[2], L[1], L[0]), dtype=np.complex128)
    for k in range(M):
        spec = {}
        for p in range(3):
            gens = (("E", gen_E), ("F", gen_F), ("dE", gen_dE), ("dF", gen_dF))
            for kind, gen in gens:
                g = gen(tau[k], hh[p], n[p])
                if kind.startswith("d"):
                    g = g / s
                spec[(p, kind)] = np.fft.fft(circulant_column(g, n[p], L[p]))
        for d in range(3):
            for q in range(3):
                a = []
                for p in range(3):
                    kind = factor_kind(p, q)
                    a.append(spec[(p, "d" + kind if p == d else kind)])
                K[d, q] -= omega[k] * (a[2][:, None, None] * a[1][None, :, None] * a[0][None, None, :])
    return (C_POT * s) * K


def apply_field_fft3d(m: np.ndarray, n, h, R: int, c0: float = 2.15, K=None) -> np.ndarray:
    """h_d [3, n3, n2, n1] by one 3D FFT convolution with the summed derivative kernels."""
    n = tuple(int(v) for v in n)
    m = np.asarray(m, dtype=np.float64)
    if K is None:
        K = dense_field_kernels(n, h, R, c0)
    L = K.shape[2:]
    X = [np.fft.fftn(m[q], s=L, axes=(0, 1, 2)) for q in range(3)]
    out = np.zeros((3, n[2], n[1], n[0]))
    for d in range(3):
        acc = sum(K[d, q] * X[q] for q in range(3))
        out[d] = np.fft.ifftn(acc).real[: n[2], : n[1], : n[0]]
    return out
