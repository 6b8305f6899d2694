"""Exact collocation of the potential (oracle; test infrastructure only).

Eq. coll / Eq. matrix_op: with piecewise-constant m and midpoint collocation,

    phi_i = (1/4pi) sum_q sum_j m_j^(q) G^(q)_ij,
    G^(q)_ij = int_{Omega_j} (xi_i - y)_q / |xi_i - y|^3 dy,

(sign + as argued in the package docstring).  No quadrature in tau is
involved: since (x - y)_q / |x - y|^3 = d/dy_q (1 / |x - y|), the volume
integral over the box Omega_j is the difference of two face integrals of
1/|x - y| (the two faces normal to axis q), and each face integral has the
classical closed form of a uniformly charged rectangle, an inclusion-exclusion
over the four corners of

    W(u, v, w) = u asinh(v / sqrt(u^2 + w^2)) + v asinh(u / sqrt(v^2 + w^2))
                 - |w| atan(u v / (|w| sqrt(u^2 + v^2 + w^2))),

which satisfies d^2 W / du dv = 1 / sqrt(u^2 + v^2 + w^2).

On a uniform grid G^(q)_ij depends on d = i - j only (Sec. 4.2, Eq. conv_op),
so the entries are tabulated per offset and phi is the discrete convolution
of that table with m (a direct sum, or scipy's FFT convolution for the larger
refinement studies; both are the same sum).
"""
from __future__ import annotations

import numpy as np


def rect_W(u, v, w):
    """Antiderivative W(u, v, w) of 1/sqrt(u^2+v^2+w^2) in u and v (w fixed)."""
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    w = np.abs(np.asarray(w, dtype=np.float64))
    r = np.sqrt(u * u + v * v + w * w)
    ruw = np.sqrt(u * u + w * w)
    rvw = np.sqrt(v * v + w * w)
    with np.errstate(divide="ignore", invalid="ignore"):
        t1 = np.where(ruw > 0, u * np.arcsinh(v / np.where(ruw > 0, ruw, 1.0)), 0.0)
        t2 = np.where(rvw > 0, v * np.arcsinh(u / np.where(rvw > 0, rvw, 1.0)), 0.0)
        t3 = np.where(w > 0, w * np.arctan(u * v / np.where(w > 0, w * r, 1.0)), 0.0)
    return t1 + t2 - t3


def rect_integral(u0, u1, v0, v1, w):
    """int_{u0}^{u1} int_{v0}^{v1} 1/sqrt(u^2 + v^2 + w^2) dv du."""
    return rect_W(u1, v1, w) - rect_W(u0, v1, w) - rect_W(u1, v0, w) + rect_W(u0, v0, w)


def box_G(q: int, lo, hi):
    """int over the box x in [lo, hi] (3-vectors, x = xi - y) of x_q / |x|^3.

    x_q/|x|^3 = -d/dx_q (1/|x|), so the integral is the face integral of 1/|x|
    at x_q = lo_q minus the one at x_q = hi_q.
    """
    lo = [np.asarray(c, dtype=np.float64) for c in lo]
    hi = [np.asarray(c, dtype=np.float64) for c in hi]
    u, v = [p for p in range(3) if p != q]
    near = rect_integral(lo[u], hi[u], lo[v], hi[v], lo[q])
    far = rect_integral(lo[u], hi[u], lo[v], hi[v], hi[q])
    return near - far


def G_table(q: int, n, hh):
    """G^(q)(d) for all offsets d = i - j, array [2n3-1, 2n2-1, 2n1-1] (d + n - 1 indexing).

    The box of x = xi_i - y for offset d is prod_p [(d_p - 1/2) hh_p, (d_p + 1/2) hh_p].
    """
    axes = []
    for p in range(3):
        d = np.arange(-(n[p] - 1), n[p], dtype=np.float64)
        axes.append(d)
    D3, D2, D1 = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    D = (D1, D2, D3)
    lo = [(D[p] - 0.5) * hh[p] for p in range(3)]
    hi = [(D[p] + 0.5) * hh[p] for p in range(3)]
    return box_G(q, lo, hi)


def collocation_exact(m: np.ndarray, n, h, method: str = "direct") -> np.ndarray:
    """phi_i = (1/4pi) sum_q sum_j G^(q)_{i-j} m_j^(q) (exact entries), float64 [n3, n2, n1].

    O(N^2) as in Eq. approx_phi.  method='fft' evaluates the same discrete
    convolution with scipy.signal.fftconvolve (for the refinement studies).
    """
    n = tuple(int(v) for v in n)
    m = np.asarray(m, dtype=np.float64)
    hh = [float(v) for v in h]  # physical cell sizes: no domain scaling here
    n1, n2, n3 = n
    phi = np.zeros((n3, n2, n1))
    for q in range(3):
        G = G_table(q, n, hh)
        if method == "fft":
            from scipy.signal import fftconvolve
            full = fftconvolve(m[q], G, mode="full")
            phi += full[n3 - 1:2 * n3 - 1, n2 - 1:2 * n2 - 1, n1 - 1:2 * n1 - 1]
        else:
            # phi[i] += G[i - j] m[j]: loop over offsets d, shift m by d.
            for d3 in range(-(n3 - 1), n3):
                i3 = slice(max(d3, 0), n3 + min(d3, 0))
                j3 = slice(max(-d3, 0), n3 - max(d3, 0))
                for d2 in range(-(n2 - 1), n2):
                    i2 = slice(max(d2, 0), n2 + min(d2, 0))
                    j2 = slice(max(-d2, 0), n2 - max(d2, 0))
                    row = G[d3 + n3 - 1, d2 + n2 - 1]
                    for d1 in range(-(n1 - 1), n1):
                        i1 = slice(max(d1, 0), n1 + min(d1, 0))
                        j1 = slice(max(-d1, 0), n1 - max(d1, 0))
                        phi[i3, i2, i1] += row[d1 + n1 - 1] * m[q][j3, j2, j1]
    return phi / (4.0 * np.pi)


def uniform_box_potential(n, h, axis: int = 2) -> np.ndarray:
    """Exact potential at the cell centres of a box magnetized uniformly along `axis`.

    phi(xi) = (1/4pi) int_Omega d/dy_q (1/|xi - y|) dy
            = (1/4pi) [int_{far face} 1/|xi - y| - int_{near face} 1/|xi - y|]
    (Eq. intop1 with div m = 0 and surface charge n.m = +-1 on the two faces
    normal to `axis`).  This is what the collocation sum gives exactly for
    uniform m, since sum_j G^(q)_ij is the same integral over all of Omega.
    """
    n = tuple(int(v) for v in n)
    L = [n[p] * float(h[p]) for p in range(3)]
    c = [(np.arange(n[p]) + 0.5) * float(h[p]) for p in range(3)]
    X3, X2, X1 = np.meshgrid(c[2], c[1], c[0], indexing="ij")
    X = (X1, X2, X3)
    q = axis
    u, v = [p for p in range(3) if p != q]
    # face integrals in coordinates relative to the collocation point
    u0, u1 = X[u] - L[u], X[u]
    v0, v1 = X[v] - L[v], X[v]
    top = rect_integral(u0, u1, v0, v1, X[q] - L[q])
    bottom = rect_integral(u0, u1, v0, v1, X[q])
    return (top - bottom) / (4.0 * np.pi)
