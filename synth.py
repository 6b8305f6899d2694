"""Seeded synthetic inputs shared by the oracle checks, the GPU tests and the bench.

This module holds no arithmetic of the demagnetizing operator: it only draws
magnetizations and tensor-format factors with the shapes and value
distributions of the paper's numerical experiments (Sec. 3.2 collocation on a
tensor grid, Sec. 4.2 structured inputs, Alg. 2 Tucker magnetizations).

Random numbers come from splitmix64 (Steele, Lea, Flood 2014) turned into
uniforms on [0, 1) by the top 53 bits, and into normals by Box-Muller.  Every
generator takes an integer seed; values are produced in float64 and returned
rounded to float32, so that the oracle (which widens them exactly to float64)
and the GPU path consume identical numbers.

Layouts match the C ABI: a full field is ``[3][n3][n2][n1]`` with i1 fastest.
"""
from __future__ import annotations

import numpy as np

_MASK = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


def splitmix64(seed: int, count: int) -> np.ndarray:
    """`count` consecutive splitmix64 outputs for state `seed` (uint64 array)."""
    idx = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK) + idx * np.uint64(_GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int) -> np.ndarray:
    """Uniform float64 samples on [0, 1)."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def normal(seed: int, count: int) -> np.ndarray:
    """Standard normal float64 samples (Box-Muller on pairs of uniforms)."""
    m = (count + 1) // 2
    u = uniform(seed, 2 * m)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = rad * np.cos(2.0 * np.pi * u2)
    z[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return z[:count]


def _normalise(m: np.ndarray) -> np.ndarray:
    nrm = np.sqrt((m * m).sum(axis=0, keepdims=True))
    nrm[nrm == 0.0] = 1.0
    return m / nrm


def cell_centres(n: int, length: float = 1.0) -> np.ndarray:
    """Midpoints of `n` equal cells on [0, length]."""
    return (np.arange(n) + 0.5) * (length / n)


def random_unit_m(n, seed: int) -> np.ndarray:
    """Gaussian vector per cell, normalised to unit length: [3][n3][n2][n1] float32."""
    n1, n2, n3 = n
    g = normal(seed, 3 * n1 * n2 * n3).reshape(3, n3, n2, n1)
    return _normalise(g).astype(np.float32)


def uniform_m(n, axis: int = 2) -> np.ndarray:
    """Uniform magnetization along `axis` (0 = x, 1 = y, 2 = z)."""
    n1, n2, n3 = n
    m = np.zeros((3, n3, n2, n1), dtype=np.float32)
    m[axis] = 1.0
    return m


def vortex_m(n, seed: int, noise: float = 0.05, h=None) -> np.ndarray:
    """Vortex state (-y, x, 0.1)/norm about the domain centre plus Gaussian noise.

    `noise` * N(0,1) is added to every component before the final
    normalisation.  Coordinates are cell centres of a domain with cell sizes
    `h` (default: unit edge along the longest axis, cubic cells).
    """
    n1, n2, n3 = n
    if h is None:
        hh = 1.0 / max(n)
        h = (hh, hh, hh)
    x = (np.arange(n1) + 0.5) * h[0] - 0.5 * n1 * h[0]
    y = (np.arange(n2) + 0.5) * h[1] - 0.5 * n2 * h[1]
    X = np.broadcast_to(x[None, None, :], (n3, n2, n1))
    Y = np.broadcast_to(y[None, :, None], (n3, n2, n1))
    m = np.stack([-Y, X, np.full((n3, n2, n1), 0.1)])
    m = _normalise(m)
    if noise:
        m = m + noise * normal(seed, 3 * n1 * n2 * n3).reshape(3, n3, n2, n1)
        m = _normalise(m)
    return m.astype(np.float32)


def smooth_vectors(n: int, count: int, seed: int, terms: int = 8) -> np.ndarray:
    """`count` smooth vectors of length n: sum_s a_s sin(2 pi s x + theta_s).

    x are the cell centres of [0, 1]; a_s ~ N(0,1)/s, theta_s ~ U[0, 2 pi).
    Returns float32 [count][n].
    """
    x = cell_centres(n)
    a = normal(seed, count * terms).reshape(count, terms) / np.arange(1, terms + 1)
    th = 2.0 * np.pi * uniform(seed ^ 0x5DEECE66D, count * terms).reshape(count, terms)
    s = np.arange(1, terms + 1)
    v = (a[:, :, None] * np.sin(2.0 * np.pi * s[None, :, None] * x[None, None, :] + th[:, :, None])).sum(axis=1)
    return v.astype(np.float32)


def cp_inputs(n, r: int, seed: int):
    """CP magnetization: lambda [3][r] (ones) and factors U [3 comp][3 mode][r][n_p].

    Factor columns are smooth random vectors.  For unequal mode sizes the
    factor array is returned as a flat float32 buffer in (comp, mode, column,
    entry) order with per-mode length n_p, which is the ABI layout.
    """
    n1, n2, n3 = n
    lam = np.ones((3, r), dtype=np.float32)
    blocks = []
    for q in range(3):
        for p, npp in enumerate((n1, n2, n3)):
            blocks.append(smooth_vectors(npp, r, seed * 131 + 7 * q + p + 1))
    if n1 == n2 == n3:
        U = np.stack(blocks).reshape(3, 3, r, n1)
    else:
        U = np.concatenate([b.ravel() for b in blocks])
    return lam, U


def tucker_inputs(n, ranks, seed: int):
    """Tucker magnetization per component: Gaussian core [3][r3][r2][r1] and
    smooth factors, flat buffer in (comp, mode, column, entry) order."""
    n1, n2, n3 = n
    r1, r2, r3 = ranks
    core = normal(seed, 3 * r1 * r2 * r3).reshape(3, r3, r2, r1).astype(np.float32)
    blocks = []
    for q in range(3):
        for p, (npp, rp) in enumerate(zip((n1, n2, n3), (r1, r2, r3))):
            blocks.append(smooth_vectors(npp, rp, seed * 977 + 11 * q + p + 1).ravel())
    return core, np.concatenate(blocks)


def tt_inputs(n, ranks, seed: int):
    """3D tensor trains per component with Gaussian cores.

    G1 [3][r1][n1], G2 [3][r1*r2][n2] (mode-2 fibres contiguous, index
    a1*r2 + a2), G3 [3][r2][n3], all float32, scaled by 1/sqrt(rank) so that
    entries of the represented tensor are O(1).
    """
    n1, n2, n3 = n
    r1, r2 = ranks
    G1 = normal(seed, 3 * r1 * n1).reshape(3, r1, n1) / np.sqrt(r1)
    G2 = normal(seed + 1, 3 * r1 * r2 * n2).reshape(3, r1 * r2, n2) / np.sqrt(r2)
    G3 = normal(seed + 2, 3 * r2 * n3).reshape(3, r2, n3)
    return G1.astype(np.float32), G2.astype(np.float32), G3.astype(np.float32)


def tt_smooth_inputs(n, ranks, seed: int):
    """3D tensor trains per component with smooth cores (each fibre from smooth_vectors).

    Same layouts as tt_inputs; the represented tensors are smooth, like a
    magnetization sampled from a smooth field, so the potential has small TT
    ranks at moderate tolerances.
    """
    n1, n2, n3 = n
    r1, r2 = ranks
    G1 = np.stack([smooth_vectors(n1, r1, seed * 131 + q) for q in range(3)])
    G2 = np.stack([smooth_vectors(n2, r1 * r2, seed * 131 + 7 + q) for q in range(3)])
    G3 = np.stack([smooth_vectors(n3, r2, seed * 131 + 17 + q) for q in range(3)])
    return G1.astype(np.float32), G2.astype(np.float32), G3.astype(np.float32)


def uneven_batch_shapes(count: int, seed: int):
    """Mixed full-format grid shapes: cubes 32^3..192^3 and thin films.

    Returns a list of (n1, n2, n3) tuples in a fixed seeded order: every
    eighth grid is a 512x512x4 film, every eighth (offset 4) a 256x64x8 film,
    the rest cubes with edge drawn from {32, 48, ..., 192}.
    """
    u = uniform(seed, count)
    edges = np.arange(32, 193, 16)
    shapes = []
    for i in range(count):
        if i % 8 == 3:
            shapes.append((512, 512, 4))
        elif i % 8 == 7:
            shapes.append((256, 64, 8))
        else:
            e = int(edges[int(u[i] * len(edges)) % len(edges)])
            shapes.append((e, e, e))
    return shapes


def smooth_m(n) -> np.ndarray:
    """A C-infinity magnetization on the unit-edge domain (no randomness).

    Used for the collocation convergence check: m = (sin(pi y) z, cos(pi x),
    x y) with coordinates of the cell centres.
    """
    n1, n2, n3 = n
    hh = 1.0 / max(n)
    x = (np.arange(n1) + 0.5) * hh
    y = (np.arange(n2) + 0.5) * hh
    z = (np.arange(n3) + 0.5) * hh
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return np.stack([np.sin(np.pi * Y) * Z, np.cos(np.pi * X), X * Y])
