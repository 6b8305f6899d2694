"""Stray field, demag energy and its gradient (oracle; test infrastructure only).

h_d = -grad phi (Sec. 1, the line introducing Eq. poisson).  The paper's
energy study (Alg. 2 and the text after Fig. 2) discretises the stray field
and the energy "second order" without giving the stencil; the reading used
here is:

* d/dx_p by central differences (phi[i+1] - phi[i-1]) / (2 h_p) in the
  interior and the 3-point one-sided formulas
  (-3 phi[0] + 4 phi[1] - phi[2]) / (2 h_p),
  ( 3 phi[n-1] - 4 phi[n-2] + phi[n-3]) / (2 h_p) at the two end cells,
  all second-order accurate (n_p >= 3; n_p = 2 uses the two-point
  difference, n_p = 1 gives 0);
* E = -1/2 * V_cell * sum_i m_i . h_d(xi_i) (midpoint rule, V_cell = h1 h2 h3).

With phi = P m linear, E = 1/2 V m^T D P m and
grad_m E = 1/2 V (D P m + P^T D^T m).
"""
from __future__ import annotations

import numpy as np

from .full import mode_product, apply_full, apply_adjoint


def fd_matrix(n: int, hp: float) -> np.ndarray:
    """1D derivative matrix D (n x n) of the stencils in the module docstring."""
    D = np.zeros((n, n))
    if n == 1:
        return D
    if n == 2:
        D[:, 0], D[:, 1] = -1.0 / hp, 1.0 / hp
        return D
    for i in range(1, n - 1):
        D[i, i - 1], D[i, i + 1] = -0.5 / hp, 0.5 / hp
    D[0, 0:3] = np.array([-3.0, 4.0, -1.0]) / (2.0 * hp)
    D[n - 1, n - 3:n] = np.array([1.0, -4.0, 3.0]) / (2.0 * hp)
    return D


def gradient(phi: np.ndarray, h) -> np.ndarray:
    """D phi: [3, n3, n2, n1], component p = d/dx_{p+1}."""
    phi = np.asarray(phi, dtype=np.float64)
    n3, n2, n1 = phi.shape
    n = (n1, n2, n3)
    return np.stack([mode_product(phi, fd_matrix(n[p], float(h[p])), p + 1) for p in range(3)])


def gradient_adjoint(g: np.ndarray, h) -> np.ndarray:
    """D^T g = sum_p D_p^T g_p for a vector field g [3, n3, n2, n1]."""
    g = np.asarray(g, dtype=np.float64)
    _, n3, n2, n1 = g.shape
    n = (n1, n2, n3)
    return sum(mode_product(g[p], fd_matrix(n[p], float(h[p])).T, p + 1) for p in range(3))


def stray_field(phi: np.ndarray, h) -> np.ndarray:
    return -gradient(phi, h)


def energy(m: np.ndarray, phi: np.ndarray, h) -> float:
    """E = -1/2 V_cell sum m . h_d."""
    V = float(h[0]) * float(h[1]) * float(h[2])
    hd = stray_field(phi, h)
    return -0.5 * V * float((np.asarray(m, dtype=np.float64) * hd).sum())


def energy_from_m(m, n, h, R: int, c0: float = 2.15) -> float:
    return energy(m, apply_full(m, n, h, R, c0), h)


def energy_gradient(m, n, h, R: int, c0: float = 2.15) -> np.ndarray:
    """grad_m E = 1/2 V (D P m + P^T D^T m), [3, n3, n2, n1]."""
    V = float(h[0]) * float(h[1]) * float(h[2])
    m = np.asarray(m, dtype=np.float64)
    DPm = gradient(apply_full(m, n, h, R, c0), h)
    PtDtm = apply_adjoint(gradient_adjoint(m, h), n, h, R, c0)
    return 0.5 * V * (DPm + PtDtm)


def energy_tucker(core, V, n, ranks, h, R: int, c0: float = 2.15) -> float:
    """Energy of a Tucker magnetization through the structured path (Alg. 2's application, then
    the second-order energy of the study after Alg. 2): m^(q) = [[G^(q); V^(q,p)]] and
    phi = sum_{k,q} w_kq [[G^(q); T_{k,q,p} V^(q,p)]] (Eq. kron_eval_tuck) are formed densely and
    E is taken by `energy`.  core: [3][r3][r2][r1]; V: the flat ABI blocks (q, p) [r_p][n_p]."""
    from . import structured as ost

    n = tuple(int(v) for v in n)
    core = np.asarray(core, dtype=np.float64)
    w, outV = ost.apply_tucker(core, V, n, ranks, h, R, c0)
    phi = ost.tucker_output_to_full(core, w, outV)
    return energy(tucker_magnetization(core, V, n, ranks), phi, h)


def tucker_magnetization(core, V, n, ranks) -> np.ndarray:
    """The dense field [3][n3][n2][n1] of a Tucker magnetization (ABI layout of core and V)."""
    from . import structured as ost

    n = tuple(int(v) for v in n)
    core = np.asarray(core, dtype=np.float64)
    Vb = ost._split_blocks(V, n, ranks)
    return np.stack([ost.tucker_to_full(core[q], [Vb[q][p] for p in range(3)]) for q in range(3)])


def energy_tt(G1, G2, G3, n, ranks, h, R: int, c0: float = 2.15) -> float:
    """Energy of a TT magnetization (Eq. tt_3d_1, cores per component in the ABI layout) through the
    TT application (App. C, Eq. tt_3d_2 with the Toeplitz factors): m and phi formed densely, E by
    `energy`."""
    from . import structured as ost

    n = tuple(int(v) for v in n)
    w, o1, o2, o3 = ost.apply_tt(G1, G2, G3, n, ranks, h, R, c0)
    phi = ost.tt_output_to_full(w, o1, o2, o3, ranks)
    m = np.stack([ost.tt_to_full(G1[q], G2[q], G3[q], ranks) for q in range(3)])
    return energy(m, phi, h)


def fd_column_sums(n: int, hp: float) -> np.ndarray:
    """1^T D for the stencils of fd_matrix, in O(n) (no dense matrix)."""
    cs = np.zeros(n)
    if n == 1:
        return cs
    if n == 2:
        cs[0], cs[1] = -2.0 / hp, 2.0 / hp
        return cs
    cs[0:3] += np.array([-3.0, 4.0, -1.0]) / (2.0 * hp)
    cs[n - 3:n] += np.array([1.0, -4.0, 3.0]) / (2.0 * hp)
    i = np.arange(1, n - 1)
    np.add.at(cs, i - 1, -0.5 / hp)
    np.add.at(cs, i + 1, 0.5 / hp)
    return cs


def uniform_cube_energy(n: int, R: int, c0: float = 2.15) -> float:
    """Energy of the unit cube of n^3 cells magnetized along axis 3 (the case of the
    energy study after Alg. 2), by one-dimensional sums, so n can reach thousands.

    m = e3 is the rank-1 Tucker tensor 1 x 1 x 1 in component 3, so Eq. kron_eval_tuck
    gives phi = sum_k w_k (E_k 1) x (E_k 1) x (F_k 1) with w_k = c s omega_k (s = 1 on
    the unit cube; E along axes 1 and 2, F along axis 3, the component's own axis), and
    the second-order energy E = -1/2 h^3 sum m . h_d = 1/2 h^3 sum_i (D_3 phi)_i
    factorises into
        E = 1/2 h^3 sum_k w_k (1^T E_k 1)^2 (1^T D F_k 1),
    with 1^T E_k 1 = sum_d (n - |d|) E_k[d] and F_k 1 the prefix sums of the generator
    F_k[d].  Pinned against energy_tucker (the dense route) on small cubes."""
    from .full import C_POT
    from .generators import gen_E, gen_F
    from .quadrature import sinc_nodes

    if R < 5 or R % 2 == 0:
        raise ValueError("R must be odd and >= 5")
    M = (R - 1) // 2
    h = 1.0 / n
    _, _, tau, omega = sinc_nodes(M, c0)
    cs = fd_column_sums(n, h)
    d = np.arange(-(n - 1), n)
    mult = (n - np.abs(d)).astype(np.float64)
    i = np.arange(n)
    total = 0.0
    for k in range(M):
        sE = float(mult @ gen_E(tau[k], h, n))
        prefix = np.concatenate([[0.0], np.cumsum(gen_F(tau[k], h, n))])
        F1 = prefix[i + n] - prefix[i]  # (F 1)_i = sum_{j < n} F[i - j], generator index i - j + n - 1
        total += C_POT * omega[k] * sE * sE * float(cs @ F1)
    return 0.5 * h ** 3 * total
