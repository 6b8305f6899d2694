"""Sinc quadrature of the Gaussian transform (oracle; test infrastructure only).

Sec. 3.3 (Eq. sinc_int, Thm. 1 / Eq. quad_err), Sec. 3.4 (Eq. gauss_trans,
Lemma 2: substitution tau = sinh t) and Cor. 3 (Eq. kron_operator: nodes
t_k = k theta, theta = c0 log(R)/R).

Reading (see package docstring): the symmetric rule has R = 2M+1 nodes
k = -M..M.  The integrand of Eq. gauss_trans after tau = sinh t,
cosh(t) sinh(t)^2 exp(-sinh(t)^2 rho), is even in t and vanishes at t = 0, so
the rule equals

    int_R tau^2 exp(-tau^2 rho) dtau  ~=  sum_{k=1..M} omega_k exp(-tau_k^2 rho),
    tau_k = sinh(k theta),  omega_k = 2 theta cosh(k theta) sinh(k theta)^2,

and theta = c0 ln(M) / M.
"""
from __future__ import annotations

import numpy as np


def sinc_nodes(M: int, c0: float = 2.15):
    """Nodes and folded weights of the M-term rule.

    Returns (theta, t, tau, omega) with t, tau, omega float64 arrays of length M
    (k = 1..M).  Requires M >= 2 (ln 1 = 0 would give a zero step).
    """
    if M < 2:
        raise ValueError("the rule needs M >= 2 (R = 2M+1 >= 5)")
    if not c0 > 0:
        raise ValueError("c0 must be positive")
    theta = c0 * np.log(M) / M
    t = theta * np.arange(1, M + 1, dtype=np.float64)
    tau = np.sinh(t)
    omega = 2.0 * theta * np.cosh(t) * tau * tau
    return theta, t, tau, omega


def inv_rho32(rho, M: int, c0: float = 2.15):
    """Quadrature approximation of rho^{-3/2} from Eq. gauss_trans:

        rho^{-3/2} = (2/sqrt(pi)) int_R tau^2 exp(-tau^2 rho) dtau.
    """
    _, _, tau, omega = sinc_nodes(M, c0)
    rho = np.asarray(rho, dtype=np.float64)
    return (2.0 / np.sqrt(np.pi)) * (omega[None, :] * np.exp(-np.outer(rho.ravel(), tau * tau))).sum(axis=1).reshape(rho.shape)


def max_rel_error(M: int, rho_min: float, rho_max: float = 3.0, c0: float = 2.15, samples: int = 400):
    """max over log-spaced rho in [rho_min, rho_max] of |Q_M(rho) rho^{3/2} - 1|.

    This is the quantity plotted in Fig. 1 (relative error of the sinc
    quadrature of Eq. gauss_trans, rho_max = 3 for the unit cube, Sec. 3.4).
    """
    rho = np.geomspace(rho_min, rho_max, samples)
    return float(np.max(np.abs(inv_rho32(rho, M, c0) * rho ** 1.5 - 1.0)))
