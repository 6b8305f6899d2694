"""Pins of the oracle's TT rounding (oracle/ttround.py).

1. The rounded train is within tol of the tensor (TT-SVD bound), and exact
   (to rounding) at tol -> 0.
2. On the potential of a TT magnetization (a sum of 3M trains, ranks 3M r) the
   ranks drop far below 3M r.
3. A planted mistake (both truncations at the full tol instead of tol / sqrt(2))
   can break the bound; the unplanted rule never does.
"""
import numpy as np
import pytest

import synth
from oracle import structured as ost
from oracle import ttround as otr

N, H, R, RK = (14, 12, 10), (1.0, 1.0, 1.0), 21, (3, 3)


def _phi():
    G1, G2, G3 = synth.tt_inputs(N, RK, 7)
    w, o1, o2, o3 = ost.apply_tt(G1, G2, G3, N, RK, H, R)
    return ost.tt_output_to_full(w, o1, o2, o3, RK), w.shape[0]


@pytest.mark.parametrize("tol", [1e-2, 1e-4, 1e-8, 1e-14])
def test_rounding_bound(tol):
    X, M = _phi()
    G1, G2, G3, rk = otr.tt_round_dense(X, tol)
    Y = ost.tt_to_full(G1, G2, G3, rk)
    err = np.linalg.norm(Y - X) / np.linalg.norm(X)
    assert err <= tol * (1 + 1e-9) + 1e-14
    assert rk[0] <= N[0] and rk[1] <= N[2]
    if tol >= 1e-4:
        assert rk[0] < 3 * M * RK[0] and rk[1] < 3 * M * RK[1]


def test_planted_split_breaks_the_bound_sometimes():
    X, _ = _phi()
    worst = 0.0
    for tol in np.logspace(-6, -1, 25):
        n3, n2, n1 = X.shape
        Xt = X.transpose(2, 1, 0)
        b2 = tol ** 2 * np.sum(Xt ** 2)  # planted: full tol at each of the two steps
        U, s, Vt = np.linalg.svd(Xt.reshape(n1, -1), full_matrices=False)
        r1 = otr._rank(s, b2)
        C = (s[:r1, None] * Vt[:r1]).reshape(r1 * n2, n3)
        U2, s2, Vt2 = np.linalg.svd(C, full_matrices=False)
        r2 = otr._rank(s2, b2)
        Y = np.einsum("ia,ajb,bk->ijk", U[:, :r1], U2[:, :r2].reshape(r1, n2, r2), s2[:r2, None] * Vt2[:r2])
        worst = max(worst, np.linalg.norm(Y - Xt) / np.linalg.norm(Xt) / tol)
        G1, G2, G3, rk = otr.tt_round_dense(X, tol)
        assert np.linalg.norm(ost.tt_to_full(G1, G2, G3, rk) - X) <= tol * np.linalg.norm(X) * (1 + 1e-9)
    assert worst > 1.0
