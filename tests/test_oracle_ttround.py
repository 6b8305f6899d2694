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


def test_known_tt_rank_is_recovered_exactly():
    # a tensor built as a train of ranks (2, 3) has exactly those TT ranks (generic cores):
    # rounding at a tiny tolerance recovers them and the tensor
    rng = np.random.default_rng(3)
    n1, n2, n3 = 9, 8, 7
    A = rng.standard_normal((2, n1))
    B = rng.standard_normal((2 * 3, n2))
    C = rng.standard_normal((3, n3))
    X = ost.tt_to_full(A, B, C, (2, 3))
    G1, G2, G3, rk = otr.tt_round_dense(X, 1e-12)
    assert rk == (2, 3)
    assert np.linalg.norm(ost.tt_to_full(G1, G2, G3, rk) - X) <= 1e-12 * np.linalg.norm(X)


def test_cores_are_left_orthonormal_and_first_truncation_is_optimal():
    X, _ = _phi()
    G1, G2, G3, (r1, r2) = otr.tt_round_dense(X, 1e-3)
    assert np.allclose(G1 @ G1.T, np.eye(r1), atol=1e-12)
    n2 = X.shape[1]
    L = G2.reshape(r1, r2, n2).transpose(0, 2, 1).reshape(r1 * n2, r2)
    assert np.allclose(L.T @ L, np.eye(r2), atol=1e-12)
    # Eckart-Young: projecting the first unfolding on G1 leaves exactly the discarded singular values
    n3, _, n1 = X.shape
    X1 = X.transpose(2, 1, 0).reshape(n1, -1)
    s = np.linalg.svd(X1, compute_uv=False)
    resid = np.linalg.norm(X1 - G1.T @ (G1 @ X1))
    assert abs(resid - np.sqrt(np.sum(s[r1:] ** 2))) <= 1e-10 * np.linalg.norm(X1)
