"""Pins of the oracle's TT conversions and Hadamard product (oracle/ttround.py), App. C:
each TT result, formed densely by Eq. tt_3d_1, equals the dense Tucker / CP tensor or the
element-wise product of the dense factors (independent oracle routines)."""
import numpy as np

from oracle import structured as ost
from oracle import ttround as otr


def test_tucker_to_tt_represents_the_tucker_tensor():
    rng = np.random.default_rng(5)
    r, n = (2, 3, 4), (7, 6, 5)
    C = rng.standard_normal((r[2], r[1], r[0]))
    V = [rng.standard_normal((r[p], n[p])) for p in range(3)]
    G1, G2, G3 = otr.tucker_to_tt(C, *V)
    assert np.allclose(ost.tt_to_full(G1, G2, G3, (r[0], r[2])), ost.tucker_to_full(C, V), atol=1e-12)


def test_cp_to_tt_represents_the_cp_tensor():
    rng = np.random.default_rng(6)
    rk, n = 3, (5, 4, 6)
    lam = rng.standard_normal(rk)
    U = [rng.standard_normal((rk, n[p])) for p in range(3)]
    G1, G2, G3 = otr.cp_to_tt(lam, *U)
    dense = np.einsum("l,li,lj,lk->kji", lam, U[0], U[1], U[2])
    assert np.allclose(ost.tt_to_full(G1, G2, G3, (rk, rk)), dense, atol=1e-12)


def test_hadamard_is_the_elementwise_product():
    rng = np.random.default_rng(7)
    n, ra, rb = (4, 5, 3), (2, 3), (3, 1)
    A = (rng.standard_normal((ra[0], n[0])), rng.standard_normal((ra[0] * ra[1], n[1])),
         rng.standard_normal((ra[1], n[2])))
    B = (rng.standard_normal((rb[0], n[0])), rng.standard_normal((rb[0] * rb[1], n[1])),
         rng.standard_normal((rb[1], n[2])))
    C = otr.tt_hadamard(A, ra, B, rb)
    lhs = ost.tt_to_full(*C, (ra[0] * rb[0], ra[1] * rb[1]))
    rhs = ost.tt_to_full(*A, ra) * ost.tt_to_full(*B, rb)
    assert np.allclose(lhs, rhs, atol=1e-12)
