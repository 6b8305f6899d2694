"""Pins of the oracle's structured-format application: each output represents
exactly the full-format result on the formed input (Eq. kron_eval_cp,
Eq. kron_eval_tuck, Eq. tt_3d_2), and TT equals its Tucker2 form."""
import numpy as np
import pytest

import synth
from oracle import full, structured as S
from oracle import energy as En

N = (12, 10, 9)
H = (0.1, 0.1, 0.1)
R = 21


def test_cp_matches_full():
    r = 3
    lam, U = synth.cp_inputs(N, r, 1215)
    blocks = S._split_blocks(U, N, (r, r, r))
    m = np.stack([S.cp_to_full(lam[q], blocks[q]) for q in range(3)])
    ref = full.apply_full(m, N, H, R)
    w, outU = S.apply_cp(lam, U, N, H, R)
    got = S.cp_output_to_full(w, outU)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))
    # Gram-matrix inner products agree with the formed tensors
    M = w.shape[0]
    f = [outU[p].reshape(M * 3 * r, -1) for p in range(3)]
    assert S.cp_inner(w.ravel(), f, w.ravel(), f) == pytest.approx((got * got).sum(), rel=1e-11)


def test_cp_entries_equal_apply_cp():
    # sampled entries read off generator rows equal the dense-matrix products
    r = 2
    n = (12, 31, 9)
    lam, U = synth.cp_inputs(n, r, 1219)
    w, outU = S.apply_cp(lam, U, n, H, R)
    for p, idx in ((0, [0, 5, 11]), (1, [0, 17, 30]), (2, [8])):
        got = S.apply_cp_entries(lam, U, n, H, R, p, idx)
        ref = outU[p][..., idx]
        assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_tucker_matches_full():
    ranks = (3, 2, 4)
    core, V = synth.tucker_inputs(N, ranks, 1216)
    blocks = S._split_blocks(V, N, ranks)
    m = np.stack([S.tucker_to_full(core[q], blocks[q]) for q in range(3)])
    ref = full.apply_full(m, N, H, R)
    w, outV = S.apply_tucker(core, V, N, ranks, H, R)
    got = S.tucker_output_to_full(core, w, outV)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_tt_matches_full_and_tucker2():
    ranks = (3, 2)
    G1, G2, G3 = synth.tt_inputs(N, ranks, 1217)
    m = np.stack([S.tt_to_full(G1[q], G2[q], G3[q], ranks) for q in range(3)])
    ref = full.apply_full(m, N, H, R)
    w, o1, o2, o3 = S.apply_tt(G1, G2, G3, N, ranks, H, R)
    got = S.tt_output_to_full(w, o1, o2, o3, ranks)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))
    # Eq. tt_3d_2: the TT is the Tucker2 tensor [[G2; G1, id, G3^T]]
    for q in range(3):
        core = np.asarray(G2[q], dtype=np.float64).reshape(ranks[0], ranks[1], N[1]).transpose(1, 2, 0)
        # core[c][b][a] ordering [r3][r2][r1] with r2 := n2 and identity factor
        t2 = S.tucker_to_full(core, [G1[q], np.eye(N[1]), G3[q]])
        assert np.allclose(t2, S.tt_to_full(G1[q], G2[q], G3[q], ranks), rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------- energy

def test_fd_stencils_exact_on_quadratics():
    n, hp = 7, 0.3
    x = (np.arange(n) + 0.5) * hp
    D = En.fd_matrix(n, hp)
    for f, df in ((x ** 2, 2 * x), (3 * x + 1, 3 + 0 * x)):
        assert np.allclose(D @ f, df, rtol=1e-12, atol=1e-12)


def test_energy_gradient_vs_central_differences():
    # central finite differences with step 1e-4 in float64 on a 6^3 grid
    n, h, R2 = (6, 6, 6), (1 / 6,) * 3, 21
    m = synth.random_unit_m(n, 1217).astype(np.float64)
    g = En.energy_gradient(m, n, h, R2)
    rng = np.random.default_rng(2)
    eps = 1e-4
    for _ in range(6):
        idx = (rng.integers(3), rng.integers(6), rng.integers(6), rng.integers(6))
        mp, mm = m.copy(), m.copy()
        mp[idx] += eps
        mm[idx] -= eps
        fd = (En.energy_from_m(mp, n, h, R2) - En.energy_from_m(mm, n, h, R2)) / (2 * eps)
        assert fd == pytest.approx(g[idx], rel=1e-6, abs=1e-12)
    # a random direction
    v = rng.standard_normal(m.shape)
    fd = (En.energy_from_m(m + eps * v, n, h, R2) - En.energy_from_m(m - eps * v, n, h, R2)) / (2 * eps)
    assert fd == pytest.approx((g * v).sum(), rel=1e-7)


def test_gradient_adjoint_dot_product():
    h = (0.1, 0.2, 0.3)
    rng = np.random.default_rng(4)
    phi = rng.standard_normal((4, 5, 6))
    g = rng.standard_normal((3, 4, 5, 6))
    assert (En.gradient(phi, h) * g).sum() == pytest.approx((phi * En.gradient_adjoint(g, h)).sum(), rel=1e-12)
