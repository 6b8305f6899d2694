"""Pins of the oracle's full-format operator against things the paper and the
mathematics fix: the exact collocation integrals (closed form), the dense
quadrature matrix built entry by entry, the uniformly magnetized box, the
quadratic convergence of Lemma 1, skew symmetry and the adjoint."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import exact, full

FACTS = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_facts.json")))


def _gl(a, b, k):
    x, w = np.polynomial.legendre.leggauss(k)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


def test_rect_W_against_gauss_legendre():
    rng = np.random.default_rng(1)
    for _ in range(20):
        u0, v0 = rng.uniform(-2, 2, 2)
        u1, v1 = u0 + rng.uniform(0.1, 1), v0 + rng.uniform(0.1, 1)
        w = rng.uniform(0.5, 2)
        xu, wu = _gl(u0, u1, 40)
        xv, wv = _gl(v0, v1, 40)
        ref = (wu[:, None] * wv[None, :] / np.sqrt(xu[:, None] ** 2 + xv[None, :] ** 2 + w * w)).sum()
        assert exact.rect_integral(u0, u1, v0, v1, w) == pytest.approx(ref, rel=1e-12)


def test_box_G_against_gauss_legendre_separated_cells():
    hh = 0.1
    for q in range(3):
        for d in [(3, 0, 0), (0, -2, 1), (2, 2, -3), (-4, 1, 0)]:
            lo = [(d[p] - 0.5) * hh for p in range(3)]
            hi = [(d[p] + 0.5) * hh for p in range(3)]
            pts = [_gl(lo[p], hi[p], 24) for p in range(3)]
            X = np.meshgrid(*[pt[0] for pt in pts], indexing="ij")
            W = np.einsum("i,j,k->ijk", *[pt[1] for pt in pts])
            r = np.sqrt(X[0] ** 2 + X[1] ** 2 + X[2] ** 2)
            ref = (W * X[q] / r ** 3).sum()
            got = exact.box_G(q, lo, hi)
            assert got == pytest.approx(ref, rel=1e-10, abs=1e-15)


def test_exact_table_skew_symmetric_and_zero_self_term():
    n, hh = (4, 5, 3), (0.2, 0.25, 0.3)
    for q in range(3):
        Gt = exact.G_table(q, n, hh)
        assert np.allclose(Gt, -Gt[::-1, ::-1, ::-1], atol=1e-15 * np.abs(Gt).max())
        assert abs(Gt[n[2] - 1, n[1] - 1, n[0] - 1]) < 1e-15  # diagonal (Sec. 4.2 odd integrand)


def test_uniform_box_closed_form_equals_exact_collocation():
    n, h = (6, 5, 4), (0.1, 0.12, 0.15)
    for axis in range(3):
        m = synth.uniform_m(n, axis).astype(np.float64)
        a = exact.uniform_box_potential(n, h, axis)
        b = exact.collocation_exact(m, n, h)
        assert np.max(np.abs(a - b)) < 1e-13 * np.max(np.abs(a))


def test_kronecker_equals_dense_entrywise_matrix():
    # Cor. 3 footnote: index order; a transposed or permuted mode would fail on this
    # non-cubic, anisotropic grid.
    n, h = (3, 4, 5), (0.1, 0.07, 0.05)
    rng = np.random.default_rng(0)
    m = rng.standard_normal((3, 5, 4, 3))
    D = full.dense_operator(n, h, 11)
    ref = sum(D[q] @ m[q].ravel() for q in range(3)).reshape(5, 4, 3)
    got = full.apply_full(m, n, h, 11)
    assert np.max(np.abs(got - ref)) < 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("n,h", [((8, 8, 8), (1 / 8,) * 3), ((7, 5, 6), (2e-9, 3e-9, 2.5e-9))])
def test_kronecker_converges_to_exact_collocation(n, h):
    # Lemma 2 / Cor. 3: the separable operator converges exponentially in the rank to
    # the exact collocation matrix (checks sign, the constant 1/(2 pi^{3/2}), the
    # weights with theta, the generators and the domain scaling).
    rng = np.random.default_rng(3)
    m = rng.standard_normal((3, n[2], n[1], n[0]))
    ref = exact.collocation_exact(m, n, h)
    errs = []
    for R in (11, 21, 41, 61):
        got = full.apply_full(m, n, h, R)
        errs.append(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    assert all(errs[i + 1] < 0.1 * errs[i] for i in range(3))
    assert errs[-1] < 1e-7


def test_uniform_cube_c1_closed_form():
    # The 16^3 case: for uniform m collocation is exact, so the only error is the
    # quadrature error (R = 41).
    n, h = (16, 16, 16), (1 / 16,) * 3
    m = synth.uniform_m(n, 2).astype(np.float64)
    ref = exact.uniform_box_potential(n, h, 2)
    got = full.apply_full(m, n, h, 41)
    assert np.max(np.abs(got - ref)) < 1e-6 * np.max(np.abs(ref))
    # positive at the top (n.m = +1 there): the sign of Eq. intop1
    assert ref[-1].mean() > 0 > ref[0].mean()


def test_brute_force_c1_gaussian():
    # 16^3 Gaussian unit m: Kronecker (R = 41) vs the O(N^2) exact sum.
    n, h = (16, 16, 16), (1 / 16,) * 3
    m = synth.random_unit_m(n, 1212).astype(np.float64)
    ref = exact.collocation_exact(m, n, h)
    got = full.apply_full(m, n, h, 41)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-5


def test_collocation_quadratic_convergence():
    # Lemma 1: smooth m, nested grids refined by 3 (coarse centres are fine
    # centres); successive differences shrink by ~3^2.
    order = FACTS["collocation_order"]["value"]
    vals = {}
    for n in (2, 6, 18, 54):
        N = (n, n, n)
        phi = exact.collocation_exact(synth.smooth_m(N), N, (1 / n,) * 3, method="fft")
        f = n // 2
        idx = np.array([f // 2, f + f // 2]) if n > 2 else np.array([0, 1])
        vals[n] = phi[np.ix_(idx, idx, idx)]
    d = [np.abs(vals[a] - vals[b]).max() for a, b in ((2, 6), (6, 18), (18, 54))]
    ratio = d[1] / d[2]
    assert 3 ** order * 0.85 < ratio < 3 ** order * 1.15


def test_skew_symmetry_and_adjoint():
    n, h, R = (5, 4, 6), (0.1, 0.1, 0.1), 21
    rng = np.random.default_rng(5)
    m = rng.standard_normal((3, 6, 4, 5))
    y = rng.standard_normal((6, 4, 5))
    Pm = full.apply_full(m, n, h, R)
    Pty = full.apply_adjoint(y, n, h, R)
    lhs, rhs = (Pm * y).sum(), (m * Pty).sum()
    assert lhs == pytest.approx(rhs, rel=1e-12)
    # each component is skew: (P^(q))^T = -P^(q)
    for q in range(3):
        e = np.zeros((3, 6, 4, 5))
        e[q] = y
        assert np.allclose(Pty[q], -full.apply_full(e, n, h, R), rtol=1e-12, atol=1e-14)


def test_uniform_cube_energy_order():
    # Text after Fig. 2: energy error ~ order 1.5 for uniform magnetization, limit 1/6.
    from oracle import energy
    target = FACTS["uniform_cube_energy"]["value"]
    errs = []
    for n in (32, 64, 128):
        h = (1 / n,) * 3
        m = synth.uniform_m((n, n, n), 2).astype(np.float64)
        phi = exact.uniform_box_potential((n, n, n), h, 2)
        errs.append(abs(energy.energy(m, phi, h) - target))
    assert errs[0] > errs[1] > errs[2]
    assert errs[-1] < 2e-5
    order = np.log2(errs[1] / errs[2])
    assert abs(order - FACTS["energy_error_order"]["value"]) < 0.3


def test_sampled_lines_equal_full_apply():
    n, h, R = (9, 7, 6), (0.1, 0.1, 0.1), 21
    rng = np.random.default_rng(8)
    m = rng.standard_normal((3, 6, 7, 9))
    ref = full.apply_full(m, n, h, R)
    lines = [(0, 0), (5, 6), (2, 3)]
    got = full.apply_full_lines(m, n, h, R, lines)
    for idx, (i3, i2) in enumerate(lines):
        assert np.allclose(got[idx], ref[i3, i2], rtol=1e-12, atol=1e-14)
