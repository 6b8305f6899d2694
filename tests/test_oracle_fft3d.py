"""Pins of the oracle's 3D FFT convolution (oracle/fft3d.py, Eq. fft_pot).

1. It is the same operator as the Kronecker mode products of Eq. kron_operator
   (oracle.full, itself pinned to brute force and closed forms) on ragged,
   non-cubic grids, to rounding.
2. It matches the exact collocation sum (O(N^2) brute force with the exact
   cell integrals) within the sinc-quadrature error.
3. Any padded length L_p >= 2 n_p - 1 gives the same result; L_p = 2 n_p - 2
   aliases and does not.
4. The dense kernel K^(q) is purely imaginary, odd in w_q and even in the
   other frequencies (E even and real-symmetric, F odd), the symmetry the GPU
   kernel's octant storage relies on.
"""
import numpy as np
import pytest

import synth
from oracle import exact, fft3d, full

SHAPES = [((7, 5, 6), (2e-9, 3e-9, 2.5e-9)), ((1, 4, 9), (0.1, 0.2, 0.05)), ((16, 3, 2), (1.0, 1.0, 3.0))]


@pytest.mark.parametrize("n,h", SHAPES)
def test_equals_kronecker_mode_products(n, h):
    rng = np.random.default_rng(11)
    m = rng.standard_normal((3, n[2], n[1], n[0]))
    ref = full.apply_full(m, n, h, 21)
    got = fft3d.apply_fft3d(m, n, h, 21)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_matches_exact_collocation():
    n, h = (6, 5, 7), (1.0, 1.2, 0.9)
    m = synth.random_unit_m(n, seed=4).astype(np.float64)
    ref = exact.collocation_exact(m, n, h)
    got = fft3d.apply_fft3d(m, n, h, 41)
    assert np.linalg.norm(got - ref) < 1e-5 * np.linalg.norm(ref)


def test_padding_length():
    n, h = (5, 6, 3), (1.0, 1.0, 1.0)
    rng = np.random.default_rng(2)
    m = rng.standard_normal((3, n[2], n[1], n[0]))
    ref = fft3d.apply_fft3d(m, n, h, 11)
    exact_L = tuple(2 * v - 1 for v in n)          # odd, not a power of two
    got = fft3d.apply_fft3d(m, n, h, 11, K=fft3d.dense_kernel(n, h, 11, L=exact_L))
    assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)
    short = (2 * n[0] - 2, exact_L[1], exact_L[2])  # one axis too short: the ends wrap
    bad = fft3d.apply_fft3d(m, n, h, 11, K=fft3d.dense_kernel(n, h, 11, L=short))
    assert np.linalg.norm(bad - ref) > 1e-4 * np.linalg.norm(ref)


def test_kernel_symmetry():
    n, h = (6, 4, 5), (1.0, 0.7, 1.3)
    K = fft3d.dense_kernel(n, h, 21)
    scale = np.abs(K).max()
    assert np.abs(K.real).max() <= 1e-13 * scale
    for q in range(3):
        Kq = K[q].imag                     # [L3, L2, L1]
        for p in range(3):
            ax = 2 - p
            mirrored = np.roll(np.flip(Kq, axis=ax), 1, axis=ax)   # w_p -> L_p - w_p
            sign = -1.0 if p == q else 1.0
            assert np.abs(mirrored - sign * Kq).max() <= 1e-13 * scale, (q, p)


def _fft_vs_modes():
    n, h = (7, 5, 6), (2e-9, 3e-9, 2.5e-9)
    rng = np.random.default_rng(11)
    m = rng.standard_normal((3, n[2], n[1], n[0]))
    ref = full.apply_full(m, n, h, 21)
    got = fft3d.apply_fft3d(m, n, h, 21)
    return np.linalg.norm(got - ref) / np.linalg.norm(ref)


def test_planted_mistakes_are_caught(monkeypatch):
    """Each plausible mistake in the FFT oracle breaks pin 1."""
    orig_col, orig_fft = fft3d.circulant_column, np.fft.fft

    def col_reversed(gen, n, L):          # kernel placed as g[-d]: F's sign flips
        return orig_col(gen[::-1], n, L)

    def col_shifted(gen, n, L):           # d = 0 at index 1
        return np.roll(orig_col(gen, n, L), 1)

    def conj_fft(x, *a, **k):             # inverse-direction kernel transform
        return np.conj(orig_fft(x, *a, **k))

    def padded_short(n):                  # L_p = 2 n_p - 2
        return tuple(max(2 * int(v) - 2, 2) for v in n)

    mutations = [
        ("circulant_column", col_reversed),
        ("circulant_column", col_shifted),
        ("padded_lengths", padded_short),
    ]
    for name, fn in mutations:
        with monkeypatch.context() as mp:
            mp.setattr(fft3d, name, fn)
            assert _fft_vs_modes() > 1e-3, name
    with monkeypatch.context() as mp:
        mp.setattr(fft3d.np.fft, "fft", conj_fft)
        assert _fft_vs_modes() > 1e-3, "conj"
    # the kernel of component q dropped into the slot of q + 1
    orig_kind = fft3d.factor_kind
    with monkeypatch.context() as mp:
        mp.setattr(fft3d, "factor_kind", lambda p, q: orig_kind(p, (q + 1) % 3))
        assert _fft_vs_modes() > 1e-3, "component"
    assert _fft_vs_modes() < 1e-12


@pytest.mark.parametrize("n,h", SHAPES[:2])
def test_field_by_fft_equals_the_kronecker_field(n, h):
    from oracle import field as ofield
    rng = np.random.default_rng(12)
    m = rng.standard_normal((3, n[2], n[1], n[0]))
    ref = ofield.apply_field(m, n, h, 21)
    got = fft3d.apply_field_fft3d(m, n, h, 21)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_field_kernels_real_symmetric_and_parities():
    # K_pq real, K_pq = K_qp, odd in w_p and w_q for p != q, even otherwise
    n, h = (6, 4, 5), (1.0, 0.7, 1.3)
    K = fft3d.dense_field_kernels(n, h, 21)
    scale = np.abs(K).max()
    assert np.abs(K.imag).max() <= 1e-13 * scale
    for p in range(3):
        for q in range(3):
            assert np.abs(K[p, q] - K[q, p]).max() <= 1e-13 * scale
            Kr = K[p, q].real
            for a in range(3):
                ax = 2 - a
                mirrored = np.roll(np.flip(Kr, axis=ax), 1, axis=ax)
                odd = (p != q) and (a == p or a == q)
                assert np.abs(mirrored - (-Kr if odd else Kr)).max() <= 1e-13 * scale, (p, q, a)
