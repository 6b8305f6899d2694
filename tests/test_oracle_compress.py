"""Pins of the oracle's compressed-kernel Alg. 2 (oracle/compress.py).

1. At full rank (tol -> 0) the compressed application is the uncompressed
   structured Tucker application of oracle.structured (itself pinned to the
   Kronecker mode products), to rounding.
2. The compressed kernel obeys the HOSVD bound ||K - K_tucker|| <= tol ||K||,
   and HOOI does not lose accuracy against its HOSVD start.
3. The potential error shrinks with tol and stays within a small multiple of it.
4. App. B Eq. t_had2 (Tucker Hadamard product) and Lemma DFT_tucker hold for
   the index conventions used (checked against dense tensors and numpy FFTs).
5. Planted mistakes (Kronecker core in the wrong index order, the rank rule
   keeping the smallest singular values) break pin 1 or pin 2.
"""
import numpy as np
import pytest

import synth
from oracle import compress as oc
from oracle import structured as ost

N, H, R = (9, 7, 8), (1.0, 1.3, 0.8), 21
RANKS = (3, 2, 4)


def _tucker_in():
    core, flat = synth.tucker_inputs(N, RANKS, 5)
    core = core.astype(np.float64)
    V, off = [], 0
    for q in range(3):
        row = []
        for p in range(3):
            size = RANKS[p] * N[p]
            row.append(flat[off:off + size].reshape(RANKS[p], N[p]).T.astype(np.float64))  # [n_p, r_p]
            off += size
        V.append(row)
    return core, flat, V


def _uncompressed_phi():
    core, flat, _ = _tucker_in()
    w, outV = ost.apply_tucker(core, flat, N, RANKS, H, R)
    return ost.tucker_output_to_full(core, w, outV)


def test_full_rank_equals_the_uncompressed_application():
    core, _, V = _tucker_in()
    ranks, comp = oc.compress_kernels(N, H, R, 1e-14)
    _, phi = oc.apply_tucker_compressed(core, V, N, comp)
    ref = _uncompressed_phi()
    assert np.linalg.norm(phi - ref) <= 1e-11 * np.linalg.norm(ref)


@pytest.mark.parametrize("tol", [1e-2, 1e-4, 1e-7])
def test_kernel_error_bound_and_hooi_gain(tol):
    ranks, comp = oc.compress_kernels(N, H, R, tol)
    for q in range(3):
        X = oc.cp_to_dense(*oc.cp_kernel(q, N, H, R))
        C, U = comp[q]
        err = np.linalg.norm(X - oc.tucker_to_dense(C, U))
        assert err <= tol * np.linalg.norm(X) * (1 + 1e-9), (q, err / np.linalg.norm(X))
        spec = oc.hosvd_spectra(X)
        Uh = [spec[p][0][:, : ranks[p]] for p in range(3)]
        Ch = X
        for p in range(3):
            Ch = oc.mode_mult(Ch, Uh[p].T, p)
        assert err <= np.linalg.norm(X - oc.tucker_to_dense(Ch, Uh)) * (1 + 1e-9) + 1e-13 * np.linalg.norm(X)


def test_potential_error_follows_tol():
    core, _, V = _tucker_in()
    ref = _uncompressed_phi()
    errs, prev_ranks = [], None
    for tol in (1e-2, 1e-4, 1e-6):
        ranks, comp = oc.compress_kernels(N, H, R, tol)
        _, phi = oc.apply_tucker_compressed(core, V, N, comp)
        errs.append(np.linalg.norm(phi - ref) / np.linalg.norm(ref))
        assert errs[-1] <= 10 * tol
        if prev_ranks is not None:
            assert all(a >= b for a, b in zip(ranks, prev_ranks))
        prev_ranks = ranks
    assert errs[0] > errs[1] > errs[2]


def test_tucker_hadamard_and_dft_lemma():
    rng = np.random.default_rng(1)
    n = (5, 4, 6)
    C = rng.standard_normal((2, 3, 2))
    D = rng.standard_normal((3, 1, 2))
    U = [rng.standard_normal((n[p], C.shape[2 - p])) for p in range(3)]
    Vf = [rng.standard_normal((n[p], D.shape[2 - p])) for p in range(3)]
    E, W = oc.tucker_hadamard(C, U, D, Vf)
    assert np.allclose(oc.tucker_to_dense(E, W), oc.tucker_to_dense(C, U) * oc.tucker_to_dense(D, Vf))
    Xh = np.fft.fftn(oc.tucker_to_dense(C, U), axes=(0, 1, 2))
    Uh = [np.fft.fft(U[p], axis=0) for p in range(3)]
    assert np.allclose(oc.tucker_to_dense(C.astype(complex), Uh), Xh)


def test_planted_mistakes_are_caught(monkeypatch):
    core, _, V = _tucker_in()
    ref = _uncompressed_phi()
    orig_einsum = np.einsum

    def l_major(spec, *ops, **kw):  # core Kronecker index (l, i) instead of (i, l)
        if spec == "abc,def->adbecf":
            spec = "abc,def->dafbec"
        return orig_einsum(spec, *ops, **kw)

    with monkeypatch.context() as mp:
        mp.setattr(oc.np, "einsum", l_major)
        ranks, comp = oc.compress_kernels(N, H, R, 1e-14)
        _, phi = oc.apply_tucker_compressed(core, V, N, comp)
        assert np.linalg.norm(phi - ref) > 1e-3 * np.linalg.norm(ref)

    orig_hooi = oc.hooi

    def smallest(X, ranks, sweeps=4):  # keeps the trailing singular vectors
        U = [oc.hosvd_spectra(X)[p][0][:, -ranks[p]:] for p in range(3)]
        C = X
        for p in range(3):
            C = oc.mode_mult(C, U[p].T, p)
        return C, U

    with monkeypatch.context() as mp:
        mp.setattr(oc, "hooi", smallest)
        ranks, comp = oc.compress_kernels(N, H, R, 1e-4)
        X = oc.cp_to_dense(*oc.cp_kernel(0, N, H, R))
        err = np.linalg.norm(X - oc.tucker_to_dense(*comp[0])) / np.linalg.norm(X)
        assert err > 1e-2
    assert oc.hooi is orig_hooi


@pytest.mark.parametrize("tol", [1e-2, 1e-4, 1e-6])
def test_recompression_bound_and_ranks(tol):
    # the summed potential of the three components (ranks 3 x 10 x 3 = 90 per mode),
    # recompressed: the HOSVD bound holds and the ranks drop below the grid size
    n, h, rk = (24, 20, 16), (1.0, 1.0, 1.0), (3, 3, 3)
    core, flat = synth.tucker_inputs(n, rk, 5)
    V, off = [], 0
    for q in range(3):
        row = []
        for p in range(3):
            size = rk[p] * n[p]
            row.append(flat[off:off + size].reshape(rk[p], n[p]).T.astype(np.float64))
            off += size
        V.append(row)
    _, comp = oc.compress_kernels(n, h, 21, 1e-8)
    parts, phi = oc.apply_tucker_compressed(core.astype(np.float64), V, n, comp)
    C, U, ranks = oc.recompress(parts, tol)
    err = np.linalg.norm(oc.tucker_to_dense(C, U) - phi) / np.linalg.norm(phi)
    assert err <= tol * (1 + 1e-9)
    assert sum(ranks) < sum(n) if tol >= 1e-4 else all(r <= n[p] for p, r in enumerate(ranks))
    for p in range(3):
        assert np.allclose(U[p].T @ U[p], np.eye(ranks[p]), atol=1e-12)
