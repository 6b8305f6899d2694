"""GPU parity of Alg. 2 with compressed kernels (demag_compress_kernel,
demag_apply_tucker_compressed) against the FP64 oracle (oracle/compress.py) and
the uncompressed structured path, through the C ABI."""
import numpy as np
import pytest

import synth
from oracle import compress as oc
from oracle import structured as ost
from gpu_helpers import dev, host, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1212_3509_gb300 as D
    return D


def _inputs(n, ranks, seed, batch=1):
    cores, flats = [], []
    for b in range(batch):
        core, flat = synth.tucker_inputs(n, ranks, seed + b)
        cores.append(core)
        flats.append(flat)
    return np.stack(cores).astype(np.float32), np.concatenate(flats).astype(np.float32)


def _factors_of(flat, n, ranks):
    V, off = [], 0
    for q in range(3):
        row = []
        for p in range(3):
            size = ranks[p] * n[p]
            row.append(flat[off:off + size].reshape(ranks[p], n[p]).T.astype(np.float64))
            off += size
        V.append(row)
    return V


def _run(D, P, n, ranks, core, flat, batch=1):
    rho = D.demag_compressed_ranks(P)
    nout = int(np.prod([rho[p] * ranks[p] for p in range(3)]))
    out_core = torch.empty(batch * 3 * nout, device="cuda")
    out_V = torch.empty(batch * sum(3 * rho[p] * ranks[p] * n[p] for p in range(3)), device="cuda")
    D.demag_apply_tucker_compressed(P, batch, ranks, dev(core.ravel()), dev(flat), out_core, out_V)
    torch.cuda.synchronize()
    return rho, host(out_core), host(out_V)


def _parts(rho, n, ranks, out_core, out_V, item=0):
    """Per-component (core [R3, R2, R1], W [n_p, R_p]) of batch item `item`, R_p = rho_p r_p."""
    Rp = [rho[p] * ranks[p] for p in range(3)]
    per_core = Rp[0] * Rp[1] * Rp[2]
    per_V = sum(3 * rho[p] * ranks[p] * n[p] for p in range(3))
    cores = out_core[item * 3 * per_core:(item + 1) * 3 * per_core].reshape(3, Rp[2], Rp[1], Rp[0]).astype(np.float64)
    flat = out_V[item * per_V:(item + 1) * per_V]
    blocks, off = [], 0
    for p in range(3):
        size = 3 * rho[p] * ranks[p] * n[p]
        blocks.append(flat[off:off + size].reshape(rho[p], 3, ranks[p], n[p]).astype(np.float64))
        off += size
    parts = []
    for q in range(3):
        W = [blocks[p][:, q].reshape(Rp[p], n[p]).T for p in range(3)]
        parts.append((cores[q], W))
    return parts


def _dense(parts):
    return sum(oc.tucker_to_dense(E, W) for E, W in parts)


N, H, R, RANKS = (9, 7, 8), (1.0, 1.3, 0.8), 21, (3, 2, 4)


@pytest.mark.parametrize("tol", [1e-2, 1e-4, 1e-6])
def test_compressed_vs_oracle(D, tol):
    P = D.demag_build_factors(N, H, R)
    D.demag_compress_kernel(P, tol)
    core, flat = _inputs(N, RANKS, 5)
    rho, oc_, oV = _run(D, P, N, RANKS, core, flat)
    ranks_ref, comp = oc.compress_kernels(N, H, R, tol)
    assert list(rho) == list(ranks_ref)
    V = _factors_of(flat, N, RANKS)
    _, phi_ref = oc.apply_tucker_compressed(core[0].astype(np.float64), V, N, comp)
    phi = _dense(_parts(rho, N, RANKS, oc_, oV))
    assert rel_l2(phi, phi_ref) <= max(2 * tol, 2e-6)
    w, outV = ost.apply_tucker(core[0].astype(np.float64), flat, N, RANKS, H, R)
    exact = ost.tucker_output_to_full(core[0].astype(np.float64), w, outV)
    assert rel_l2(phi, exact) <= 10 * tol


@pytest.mark.parametrize("tol", [1e-3, 1e-6])
def test_compressed_kernel_bound(D, tol):
    n, h = (12, 10, 16), (1.0, 1.0, 1.0)
    P = D.demag_build_factors(n, h, 31)
    D.demag_compress_kernel(P, tol)
    rho = D.demag_compressed_ranks(P)
    glen = 2 * max(n) - 1
    gen = torch.empty(max(rho) * 9 * glen, dtype=torch.float64, device="cuda")
    core = torch.empty(3 * rho[0] * rho[1] * rho[2], device="cuda")
    D.demag_copy_compressed(P, gen, core)
    g = host(gen).reshape(max(rho), 3, 3, glen)
    C = host(core).reshape(3, rho[2], rho[1], rho[0]).astype(np.float64)
    for q in range(3):
        U = [g[: rho[p], q, p, : 2 * n[p] - 1].T for p in range(3)]
        K = oc.cp_to_dense(*oc.cp_kernel(q, n, h, 31))
        err = np.linalg.norm(oc.tucker_to_dense(C[q], U) - K) / np.linalg.norm(K)
        assert err <= tol * 1.05 + 1e-6, (q, err)
        for p in range(3):  # orthonormal factors
            assert np.allclose(U[p].T @ U[p], np.eye(rho[p]), atol=1e-10)


def test_full_rank_matches_uncompressed(D):
    P = D.demag_build_factors(N, H, R)
    D.demag_compress_kernel(P, 1e-12)
    core, flat = _inputs(N, RANKS, 8)
    rho, oc_, oV = _run(D, P, N, RANKS, core, flat)
    phi = _dense(_parts(rho, N, RANKS, oc_, oV))
    w, outV = ost.apply_tucker(core[0].astype(np.float64), flat, N, RANKS, H, R)
    assert rel_l2(phi, ost.tucker_output_to_full(core[0].astype(np.float64), w, outV)) <= 1e-5


def test_batch_equals_single_items(D):
    n, ranks = (33, 20, 17), (3, 4, 2)
    P = D.demag_build_factors(n, (1.0, 1.0, 1.0), 31)
    D.demag_compress_kernel(P, 1e-5)
    core, flat = _inputs(n, ranks, 21, batch=3)
    rho, cb, Vb = _run(D, P, n, ranks, core, flat, batch=3)
    per_in = len(flat) // 3
    for b in range(3):
        _, c1, V1 = _run(D, P, n, ranks, core[b:b + 1], flat[b * per_in:(b + 1) * per_in])
        pb = _parts(rho, n, ranks, cb, Vb, item=b)
        p1 = _parts(rho, n, ranks, c1, V1)
        for (E_b, W_b), (E_1, W_1) in zip(pb, p1):
            assert np.array_equal(E_b, E_1)
            for p in range(3):
                assert np.array_equal(W_b[p], W_1[p])


def test_tucker_1024_against_the_uncompressed_gpu_path(D):
    # the measured workload: n = 1024, ranks (8, 8, 8), R = 61; phi compared at sampled points
    n, ranks, R61, tol = (1024, 1024, 1024), (8, 8, 8), 61, 1e-6
    h = (1.0 / 1024,) * 3
    P = D.demag_build_factors(n, h, R61)
    D.demag_compress_kernel(P, tol)
    core, flat = _inputs(n, ranks, 3)
    rho, oc_, oV = _run(D, P, n, ranks, core, flat)
    parts = _parts(rho, n, ranks, oc_, oV)
    M = P.M
    out_w = torch.empty(M * 3, device="cuda")
    out_V = torch.empty(M * 3 * sum(ranks[p] * n[p] for p in range(3)), device="cuda")
    D.demag_apply_tucker(P, ranks, dev(flat), out_w, out_V)
    torch.cuda.synchronize()
    w = host(out_w).reshape(M, 3).astype(np.float64)
    blocks, off = [], 0
    oVh = host(out_V)
    for p in range(3):
        size = M * 3 * ranks[p] * n[p]
        blocks.append(oVh[off:off + size].reshape(M, 3, ranks[p], n[p]).astype(np.float64))
        off += size
    rng = np.random.default_rng(0)
    pts = rng.integers(0, 1024, size=(24, 3))
    G = core[0].astype(np.float64)
    num = den = 0.0
    for i1, i2, i3 in pts:
        a = sum(np.einsum("cba,a,b,c->", E, W[0][i1], W[1][i2], W[2][i3]) for E, W in parts)
        b = sum(w[k, q] * np.einsum("cba,a,b,c->", G[q], blocks[0][k, q, :, i1], blocks[1][k, q, :, i2],
                                    blocks[2][k, q, :, i3]) for k in range(M) for q in range(3))
        num += (a - b) ** 2
        den += b ** 2
    assert (num / den) ** 0.5 <= 20 * tol
    assert max(rho) < M


def test_needs_compression_first(D):
    P = D.demag_build_factors((8, 8, 8), (1.0, 1.0, 1.0), 11)
    with pytest.raises(D.DemagError):
        D.demag_compressed_ranks(P)
    with pytest.raises(D.DemagError):
        D.demag_compress_kernel(P, 0.0)


def test_implicit_core_gives_the_same_factors(D):
    n, ranks = (20, 24, 16), (2, 3, 2)
    P = D.demag_build_factors(n, (1.0, 1.0, 1.0), 21)
    D.demag_compress_kernel(P, 1e-5)
    core, flat = _inputs(n, ranks, 4)
    rho, _, oV = _run(D, P, n, ranks, core, flat)
    out_V = torch.empty(len(oV), device="cuda")
    D.demag_apply_tucker_compressed(P, 1, ranks, None, dev(flat), None, out_V)
    torch.cuda.synchronize()
    assert np.array_equal(host(out_V), oV)


@pytest.mark.parametrize("tol", [1e-2, 1e-4])
def test_recompression_bound(D, tol):
    # Alg. 2's approximate summation on the GPU: the recompressed Tucker tensor is within
    # tol of the summed potential, its factors are orthonormal, and its ranks are those of
    # the oracle's dense HOSVD of the same potential (up to the sketch)
    n, h, ranks = (24, 20, 16), (1.0, 1.0, 1.0), (3, 3, 3)
    P = D.demag_build_factors(n, h, 21)
    D.demag_compress_kernel(P, 1e-8)
    core, flat = _inputs(n, ranks, 5)
    rho, oc_, oV = _run(D, P, n, ranks, core, flat)
    parts = _parts(rho, n, ranks, oc_, oV)
    phi = _dense(parts)
    rk, C, Us, err = D.demag_recompress_tucker(P, ranks, dev(core.ravel()), dev(oV), tol)
    approx = oc.tucker_to_dense(host(C).astype(np.float64), [host(U).astype(np.float64).T for U in Us])
    assert rel_l2(approx, phi) <= tol * 1.01 + 1e-6
    assert err <= tol * (1 + 1e-9)
    for U in Us:
        Uh = host(U).astype(np.float64)
        assert np.allclose(Uh @ Uh.T, np.eye(Uh.shape[0]), atol=1e-5)
    _, _, ref_ranks = oc.recompress(parts, tol)
    assert all(a <= b + 2 for a, b in zip(rk, ref_ranks)), (rk, ref_ranks)
    assert sum(rk) < sum(3 * rho[p] * ranks[p] for p in range(3))


def test_recompression_1024(D):
    n, ranks, tol = (1024, 1024, 1024), (8, 8, 8), 1e-5
    P = D.demag_build_factors(n, (1.0 / 1024,) * 3, 61)
    D.demag_compress_kernel(P, 1e-6)
    core, flat = _inputs(n, ranks, 3)
    rho, oc_, oV = _run(D, P, n, ranks, core, flat)
    parts = _parts(rho, n, ranks, oc_, oV)
    rk, C, Us, err = D.demag_recompress_tucker(P, ranks, dev(core.ravel()), dev(oV), tol)
    assert err <= tol and max(rk) <= 64
    Ch = host(C).astype(np.float64)
    Uh = [host(U).astype(np.float64) for U in Us]
    pts = np.random.default_rng(1).integers(0, 1024, size=(24, 3))
    num = den = 0.0
    for i1, i2, i3 in pts:
        a = sum(np.einsum("cba,a,b,c->", E, W[0][i1], W[1][i2], W[2][i3]) for E, W in parts)
        b = np.einsum("cba,a,b,c->", Ch, Uh[0][:, i1], Uh[1][:, i2], Uh[2][:, i3])
        num += (a - b) ** 2
        den += a ** 2
    assert (num / den) ** 0.5 <= 10 * tol
