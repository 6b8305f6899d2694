"""GPU parity against the FP64 oracle on the same seeded inputs (through the C ABI).

Small and ragged shapes that span several tiles and end in partial tiles,
degenerate grids (n = 1, 2, thin films) and every format of the boundary."""
import numpy as np
import pytest

import synth
from oracle import energy as oen
from oracle import exact as oex
from oracle import full as ofull
from oracle import generators as ogen
from oracle import quadrature as oq
from oracle import structured as ost
from gpu_helpers import assert_close, TOL, dev, host, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1212_3509_gb300 as D
    return D


SHAPES = [
    ((16, 16, 16), (1 / 16,) * 3, 41),
    ((20, 13, 7), (0.1, 0.2, 0.15), 41),
    ((1, 1, 1), (1.0, 1.0, 1.0), 5),
    ((2, 3, 1), (0.5, 0.5, 1.0), 11),
    ((130, 3, 5), (0.01, 0.01, 0.02), 21),
    ((33, 129, 2), (1.0, 1.0, 1.0), 21),
    ((64, 64, 4), (1 / 64, 1 / 64, 1 / 64), 41),
]


def _plan(D, n, h, R):
    return D.demag_build_factors(n, h, R)


@pytest.mark.parametrize("n,h,R", SHAPES[:2] + SHAPES[4:5])
def test_nodes_and_generators_fp64(D, n, h, R):
    P = _plan(D, n, h, R)
    M = P.M
    nodes = torch.empty(3 * M, dtype=torch.float64, device="cuda")
    D.demag_copy_nodes(P, nodes)
    nodes = host(nodes).reshape(3, M)
    _, t, tau, om = oq.sinc_nodes(M, 2.15)
    assert np.allclose(nodes[0], t, rtol=1e-14)
    assert np.allclose(nodes[1], tau, rtol=1e-13)
    assert np.allclose(nodes[2], om, rtol=1e-13)
    g = torch.empty(D.demag_generators_size(P), dtype=torch.float64, device="cuda")
    D.demag_copy_generators(P, g)
    nmax = max(n)
    g = host(g).reshape(M, 2, 3, 2 * nmax - 1)
    s, hh = ogen.scaled_spacing(n, h)
    for k in range(M):
        for p in range(3):
            E = ogen.gen_E(tau[k], hh[p], n[p])
            F = ogen.gen_F(tau[k], hh[p], n[p])
            L = 2 * n[p] - 1
            for typ, ref in ((0, E), (1, F)):
                got = g[k, typ, p, :L]
                scale = np.abs(ref).max()
                assert np.all(np.abs(got - ref) <= 1e-13 * np.abs(ref) + 1e-15 * scale), (k, typ, p)
                assert np.all(g[k, typ, p, L:] == 0)


def test_symbols_match_numpy_fft_of_oracle_generators(D):
    n, h, R = (20, 13, 7), (0.1, 0.2, 0.15), 21
    P = _plan(D, n, h, R)
    M = P.M
    sym = torch.empty(D.demag_symbols_size(P), dtype=torch.float32, device="cuda")
    D.demag_copy_symbols(P, sym)
    Lmax = max(1 << int(np.ceil(np.log2(max(2 * v - 1, 2)))) for v in n)
    sym = host(sym).reshape(M, 2, 3, Lmax // 2 + 1)
    _, _, tau, _ = oq.sinc_nodes(M, 2.15)
    s, hh = ogen.scaled_spacing(n, h)
    for k in (0, M // 2, M - 1):
        for p in range(3):
            L = max(2, 1 << int(np.ceil(np.log2(2 * n[p] - 1))))
            for typ, fn in ((0, ogen.gen_E), (1, ogen.gen_F)):
                t = fn(tau[k], hh[p], n[p])
                c = np.zeros(L)
                c[:n[p]] = t[n[p] - 1:]
                for d in range(1, n[p]):
                    c[L - d] = t[n[p] - 1 - d]
                ref = np.fft.rfft(c) / L
                ref = ref.real if typ == 0 else ref.imag
                got = sym[k, typ, p, :L // 2 + 1]
                assert np.max(np.abs(got - ref)) <= 2e-7 * np.max(np.abs(ref)) + 1e-30


@pytest.mark.parametrize("n,h,R", SHAPES)
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_full_format_vs_oracle(D, n, h, R, prec):
    m = synth.random_unit_m(n, 1212 + sum(n))
    P = _plan(D, n, h, R)
    phi = torch.empty(n[2], n[1], n[0], dtype=torch.float32, device="cuda")
    D.demag_apply_full(P, dev(m), phi, prec)
    torch.cuda.synchronize()
    ref = ofull.apply_full(m, n, h, R)
    err = rel_l2(host(phi), ref)
    assert_close(host(phi), ref, TOL[prec])


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_c1_uniform_cube_against_closed_form(D, prec):
    # 16^3, R = 41: parity with the oracle, and the GPU result is within the
    # quadrature error of the exact collocation (closed form) potential.
    n, h = (16, 16, 16), (1 / 16,) * 3
    m = synth.uniform_m(n, 2)
    P = _plan(D, n, h, 41)
    phi = torch.empty(16, 16, 16, device="cuda")
    D.demag_apply_full(P, dev(m), phi, prec)
    torch.cuda.synchronize()
    got = host(phi)
    assert_close(got, ofull.apply_full(m, n, h, 41), TOL[prec])
    exact = oex.uniform_box_potential(n, h, 2)
    assert np.max(np.abs(got - exact)) < 2e-6 * np.max(np.abs(exact))


def test_c1_brute_force(D):
    n, h = (16, 16, 16), (1 / 16,) * 3
    m = synth.random_unit_m(n, 1212)
    P = _plan(D, n, h, 41)
    phi = torch.empty(16, 16, 16, device="cuda")
    D.demag_apply_full(P, dev(m), phi, "fp64")
    torch.cuda.synchronize()
    ref = oex.collocation_exact(m, n, h)
    assert rel_l2(host(phi), ref) < 1e-5


@pytest.mark.parametrize("n,h,R", SHAPES[:2] + SHAPES[4:6])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_adjoint_vs_oracle(D, n, h, R, prec):
    rng = np.random.default_rng(11)
    y = rng.standard_normal((n[2], n[1], n[0])).astype(np.float32)
    P = _plan(D, n, h, R)
    g = torch.empty(3, n[2], n[1], n[0], device="cuda")
    D.demag_apply_adjoint(P, dev(y), g, prec)
    torch.cuda.synchronize()
    ref = ofull.apply_adjoint(y, n, h, R)
    assert_close(host(g), ref, TOL[prec])


@pytest.mark.parametrize("n", [(16, 16, 16), (37, 50, 9), (1, 4, 2), (128, 128, 128)])
def test_cp_vs_oracle(D, n):
    h = (1.0 / max(n),) * 3
    r, R = 3, 21
    lam, U = synth.cp_inputs(n, r, 1215)
    P = _plan(D, n, h, R)
    M, ns = P.M, sum(n)
    w = torch.empty(M * 3 * r, device="cuda")
    oU = torch.empty(M * 3 * r * ns, device="cuda")
    D.demag_apply_cp(P, r, dev(lam), dev(U.ravel()), w, oU)
    torch.cuda.synchronize()
    rw, rU = ost.apply_cp(lam, U, n, h, R)
    assert rel_l2(host(w), rw.ravel()) < 1e-6
    ref = np.concatenate([rU[p].ravel() for p in range(3)])
    assert_close(host(oU), ref, TOL["fp32"])


def test_cp_matches_full_format_at_128(D):
    # the C3 cross-check: CP apply vs the full format on the formed tensor (n = 128)
    n, h, R, r = (128, 128, 128), (1 / 128,) * 3, 61, 4
    lam, U = synth.cp_inputs(n, r, 1215)
    blocks = ost._split_blocks(U, n, (r, r, r))
    m = np.stack([ost.cp_to_full(lam[q], blocks[q]) for q in range(3)]).astype(np.float32)
    P = _plan(D, n, h, R)
    M = P.M
    w = torch.empty(M * 3 * r, device="cuda")
    oU = torch.empty(M * 3 * r * 384, device="cuda")
    D.demag_apply_cp(P, r, dev(lam), dev(U.ravel()), w, oU)
    phi = torch.empty(128, 128, 128, device="cuda")
    D.demag_apply_full(P, dev(m), phi, "fp32")
    torch.cuda.synchronize()
    oUh = host(oU)
    f = [oUh[p * M * 3 * r * 128:(p + 1) * M * 3 * r * 128].reshape(M * 3 * r, 128) for p in range(3)]
    phi_cp = ost.cp_to_full(host(w), f)
    assert rel_l2(phi_cp, host(phi)) < 2e-5


@pytest.mark.parametrize("n,ranks", [((16, 16, 16), (3, 2, 4)), ((37, 50, 9), (2, 5, 1))])
def test_tucker_vs_oracle(D, n, ranks):
    h = (1.0 / max(n),) * 3
    R = 21
    core, V = synth.tucker_inputs(n, ranks, 1216)
    P = _plan(D, n, h, R)
    M = P.M
    tot = sum(ranks[p] * n[p] for p in range(3))
    w = torch.empty(M * 3, device="cuda")
    oV = torch.empty(M * 3 * tot, device="cuda")
    D.demag_apply_tucker(P, ranks, dev(V), w, oV)
    torch.cuda.synchronize()
    rw, rV = ost.apply_tucker(core, V, n, ranks, h, R)
    assert rel_l2(host(w), rw.ravel()) < 1e-6
    assert_close(host(oV), np.concatenate([rV[p].ravel() for p in range(3)]), TOL["fp32"])


@pytest.mark.parametrize("n,ranks", [((16, 16, 16), (3, 2)), ((37, 50, 9), (4, 1))])
def test_tt_vs_oracle(D, n, ranks):
    h = (1.0 / max(n),) * 3
    R = 21
    G1, G2, G3 = synth.tt_inputs(n, ranks, 1217)
    P = _plan(D, n, h, R)
    M = P.M
    r1, r2 = ranks
    w = torch.empty(M * 3, device="cuda")
    o1 = torch.empty(M * 3 * r1 * n[0], device="cuda")
    o2 = torch.empty(M * 3 * r1 * r2 * n[1], device="cuda")
    o3 = torch.empty(M * 3 * r2 * n[2], device="cuda")
    D.demag_apply_tt(P, ranks, dev(G1), dev(G2), dev(G3), w, o1, o2, o3)
    torch.cuda.synchronize()
    rw, r1o, r2o, r3o = ost.apply_tt(G1, G2, G3, n, ranks, h, R)
    assert rel_l2(host(w), rw.ravel()) < 1e-6
    for got, ref in ((o1, r1o), (o2, r2o), (o3, r3o)):
        assert_close(host(got), ref.ravel(), TOL["fp32"])


def test_stray_field_energy_gradient(D):
    n, h, R = (16, 16, 16), (1 / 16,) * 3, 41
    m = synth.random_unit_m(n, 1217)
    P = _plan(D, n, h, R)
    md = dev(m)
    phi = torch.empty(16, 16, 16, device="cuda")
    D.demag_apply_full(P, md, phi, "fp32")
    hd = torch.empty(3, 16, 16, 16, device="cuda")
    D.demag_stray_field(P, phi, hd)
    E = torch.empty((), dtype=torch.float64, device="cuda")
    grad = torch.empty_like(md)
    D.demag_energy(P, md, E, grad, "fp32")
    torch.cuda.synchronize()
    phi_ref = ofull.apply_full(m, n, h, R)
    assert rel_l2(host(hd), oen.stray_field(phi_ref, h)) < 1e-5
    assert float(E) == pytest.approx(oen.energy(m, phi_ref, h), rel=1e-5)
    assert rel_l2(host(grad), oen.energy_gradient(m, n, h, R)) < 1e-5


def test_uniform_cube_energy_one_sixth(D):
    n, h = (32, 32, 32), (1 / 32,) * 3
    P = _plan(D, n, h, 41)
    E = torch.empty((), dtype=torch.float64, device="cuda")
    D.demag_energy(P, dev(synth.uniform_m(n, 2)), E, None, "fp32")
    torch.cuda.synchronize()
    assert float(E) == pytest.approx(1 / 6, abs=2e-4)


def test_autograd_energy(D):
    n, h, R = (8, 8, 8), (1 / 8,) * 3, 21
    m = synth.random_unit_m(n, 1218)
    P = _plan(D, n, h, R)
    mt = dev(m).requires_grad_(True)
    E = D.demag_energy_fn(mt, P, "fp32")
    E.backward()
    assert float(E) == pytest.approx(oen.energy_from_m(m, n, h, R), rel=1e-5)
    assert rel_l2(host(mt.grad), oen.energy_gradient(m, n, h, R)) < 1e-5


def test_invalid_arguments_raise(D):
    P = _plan(D, (4, 4, 4), (1, 1, 1), 11)
    with pytest.raises(ValueError):
        D.demag_apply_full(P, torch.empty(5, device="cuda"), torch.empty(64, device="cuda"))
    # raw (non-null) pointers skip the binding's checks: the C side must reject r = 0
    # before touching them
    with pytest.raises(D.DemagError):
        D.demag_apply_cp_batched(P, 1, 0, 16, 16, 16, 16)
    D.demag_sync_status(P)
