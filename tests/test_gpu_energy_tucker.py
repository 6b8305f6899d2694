"""GPU parity of the Tucker-format demag energy (demag_energy_tucker, demag_energy_tucker_phi)
against the oracle (oracle/energy.py: energy_tucker), the exact-collocation cube energy and the
full-format GPU energy, through the C ABI."""
import numpy as np
import pytest

import synth
from oracle import energy as oe
from oracle import exact
from gpu_helpers import dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1212_3509_gb300 as D
    return D


def _energy(D, P, n, ranks, core, V):
    tot = sum(ranks[p] * n[p] for p in range(3))
    w = torch.empty(P.M * 3, device="cuda")
    oV = torch.empty(P.M * 3 * tot, device="cuda")
    cd, Vd = dev(np.ascontiguousarray(core, dtype=np.float32).ravel()), dev(np.ascontiguousarray(V, dtype=np.float32))
    D.demag_apply_tucker(P, ranks, Vd, w, oV)
    E = torch.empty((), dtype=torch.float64, device="cuda")
    D.demag_energy_tucker(P, ranks, cd, Vd, w, oV, E)
    torch.cuda.synchronize()
    return float(E.item()), (cd, Vd, w, oV)


@pytest.mark.parametrize("n,ranks,R", [((12, 10, 8), (2, 3, 2), 21), ((17, 9, 23), (1, 4, 3), 41),
                                       ((2, 5, 3), (1, 2, 2), 21),
                                       ((12, 10, 8), (40, 40, 40), 21)])  # Grams above 48 KB of shared memory
def test_energy_tucker_vs_oracle(D, n, ranks, R):
    h = (1.0 / max(n),) * 3
    core, V = synth.tucker_inputs(n, ranks, 77)
    P = D.demag_build_factors(n, h, R)
    E, _ = _energy(D, P, n, ranks, core, V)
    ref = oe.energy_tucker(core, V, n, ranks, h, R)
    assert abs(E - ref) <= 1e-5 * abs(ref) + 1e-12, (E, ref)


def test_energy_tucker_vs_full_format_gpu_energy(D):
    n, ranks, R = (64, 48, 40), (3, 3, 3), 41
    h = (1.0 / 64,) * 3
    core, V = synth.tucker_inputs(n, ranks, 78)
    P = D.demag_build_factors(n, h, R)
    E, _ = _energy(D, P, n, ranks, core, V)
    m = torch.from_numpy(oe.tucker_magnetization(core, V, n, ranks).astype(np.float32)).cuda().contiguous()
    Ef = torch.empty((), dtype=torch.float64, device="cuda")
    D.demag_energy(P, m, Ef, None, "fp32")
    torch.cuda.synchronize()
    assert abs(E - Ef.item()) <= 2e-5 * abs(Ef.item())


@pytest.mark.parametrize("n", [32, 64])
def test_uniform_cube_energy_is_the_exact_collocation_energy(D, n):
    # the case of the energy study after Alg. 2: rank-1 Tucker m = z, R = 129
    h = (1.0 / n,) * 3
    core = np.zeros((3, 1, 1, 1), dtype=np.float32)
    core[2] = 1.0
    V = np.ones(3 * 3 * n, dtype=np.float32)
    P = D.demag_build_factors((n, n, n), h, 129)
    E, _ = _energy(D, P, (n, n, n), (1, 1, 1), core, V)
    m = synth.uniform_m((n, n, n), 2).astype(np.float64)
    ref = oe.energy(m, exact.uniform_box_potential((n, n, n), h, 2), h)
    assert abs(E - ref) <= 1e-5 * ref, (E, ref)


def test_energy_of_the_recompressed_potential(D):
    # Alg. 2 end to end: compressed kernels, application, approximate summation, energy of the
    # single Tucker potential; it agrees with the energy of the unsummed output within the tolerances
    n, ranks, R = (24, 20, 16), (2, 2, 2), 21
    h = (1.0 / 24,) * 3
    core, V = synth.tucker_inputs(n, ranks, 79)
    P = D.demag_build_factors(n, h, R)
    E0, _ = _energy(D, P, n, ranks, core, V)
    D.demag_compress_kernel(P, 1e-8)
    rho = D.demag_compressed_ranks(P)
    cd, Vd = dev(core.ravel()), dev(V)
    out_V = torch.empty(sum(3 * rho[p] * ranks[p] * n[p] for p in range(3)), device="cuda")
    D.demag_apply_tucker_compressed(P, 1, ranks, cd, Vd, None, out_V)
    rk, C, Us, err = D.demag_recompress_tucker(P, ranks, cd, out_V, 1e-7)
    E = torch.empty((), dtype=torch.float64, device="cuda")
    D.demag_energy_tucker_phi(P, ranks, cd, Vd, rk, C.contiguous().view(-1),
                              torch.cat([u.reshape(-1) for u in Us]), E)
    torch.cuda.synchronize()
    assert abs(E.item() - E0) <= 2e-5 * abs(E0), (E.item(), E0)
    ref = oe.energy_tucker(core, V, n, ranks, h, R)
    assert abs(E.item() - ref) <= 2e-5 * abs(ref)


def test_rejects_bad_ranks(D):
    n = (8, 8, 8)
    P = D.demag_build_factors(n, (1 / 8,) * 3, 21)
    core, V = synth.tucker_inputs(n, (1, 1, 1), 1)
    E = torch.empty((), dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError, match="ranks"):
        D.demag_energy_tucker_phi(P, (1, 1, 1), dev(core.ravel()), dev(V), (65, 1, 1),
                                  torch.zeros(65, device="cuda"), torch.zeros(65 * 8 + 16, device="cuda"), E)


def _apply_tt(D, P, n, ranks, G):
    M, (r1, r2) = P.M, ranks
    w = torch.empty(M * 3, device="cuda")
    o = [torch.empty(M * 3 * s, device="cuda") for s in (r1 * n[0], r1 * r2 * n[1], r2 * n[2])]
    D.demag_apply_tt(P, ranks, *G, w, *o)
    return w, o


@pytest.mark.parametrize("n,ranks,R", [((10, 8, 6), (2, 3), 21), ((3, 17, 2), (1, 2), 41),
                                       ((16, 12, 10), (8, 8), 21)])
def test_energy_tt_vs_oracle(D, n, ranks, R):
    h = (1.0 / max(n),) * 3
    G1, G2, G3 = synth.tt_inputs(n, ranks, 81)
    P = D.demag_build_factors(n, h, R)
    G = [dev(x) for x in (G1, G2, G3)]
    w, o = _apply_tt(D, P, n, ranks, G)
    E = torch.empty((), dtype=torch.float64, device="cuda")
    D.demag_energy_tt(P, ranks, *G, w, *o, E)
    torch.cuda.synchronize()
    ref = oe.energy_tt(G1, G2, G3, n, ranks, h, R)
    assert abs(E.item() - ref) <= 1e-5 * abs(ref), (E.item(), ref)


def test_energy_tt_of_a_converted_tucker_equals_the_tucker_energy(D):
    n, ranks, R = (48, 40, 32), (2, 3, 2), 41
    h = (1.0 / 48,) * 3
    core, V = synth.tucker_inputs(n, ranks, 82)
    P = D.demag_build_factors(n, h, R)
    Et, _ = _energy(D, P, n, ranks, core, V)
    t = (ranks[0], ranks[2])
    G = (torch.empty(3 * t[0] * n[0], device="cuda"), torch.empty(3 * t[0] * t[1] * n[1], device="cuda"),
         torch.empty(3 * t[1] * n[2], device="cuda"))
    D.demag_tucker_to_tt(P, ranks, dev(core.ravel()), dev(V), *G)
    w, o = _apply_tt(D, P, n, t, G)
    E = torch.empty((), dtype=torch.float64, device="cuda")
    D.demag_energy_tt(P, t, *G, w, *o, E)
    torch.cuda.synchronize()
    assert abs(E.item() - Et) <= 2e-5 * abs(Et), (E.item(), Et)


def test_energy_tt_rejects_large_ranks(D):
    n = (8, 8, 8)
    P = D.demag_build_factors(n, (1 / 8,) * 3, 21)
    r = (12, 12)
    G = [torch.zeros(3 * s, device="cuda") for s in (12 * 8, 144 * 8, 12 * 8)]
    o = [torch.zeros(3 * P.M * s, device="cuda") for s in (12 * 8, 144 * 8, 12 * 8)]
    E = torch.empty((), dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError, match="ranks"):
        D.demag_energy_tt(P, r, *G, torch.zeros(3 * P.M, device="cuda"), *o, E)


def test_energy_1024_tucker_and_tt_routes_agree(D):
    # the 1024^3 workload (ranks 8, R = 61): the Tucker energy and the TT energy of the same
    # magnetization converted to a train (independent kernels) agree
    n, ranks, R = (1024, 1024, 1024), (8, 8, 8), 61
    core, V = synth.tucker_inputs(n, ranks, 1500)
    P = D.demag_build_factors(n, (1.0 / 1024,) * 3, R)
    Et, _ = _energy(D, P, n, ranks, core, V)
    t = (8, 8)
    G = (torch.empty(3 * 8 * 1024, device="cuda"), torch.empty(3 * 64 * 1024, device="cuda"),
         torch.empty(3 * 8 * 1024, device="cuda"))
    D.demag_tucker_to_tt(P, ranks, dev(core.ravel()), dev(V), *G)
    w, o = _apply_tt(D, P, n, t, G)
    E = torch.empty((), dtype=torch.float64, device="cuda")
    D.demag_energy_tt(P, t, *G, w, *o, E)
    torch.cuda.synchronize()
    assert abs(E.item() - Et) <= 2e-5 * abs(Et), (E.item(), Et)


@pytest.mark.parametrize("n,ranks,R", [((12, 10, 8), (2, 3, 2), 21), ((17, 9, 23), (1, 4, 3), 41),
                                       ((12, 10, 8), (40, 40, 40), 21)])
def test_energy_tucker_fp64_vs_oracle(D, n, ranks, R):
    """The FP64 Tucker application and energy equal the oracle's dense FP64 route to
    rounding (sums of ~10^3 FP64 terms with some cancellation: 1e-10; the FP32 route is
    held to 1e-5)."""
    h = (1.0 / max(n),) * 3
    core, V = synth.tucker_inputs(n, ranks, 79)
    P = D.demag_build_factors(n, h, R)
    E = torch.empty((), dtype=torch.float64, device="cuda")
    D.demag_energy_tucker_fp64(P, ranks, torch.from_numpy(np.ascontiguousarray(core, dtype=np.float64).ravel()).cuda(),
                               torch.from_numpy(np.ascontiguousarray(V, dtype=np.float64)).cuda(), E)
    torch.cuda.synchronize()
    ref = oe.energy_tucker(core, V, n, ranks, h, R)
    assert abs(E.item() - ref) <= 1e-10 * abs(ref), (E.item(), ref)


@pytest.mark.parametrize("n,R", [(512, 257), (2048, 257)])
def test_uniform_cube_energy_fp64_vs_oracle_1d_sums(D, n, R):
    """The energy study's cube (m = e3, rank 1) on fine grids: the FP64 route equals the
    oracle's one-dimensional FP64 sums to rounding, below the FP32 route's floor."""
    P = D.demag_build_factors((n, n, n), (1.0 / n,) * 3, R)
    core = torch.zeros(3, dtype=torch.float64, device="cuda")
    core[2] = 1.0
    V = torch.ones(9 * n, dtype=torch.float64, device="cuda")
    E = torch.empty((), dtype=torch.float64, device="cuda")
    D.demag_energy_tucker_fp64(P, (1, 1, 1), core, V, E)
    torch.cuda.synchronize()
    ref = oe.uniform_cube_energy(n, R)
    assert abs(E.item() - ref) <= 1e-11 * ref, (E.item(), ref)
    assert abs(E.item() - 1.0 / 6.0) * 6.0 < 1e-5


def test_energy_tucker_fp64_rejects_what_it_cannot_do(D):
    """A graded (non-uniform) grid has no Toeplitz generators and ranks past 64 do not fit the
    Gram tiles: both are errors before any launch."""
    edges = [np.concatenate([[0.0], np.cumsum(1.05 ** np.arange(k))]) / 16 for k in (12, 10, 8)]
    Pn = D.demag_build_factors_nonuniform(edges, 21)
    core = torch.zeros(3, dtype=torch.float64, device="cuda")
    V = torch.ones(3 * 30, dtype=torch.float64, device="cuda")
    E = torch.empty((), dtype=torch.float64, device="cuda")
    with pytest.raises(D.DemagError):
        D.demag_energy_tucker_fp64(Pn, (1, 1, 1), core, V, E)
    P = D.demag_build_factors((12, 10, 8), (1 / 12,) * 3, 21)
    with pytest.raises(D.DemagError):
        D.demag_energy_tucker_fp64(P, (65, 1, 1), torch.zeros(3 * 65, dtype=torch.float64, device="cuda"),
                                   torch.ones(3 * (65 * 12 + 10 + 8), dtype=torch.float64, device="cuda"), E)
