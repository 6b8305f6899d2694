"""GPU parity on non-uniform tensor grids (demag_build_factors_nonuniform) against
the FP64 oracle (oracle/nonuniform.py), through the C ABI.

Graded and jittered cell widths, single-cell and short (<= 16, CUDA-core stage)
axes, every full-format precision, the adjoint on CUDA cores, mixing with a
uniform plan in one grouped launch, and the paths that need a uniform grid
refusing the plan."""
import numpy as np
import pytest

import synth
from oracle import full as ofull
from oracle import nonuniform as onu
from gpu_helpers import assert_close, TOL, dev, host, rel_l2
from test_oracle_nonuniform import _brute, _graded

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1212_3509_gb300 as D
    return D


def _grid(n, seed):
    rng = np.random.default_rng(seed)
    ratios = (1.04, 0.97, 1.1)
    return [_graded(n[p], 1e-6 * (1.0 + 0.3 * p), ratios[p] if n[p] > 1 else 1.0, rng) for p in range(3)]


SHAPES = [(20, 13, 7), (1, 5, 3), (130, 3, 5), (64, 64, 4), (33, 40, 17), (48, 48, 48)]


@pytest.mark.parametrize("n", SHAPES)
@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "bf16x3"])
def test_nonuniform_forward_vs_oracle(D, n, prec):
    edges = _grid(n, sum(n))
    m = synth.random_unit_m(n, 77 + sum(n))
    P = D.demag_build_factors_nonuniform(edges, 41)
    phi = torch.empty(n[2], n[1], n[0], device="cuda")
    D.demag_apply_full(P, dev(m), phi, prec)
    torch.cuda.synchronize()
    ref = onu.apply_full(m, edges, 41)
    assert_close(host(phi), ref, TOL[prec])


def test_nonuniform_brute_force(D):
    # exact collocation sum on a tiny graded grid (O(N^2) cell integrals)
    edges = [_graded(5, 1.0, 1.3), _graded(4, 0.8, 0.7), _graded(6, 1.2, 1.15)]
    n = [len(e) - 1 for e in edges]
    m = synth.random_unit_m(n, 3)
    P = D.demag_build_factors_nonuniform(edges, 41)
    phi = torch.empty(n[2], n[1], n[0], device="cuda")
    D.demag_apply_full(P, dev(m), phi, "fp64")
    torch.cuda.synchronize()
    assert rel_l2(host(phi), _brute(m.astype(np.float64), edges)) < 2e-5


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_uniform_edges_match_the_uniform_plan(D, prec):
    n, h = (24, 17, 9), (0.1, 0.2, 0.15)
    edges = [np.arange(n[p] + 1) * h[p] for p in range(3)]
    m = dev(synth.random_unit_m(n, 5))
    Pu = D.demag_build_factors(n, h, 41)
    Pn = D.demag_build_factors_nonuniform(edges, 41)
    a = torch.empty(n[2], n[1], n[0], device="cuda")
    b = torch.empty_like(a)
    D.demag_apply_full(Pu, m, a, prec)
    D.demag_apply_full(Pn, m, b, prec)
    torch.cuda.synchronize()
    if prec == "fp64":
        assert rel_l2(host(b), host(a)) <= 1e-12
    else:
        # the uniform plan folds its 24-cell axis into even / odd halves on the
        # tensor cores (Toeplitz factors are centro-symmetric); the non-uniform
        # plan's dense factors are not, so the two round differently: both
        # meet the split-form tolerance against the oracle and each other
        ref = ofull.apply_full(host(m), n, h, 41)
        assert_close(host(a), ref, TOL[prec], "uniform plan")
        assert_close(host(b), ref, TOL[prec], "uniform edges")
        assert rel_l2(host(b), host(a)) <= 2 * TOL[prec]


@pytest.mark.parametrize("n", [(20, 13, 7), (40, 9, 33)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_nonuniform_adjoint_vs_oracle_transpose(D, n, prec):
    edges = _grid(n, 11)
    y = np.random.default_rng(6).standard_normal((n[2], n[1], n[0])).astype(np.float32)
    P = D.demag_build_factors_nonuniform(edges, 21)
    g = torch.empty(3, n[2], n[1], n[0], device="cuda")
    D.demag_apply_adjoint(P, dev(y), g, prec)
    torch.cuda.synchronize()
    ref = onu.apply_full(y, edges, 21, transpose=True)
    assert_close(host(g), ref, TOL[prec])


def test_mixed_batch_with_a_uniform_plan(D):
    shapes = [(48, 40, 36), (64, 64, 4)]
    plans = [D.demag_build_factors_nonuniform(_grid(shapes[0], 1), 41), D.demag_build_factors(shapes[1], (1.0, 1.0, 0.5), 41)]
    ms = [dev(synth.random_unit_m(s, 9 + i)) for i, s in enumerate(shapes)]
    single = [torch.empty(s[2], s[1], s[0], device="cuda") for s in shapes]
    batched = [torch.empty_like(t) for t in single]
    for P, m, o in zip(plans, ms, single):
        D.demag_apply_full(P, m, o, "bf16x3")
    D.demag_apply_full_batched(plans, ms, batched, "bf16x3")
    torch.cuda.synchronize()
    # bit for bit where every stage runs on the tensor cores in both calls; the
    # 4-cell axis runs on CUDA cores in a single call, as a padded tensor-core
    # tile in the batch
    assert torch.equal(single[0], batched[0])
    assert_close(host(batched[1]), host(single[1]), TOL["bf16x3"])
    ref = onu.apply_full(host(ms[0]), _grid(shapes[0], 1), 41)
    assert_close(host(batched[0]), ref, TOL["bf16x3"])
    ref1 = ofull.apply_full(host(ms[1]), shapes[1], (1.0, 1.0, 0.5), 41)
    assert_close(host(batched[1]), ref1, TOL["bf16x3"])


def test_uniform_only_paths_refuse_the_plan(D):
    n = (16, 8, 4)
    P = D.demag_build_factors_nonuniform(_grid(n, 2), 11)
    m = torch.zeros(3, n[2], n[1], n[0], device="cuda")
    phi = torch.empty(n[2], n[1], n[0], device="cuda")
    calls = [
        lambda: D.demag_apply_adjoint(P, phi, m, "bf16x3"),
        lambda: D.demag_apply_full_fft(P, m, phi),
        lambda: D.demag_stray_field_exact(P, m, m.clone(), "fp32"),
        lambda: D.demag_stray_field(P, phi, m),
        lambda: D.demag_energy(P, m, torch.empty(1, dtype=torch.float64, device="cuda"), None, "fp32"),
    ]
    for call in calls:
        with pytest.raises(D.DemagError) as ei:
            call()
        assert ei.value.status == 5  # DEMAG_EUNSUPPORTED
    lam = torch.ones(3, 1, device="cuda")
    U = torch.ones(3 * (n[0] + n[1] + n[2]), device="cuda")
    with pytest.raises(D.DemagError) as ei:
        D.demag_apply_cp(P, 1, lam, U, torch.empty(P.M * 3, device="cuda"),
                         torch.empty(P.M * 3 * sum(n), device="cuda"))
    assert ei.value.status == 5
