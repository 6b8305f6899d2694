"""Tensor-core (tcgen05) split-precision forms against the FP64 oracle.

Shapes cover partial row tiles, contraction lengths that are not multiples of
the 32-wide k-block, output widths below and above the 256-wide N tile, and
thin films."""
import numpy as np
import pytest

import synth
from oracle import full as ofull
from gpu_helpers import TOL, dev, host, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TC_SHAPES = [
    ((16, 16, 16), (1 / 16,) * 3, 41),
    ((20, 13, 7), (0.1, 0.2, 0.15), 41),
    ((1, 1, 1), (1.0, 1.0, 1.0), 5),
    ((130, 3, 5), (0.01, 0.01, 0.02), 21),
    ((33, 129, 2), (1.0, 1.0, 1.0), 21),
    ((64, 64, 4), (1 / 64, 1 / 64, 1 / 64), 41),
    ((300, 20, 10), (1 / 300,) * 3, 11),
    ((48, 40, 264), (1.0, 1.0, 1.0), 11),
]


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1212_3509_gb300 as D
    return D


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
@pytest.mark.parametrize("n,h,R", TC_SHAPES)
def test_split_full_vs_oracle(D, n, h, R, prec):
    m = synth.random_unit_m(n, 1212 + sum(n))
    P = D.demag_build_factors(n, h, R)
    phi = torch.empty(n[2], n[1], n[0], device="cuda")
    D.demag_apply_full(P, dev(m), phi, prec)
    torch.cuda.synchronize()
    D.demag_sync_status(P)
    err = rel_l2(host(phi), ofull.apply_full(m, n, h, R))
    print(f"{prec} {n}: rel L2 {err:.3e}")
    assert err <= TOL[prec], err


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
@pytest.mark.parametrize("n,h,R", [TC_SHAPES[1], TC_SHAPES[3], TC_SHAPES[6]])
def test_split_adjoint_vs_oracle(D, n, h, R, prec):
    rng = np.random.default_rng(11)
    y = rng.standard_normal((n[2], n[1], n[0])).astype(np.float32)
    P = D.demag_build_factors(n, h, R)
    g = torch.empty(3, n[2], n[1], n[0], device="cuda")
    D.demag_apply_adjoint(P, dev(y), g, prec)
    torch.cuda.synchronize()
    D.demag_sync_status(P)
    err = rel_l2(host(g), ofull.apply_adjoint(y, n, h, R))
    print(f"{prec} adjoint {n}: rel L2 {err:.3e}")
    assert err <= TOL[prec], err


def test_bf16x3_repeated_calls_are_identical(D):
    n, h, R = (40, 24, 16), (0.05,) * 3, 21
    m = dev(synth.random_unit_m(n, 99))
    P = D.demag_build_factors(n, h, R)
    a = torch.empty(n[2], n[1], n[0], device="cuda")
    b = torch.empty_like(a)
    D.demag_apply_full(P, m, a, "bf16x3")
    D.demag_apply_full(P, m, b, "bf16x3")
    torch.cuda.synchronize()
    assert torch.equal(a, b)
