"""GPU parity of the full format by per-fibre 1D Toeplitz FFTs (demag_apply_full_fibres) against
the FP64 oracle (oracle/full.py) and the other full-format paths, through the C ABI."""
import numpy as np
import pytest

import synth
from oracle import full as ofull
from gpu_helpers import dev, host, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1212_3509_gb300 as D
    return D


@pytest.mark.parametrize("n,R", [((9, 7, 5), 21), ((16, 12, 8), 41), ((5, 1, 3), 21), ((33, 17, 20), 41),
                                 ((1, 1, 1), 5), ((64, 2, 40), 21)])
def test_fibres_vs_oracle(D, n, R):
    h = (1.0 / max(n),) * 3
    m = synth.random_unit_m(n, 1300 + sum(n))
    P = D.demag_build_factors(n, h, R)
    phi = torch.empty(n[2], n[1], n[0], device="cuda")
    D.demag_apply_full_fibres(P, dev(m), phi)
    torch.cuda.synchronize()
    ref = ofull.apply_full(m, n, h, R)
    assert rel_l2(host(phi), ref) <= 1e-5


def test_fibres_vs_fft3d_and_repeatable(D):
    n, R = (128, 96, 80), 41
    h = (1.0 / 128,) * 3
    m = dev(synth.vortex_m(n, 1301))
    P = D.demag_build_factors(n, h, R)
    a = torch.empty(n[2], n[1], n[0], device="cuda")
    b = torch.empty_like(a)
    c = torch.empty_like(a)
    D.demag_apply_full_fibres(P, m, a)
    D.demag_apply_full_fibres(P, m, b)
    D.demag_apply_full_fft(P, m, c)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert rel_l2(host(a), host(c)) <= 2e-6


def test_fibres_256_sampled_lines(D):
    # the bench's 256^3 workload (R = 41, vortex state) at four output lines against the oracle
    from oracle import full as of
    n3, h, R = (256, 256, 256), (1 / 256,) * 3, 41
    m = synth.vortex_m(n3, 1213)
    P = D.demag_build_factors(n3, h, R)
    phi = torch.empty(256, 256, 256, device="cuda")
    D.demag_apply_full_fibres(P, dev(m), phi)
    torch.cuda.synchronize()
    lines = [(0, 0), (17, 200), (128, 129), (255, 31)]
    ref = of.apply_full_lines(m, n3, h, R, lines)
    got = host(phi)
    assert rel_l2(np.stack([got[i3, i2] for i3, i2 in lines]), ref) <= 1e-5
