"""GPU parity of the 3D FFT convolution (demag_apply_full_fft, Eq. fft_pot)
against the FP64 oracle on the same seeded inputs, through the C ABI.

Ragged and degenerate grids (n_p = 1, odd, non-power-of-two, thin films)
exercise every FFT length from 2 to 1024 and partial fibre tiles in all five
passes; 256^3 is checked on sampled output lines."""
import numpy as np
import pytest

import synth
from oracle import exact as oex
from oracle import fft3d as of3
from oracle import full as ofull
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
    ((5, 40, 67), (2e-9, 3e-9, 1e-9), 41),
    ((9, 17, 257), (1.0, 1.0, 1.0), 21),
]


def _apply(D, P, m, n):
    phi = torch.empty(n[2], n[1], n[0], dtype=torch.float32, device="cuda")
    D.demag_apply_full_fft(P, dev(m), phi)
    torch.cuda.synchronize()
    return host(phi)


@pytest.mark.parametrize("n,h,R", SHAPES)
def test_fft3d_vs_oracle(D, n, h, R):
    m = synth.random_unit_m(n, 1212 + sum(n))
    P = D.demag_build_factors(n, h, R)
    got = _apply(D, P, m, n)
    ref = ofull.apply_full(m, n, h, R)
    assert_close(got, ref, TOL["fp32"])
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref))


def test_fft3d_equals_fft_oracle_and_mode_products(D):
    # the oracle's own FFT form and the Kronecker form agree (pinned on CPU);
    # the GPU matches both, and the tensor-core form within their tolerances
    n, h, R = (48, 40, 36), (1.0, 1.0, 1.0), 41
    m = synth.vortex_m(n, 7)
    P = D.demag_build_factors(n, h, R)
    got = _apply(D, P, m, n)
    ref = of3.apply_fft3d(m, n, h, R)
    assert rel_l2(got, ref) <= 1e-5
    tc = torch.empty(n[2], n[1], n[0], device="cuda")
    D.demag_apply_full(P, dev(m), tc, "tf32x3")
    torch.cuda.synchronize()
    assert rel_l2(got, host(tc)) <= 2e-5


def test_fft3d_uniform_cube_closed_form(D):
    n, h = (16, 16, 16), (1 / 16,) * 3
    m = synth.uniform_m(n, 2)
    P = D.demag_build_factors(n, h, 41)
    got = _apply(D, P, m, n)
    exact = oex.uniform_box_potential(n, h, 2)
    assert np.max(np.abs(got - exact)) < 3e-6 * np.max(np.abs(exact))


def test_fft3d_longest_axis_512(D):
    # L = 1024 on the fastest axis (the largest FFT this path takes)
    n, h, R = (512, 6, 5), (1.0, 1.0, 1.0), 21
    m = synth.random_unit_m(n, 5)
    P = D.demag_build_factors(n, h, R)
    got = _apply(D, P, m, n)
    ref = ofull.apply_full(m, n, h, R)
    assert_close(got, ref, TOL["fp32"])


@pytest.mark.parametrize("n", [(6, 512, 5), (5, 6, 512)])
def test_fft3d_longest_slow_axes(D, n):
    h, R = (1.0, 1.0, 1.0), 11
    m = synth.random_unit_m(n, 6)
    P = D.demag_build_factors(n, h, R)
    got = _apply(D, P, m, n)
    ref = ofull.apply_full(m, n, h, R)
    assert_close(got, ref, TOL["fp32"])


def test_fft3d_256_sampled_lines(D):
    # the measured workload: 256^3, R = 41, vortex state; output lines sampled
    n, h, R = (256, 256, 256), (1 / 256,) * 3, 41
    m = synth.vortex_m(n, 1212)
    P = D.demag_build_factors(n, h, R)
    got = _apply(D, P, m, n)
    lines = [(0, 0), (255, 255), (128, 3), (17, 200)]
    ref = ofull.apply_full_lines(m, n, h, R, lines)
    for (i3, i2), r in zip(lines, ref):
        assert_close(got[i3, i2], r, TOL["fp32"])


def test_fft3d_repeatable_and_graph_capturable(D):
    n, h, R = (40, 33, 24), (1.0, 1.0, 1.0), 21
    m = dev(synth.random_unit_m(n, 9))
    P = D.demag_build_factors(n, h, R)
    a = torch.empty(n[2], n[1], n[0], device="cuda")
    b = torch.empty_like(a)
    D.demag_apply_full_fft(P, m, a)   # first call builds the kernel and workspace
    D.demag_apply_full_fft(P, m, b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    c = torch.zeros_like(a)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            D.demag_apply_full_fft(P, m, c, stream=s)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(a, c)


@pytest.mark.parametrize("n", [(1024, 6, 5), (6, 1024, 5), (5, 6, 1024)])
def test_fft3d_length_2048_axes(D, n):
    # n_p = 1024: FFT length 2048, two warps per fibre
    h, R = (1.0, 1.0, 1.0), 11
    m = synth.random_unit_m(n, 8)
    P = D.demag_build_factors(n, h, R)
    got = _apply(D, P, m, n)
    assert_close(got, ofull.apply_full(m, n, h, R), TOL["fp32"])
    from oracle import field as ofield
    hd = torch.empty(3, n[2], n[1], n[0], device="cuda")
    D.demag_stray_field_fft(P, dev(m), hd)
    torch.cuda.synchronize()
    assert rel_l2(host(hd), ofield.apply_field(m, n, h, R)) <= 1e-5


def test_fft3d_1024_cubed_uniform_box(D):
    # 1024^3 (1.07 G cells, ~110 GB of spectra and kernel) on one GPU: the uniformly
    # magnetized cube against its closed-form potential at sampled cells.  R = 129: the
    # largest node must exceed ~2/h for the near field (with R = 81 the boundary cells are
    # off by 2e-4; on 64^3 the same ratio of nodes to 1/h gives 1.6e-5 and 2.7e-7 at R = 33, 41)
    free, _ = torch.cuda.mem_get_info()
    if free < 160e9:
        pytest.skip("needs ~110 GB of free device memory")
    import gc
    n, h = (1024, 1024, 1024), (1 / 1024,) * 3
    P = D.demag_build_factors(n, h, 129)
    m = torch.zeros(3, 1024, 1024, 1024, device="cuda")
    m[2] = 1.0
    phi = torch.empty(1024, 1024, 1024, device="cuda")
    D.demag_apply_full_fft(P, m, phi)
    torch.cuda.synchronize()
    pts = [(0, 0, 0), (1023, 511, 7), (512, 512, 512), (100, 900, 1023), (3, 1020, 600)]
    got = np.array([float(phi[i3, i2, i1]) for i1, i2, i3 in pts])
    ref = []
    for i1, i2, i3 in pts:  # (1/4pi)(far face - near face) of the charged faces normal to z
        x = [(i + 0.5) / 1024 for i in (i1, i2, i3)]
        top = oex.rect_integral(x[0] - 1, x[0], x[1] - 1, x[1], x[2] - 1)
        bottom = oex.rect_integral(x[0] - 1, x[0], x[1] - 1, x[1], x[2])
        ref.append(float((top - bottom) / (4 * np.pi)))
    ref = np.array(ref)
    assert np.max(np.abs(got - ref)) < 1e-4 * np.max(np.abs(ref)), (got, ref)
    del P, m, phi
    gc.collect()
    torch.cuda.empty_cache()


def test_fft3d_too_long_axis_is_rejected(D):
    P = D.demag_build_factors((1025, 2, 2), (1.0, 1.0, 1.0), 5)
    m = torch.zeros(3, 2, 2, 1025, device="cuda")
    phi = torch.empty(2, 2, 1025, device="cuda")
    with pytest.raises(D.DemagError) as ei:
        D.demag_apply_full_fft(P, m, phi)
    assert ei.value.status == 5  # DEMAG_EUNSUPPORTED


FIELD_SHAPES = [
    ((16, 16, 16), (1 / 16,) * 3, 41),
    ((20, 13, 7), (0.1, 0.2, 0.15), 41),
    ((1, 1, 1), (1.0, 1.0, 1.0), 5),
    ((2, 3, 1), (0.5, 0.5, 1.0), 11),
    ((130, 3, 5), (0.01, 0.01, 0.02), 21),
    ((33, 129, 2), (1.0, 1.0, 1.0), 21),
    ((5, 40, 67), (2e-9, 3e-9, 1e-9), 41),
]


@pytest.mark.parametrize("n,h,R", FIELD_SHAPES)
def test_field_fft_vs_oracle(D, n, h, R):
    from oracle import field as ofield
    m = synth.random_unit_m(n, 33 + sum(n))
    P = D.demag_build_factors(n, h, R)
    hd = torch.empty(3, n[2], n[1], n[0], device="cuda")
    D.demag_stray_field_fft(P, dev(m), hd)
    torch.cuda.synchronize()
    ref = ofield.apply_field(m, n, h, R)
    assert rel_l2(host(hd), ref) <= 1e-5, rel_l2(host(hd), ref)


def test_field_fft_cube_demag_factor(D):
    n, h = (24, 24, 24), (1 / 24,) * 3
    P = D.demag_build_factors(n, h, 41)
    for q in range(3):
        m = synth.uniform_m(n, q)
        hd = torch.empty(3, 24, 24, 24, device="cuda")
        D.demag_stray_field_fft(P, dev(m), hd)
        torch.cuda.synchronize()
        mean = host(hd).reshape(3, -1).mean(axis=1)
        assert abs(mean[q] + 1.0 / 3.0) < 5e-3
        assert np.all(np.abs(np.delete(mean, q)) < 1e-5)


def test_field_fft_matches_the_tensor_core_field_at_128(D):
    n, h = (128, 128, 128), (1 / 128,) * 3
    m = dev(synth.vortex_m(n, 4))
    P = D.demag_build_factors(n, h, 41)
    a = torch.empty(3, 128, 128, 128, device="cuda")
    b = torch.empty_like(a)
    D.demag_stray_field_fft(P, m, a)
    D.demag_stray_field_exact(P, m, b, "tf32x3")
    torch.cuda.synchronize()
    assert rel_l2(host(a), host(b)) <= 2e-5
    # the potential path still works on the same plan after the field grew the workspace
    phi = torch.empty(128, 128, 128, device="cuda")
    D.demag_apply_full_fft(P, m, phi)
    tc = torch.empty_like(phi)
    D.demag_apply_full(P, m, tc, "tf32x3")
    torch.cuda.synchronize()
    assert rel_l2(host(phi), host(tc)) <= 2e-5


def test_energy_from_the_fft_field(D):
    from oracle import field as ofield
    n, h, R = (20, 13, 7), (0.1, 0.2, 0.15), 41
    m = synth.random_unit_m(n, 71)
    P = D.demag_build_factors(n, h, R)
    e = torch.empty(1, dtype=torch.float64, device="cuda")
    g = torch.empty(3, n[2], n[1], n[0], device="cuda")
    D.demag_energy_field_fft(P, dev(m), e, g)
    torch.cuda.synchronize()
    hd = ofield.apply_field(m, n, h, R)
    V = h[0] * h[1] * h[2]
    ref = -0.5 * V * np.sum(m.astype(np.float64) * hd)
    assert abs(float(host(e)[0]) - ref) <= 1e-5 * abs(ref)
    assert rel_l2(host(g), -V * hd) <= 1e-5
    # uniform cube: E = V_total / 6 (demagnetizing factor 1/3, E = 1/2 N |m|^2 V)
    n, h = (16, 16, 16), (1 / 16,) * 3
    P = D.demag_build_factors(n, h, 41)
    D.demag_energy_field_fft(P, dev(synth.uniform_m(n, 2)), e, None)
    torch.cuda.synchronize()
    assert abs(float(host(e)[0]) - 1.0 / 6.0) < 2e-3


def test_autograd_energy_fft_field(D):
    from paper_1212_3509_gb300.autograd import demag_energy_fn
    n, h = (12, 10, 8), (0.1, 0.1, 0.1)
    P = D.demag_build_factors(n, h, 21)
    m = dev(synth.random_unit_m(n, 5)).requires_grad_()
    E = demag_energy_fn(m, P, "fft_field")
    E.backward()
    g = torch.empty_like(m)
    e = torch.empty(1, dtype=torch.float64, device="cuda")
    D.demag_energy_field_fft(P, m.detach(), e, g)
    torch.cuda.synchronize()
    assert float(E.detach()) == pytest.approx(float(host(e)[0]), rel=1e-12)
    assert torch.equal(m.grad, g)
