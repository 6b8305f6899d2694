"""The analytic stray field on the GPU (demag_stray_field_exact) against the
FP64 oracle (oracle/field.py, pinned to the derivative of the potential and
to the closed-form field of a uniformly magnetized box)."""
import numpy as np
import pytest

import synth
from oracle import field as ofield
from gpu_helpers import assert_close, TOL, dev, host, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SHAPES = [
    ((16, 12, 8), (1 / 16,) * 3, 21),           # every axis short: CUDA-core stages in the split forms
    ((40, 24, 36), (0.025, 0.03, 0.02), 21),    # tensor-core stages
    ((64, 32, 96), (1 / 96,) * 3, 21),          # TMA-stored epilogues
    ((20, 13, 7), (0.1, 0.2, 0.15), 11),        # mixed
]


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1212_3509_gb300 as D
    return D


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("n,h,R", SHAPES)
def test_exact_stray_field_vs_oracle(D, n, h, R, prec):
    m = synth.random_unit_m(n, 1700 + sum(n))
    P = D.demag_build_factors(n, h, R)
    hd = torch.empty(3, n[2], n[1], n[0], device="cuda")
    D.demag_stray_field_exact(P, dev(m), hd, prec)
    torch.cuda.synchronize()
    D.demag_sync_status(P)
    ref = ofield.apply_field(m, n, h, R)
    err = rel_l2(host(hd), ref)
    print(f"{prec} {n}: rel L2 {err:.3e}")
    assert_close(host(hd), ref, TOL[prec])


def test_exact_field_close_to_difference_field(D):
    # smooth magnetization: the finite-difference field of the same operator
    # differs from the analytic one by O(h^2) away from the faces
    n, h, R = (32, 32, 32), (1 / 32,) * 3, 21
    m = synth.smooth_m(n).astype(np.float32)
    P = D.demag_build_factors(n, h, R)
    hd = torch.empty(3, 32, 32, 32, device="cuda")
    phi = torch.empty(32, 32, 32, device="cuda")
    fd = torch.empty_like(hd)
    D.demag_stray_field_exact(P, dev(m), hd, "bf16x3")
    D.demag_apply_full(P, dev(m), phi, "bf16x3")
    D.demag_stray_field(P, phi, fd)
    torch.cuda.synchronize()
    inner = (slice(None), slice(6, -6), slice(6, -6), slice(6, -6))
    a, b = host(hd)[inner], host(fd)[inner]
    assert np.linalg.norm(a - b) / np.linalg.norm(a) < 5e-3


def test_uniform_cube_field_opposes_m(D):
    n, h = (24, 24, 24), (1 / 24,) * 3
    m = synth.uniform_m(n, 2)
    P = D.demag_build_factors(n, h, 41)
    hd = torch.empty(3, 24, 24, 24, device="cuda")
    D.demag_stray_field_exact(P, dev(m), hd, "bf16x3")
    torch.cuda.synchronize()
    g = host(hd)
    # the demagnetizing factor of a cube is 1/3: the mean field is -m/3
    assert abs(g[2].mean() + 1.0 / 3.0) < 5e-3
    assert abs(g[0].mean()) < 1e-6 and abs(g[1].mean()) < 1e-6
