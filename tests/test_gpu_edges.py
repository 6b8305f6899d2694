"""Edge cases of the GPU path: the longest FFT axis (n_p = 8192), the largest
number of quadrature terms (R = 513, M = 256), the smallest (R = 5), axes too
long for the FFT path, and single-cell axes, each against the FP64 oracle."""
import numpy as np
import pytest

import synth
from oracle import full as ofull, structured as ost
from gpu_helpers import assert_close, TOL, dev, host, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1212_3509_gb300 as D
    return D


def test_cp_longest_fft_axis_8192(D):
    # axis 1 at the largest supported FFT length (complex length 8192, the
    # 2^13 kernel with one block per SM); axes 2 and 3 short, one launch each
    n, h, R, r = (8192, 40, 3), (1 / 8192,) * 3, 21, 2
    lam, U = synth.cp_inputs(n, r, 1220)
    P = D.demag_build_factors(n, h, R)
    M, ns = P.M, sum(n)
    w = torch.empty(M * 3 * r, device="cuda")
    oU = torch.empty(M * 3 * r * ns, device="cuda")
    D.demag_apply_cp(P, r, dev(lam), dev(U.ravel()), w, oU)
    torch.cuda.synchronize()
    got = host(oU)
    off = 0
    for p, idx in ((0, [0, 1, 2, 777, 4095, 4096, 6000, 8190, 8191]), (1, list(range(40))), (2, [0, 1, 2])):
        blk = got[off:off + M * 3 * r * n[p]].reshape(M, 3, r, n[p])[..., idx]
        ref = ost.apply_cp_entries(lam, U, n, h, R, p, idx)
        err = rel_l2(blk, ref)
        print(f"axis {p + 1} (n = {n[p]}): rel L2 {err:.3e}")
        assert_close(blk, ref, TOL["fp32"])
        off += M * 3 * r * n[p]


def test_fft_axis_too_long_is_rejected(D):
    P = D.demag_build_factors((8193, 2, 2), (1.0, 1.0, 1.0), 11)
    w = torch.empty(P.M * 3, device="cuda")
    oU = torch.empty(P.M * 3 * (8193 + 4), device="cuda")
    with pytest.raises(D.DemagError) as ei:
        D.demag_apply_cp(P, 1, torch.ones(3, device="cuda"), torch.ones(3 * (8193 + 4), device="cuda"), w, oU)
    assert ei.value.status == 5  # DEMAG_EUNSUPPORTED


@pytest.mark.parametrize("R", [5, 129, 513])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x3", "tf32x3"])
def test_fewest_and_most_terms_full_and_adjoint(D, R, prec):
    n, h = (12, 9, 16), (1 / 16,) * 3
    m = synth.random_unit_m(n, 1221)
    P = D.demag_build_factors(n, h, R)
    assert P.M == (R - 1) // 2
    phi = torch.empty(n[2], n[1], n[0], device="cuda")
    D.demag_apply_full(P, dev(m), phi, prec)
    rng = np.random.default_rng(5)
    y = rng.standard_normal((n[2], n[1], n[0])).astype(np.float32)
    g = torch.empty(3, n[2], n[1], n[0], device="cuda")
    D.demag_apply_adjoint(P, dev(y), g, prec)
    torch.cuda.synchronize()
    D.demag_sync_status(P)
    ref_f, ref_a = ofull.apply_full(m, n, h, R), ofull.apply_adjoint(y, n, h, R)
    e1 = rel_l2(host(phi), ref_f)
    e2 = rel_l2(host(g), ref_a)
    print(f"R = {R} {prec}: forward {e1:.3e}, adjoint {e2:.3e}")
    assert_close(host(phi), ref_f, TOL[prec], "forward")
    assert_close(host(g), ref_a, TOL[prec], "adjoint")


@pytest.mark.parametrize("R", [129, 513])
def test_most_terms_cp(D, R):
    n, h, r = (64, 33, 7), (1 / 64,) * 3, 3
    lam, U = synth.cp_inputs(n, r, 1222)
    P = D.demag_build_factors(n, h, R)
    M, ns = P.M, sum(n)
    w = torch.empty(M * 3 * r, device="cuda")
    oU = torch.empty(M * 3 * r * ns, device="cuda")
    D.demag_apply_cp(P, r, dev(lam), dev(U.ravel()), w, oU)
    torch.cuda.synchronize()
    rw, rU = ost.apply_cp(lam, U, n, h, R)
    assert rel_l2(host(w), rw.ravel()) < 1e-6
    assert_close(host(oU), np.concatenate([rU[p].ravel() for p in range(3)]), TOL["fp32"])


@pytest.mark.parametrize("n", [(1, 17, 9), (23, 1, 1), (1, 1, 30)])
def test_single_cell_axes(D, n):
    h, R = (0.05,) * 3, 21
    m = synth.random_unit_m(n, 1223)
    P = D.demag_build_factors(n, h, R)
    ref = ofull.apply_full(m, n, h, R)
    for prec in ("fp32", "bf16x3"):
        phi = torch.empty(n[2], n[1], n[0], device="cuda")
        D.demag_apply_full(P, dev(m), phi, prec)
        torch.cuda.synchronize()
        assert_close(host(phi), ref, TOL[prec])


def test_compression_term_limit(D):
    # the compression of Alg. 2 keeps M x M Gram matrices in shared memory: M <= 64
    P = D.demag_build_factors((16, 16, 16), (1 / 16,) * 3, 131)
    with pytest.raises(D.DemagError) as ei:
        D.demag_compress_kernel(P, 1e-6)
    assert ei.value.status == 5  # DEMAG_EUNSUPPORTED
