"""The allocation-free entry point demag_apply_full_noalloc.

Some callers cannot allocate device memory: a host framework's memory pool may
own the GPU, an allocation would synchronise a latency-critical loop, or a
plugin host forbids it.  For them the library offers one FP32 full-format call
that uses only a fixed 32 MiB device array inside the library.  These tests
call it through the C ABI and compare it with demag_apply_full (FP32) and with
the FP64 oracle at the FP32 tolerance, on three calls in a row with different
grids and inputs (each call reuses the array the one before left behind; the
last grid fills the array to within 7 KB of its end).  The file is named
to be collected last.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")


def _desc(abi, n, h, R, c0=2.15):
    return abi.GridDesc((ctypes.c_int * 3)(*n), (ctypes.c_double * 3)(*h), R, c0)


def _need(n, R):
    """Scratch bytes of one call, as the header states them (parts rounded to 256)."""
    M = (R - 1) // 2
    glen = 2 * max(n) - 1
    N = n[0] * n[1] * n[2]

    def al(b):
        return (b + 255) & ~255

    return (al(8 * 3 * M) + al(8 * M) + al(8 * M * 6 * glen) + al(4 * M * 2 * sum(x * x for x in n))
            + al(4 * (2 * M + 3) * N))


LIMIT = 32 << 20


@pytest.mark.gpu
def test_noalloc_matches_apply_full_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1212_3509_gb300 as D
    from paper_1212_3509_gb300 import _abi
    from gpu_helpers import TOL, assert_close
    from oracle import full as ofull

    stream = torch.cuda.current_stream().cuda_stream
    # the third grid needs all but 6912 bytes of the array, so its far end is used
    cases = [((24, 20, 16), (1 / 24,) * 3, 41, 4242), ((32, 32, 32), (1 / 32,) * 3, 41, 4243),
             ((52, 46, 77), (1 / 77,) * 3, 41, 4244)]
    assert LIMIT - 8192 < _need(cases[2][0], 41) <= LIMIT
    for n, h, R, seed in cases:
        m_h = synth.random_unit_m(n, seed)
        m = torch.from_numpy(m_h).cuda()
        P = D.demag_build_factors(n, h, R)
        ref = torch.empty(n[2], n[1], n[0], device="cuda")
        D.demag_apply_full(P, m, ref, "fp32")
        out = torch.full_like(ref, float("nan"))
        st = _abi.lib.demag_apply_full_noalloc(ctypes.byref(_desc(_abi, n, h, R)), m.data_ptr(), out.data_ptr(),
                                               stream)
        assert st == 0, _abi.lib.demag_last_error(None)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert_close(got, ref.cpu().numpy(), TOL["fp32"], ("against demag_apply_full", n))
        assert_close(got, ofull.apply_full(m_h, n, h, R), TOL["fp32"], ("against the oracle", n))


def test_noalloc_rejects_grids_beyond_its_array():
    # validation happens on the host before any device work
    from paper_1212_3509_gb300 import _abi

    for n in ((64, 64, 64), (48, 55, 70)):  # the second needs 2560 bytes more than the array holds
        assert _need(n, 41) > LIMIT
        d = _desc(_abi, n, (1 / max(n),) * 3, 41)
        st = _abi.lib.demag_apply_full_noalloc(ctypes.byref(d), ctypes.c_void_p(256), ctypes.c_void_p(256), None)
        assert st == 5  # DEMAG_EUNSUPPORTED
        msg = _abi.lib.demag_last_error(None).decode()
        assert "32 MiB" in msg and str(_need(n, 41)) in msg
