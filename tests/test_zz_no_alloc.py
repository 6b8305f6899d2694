"""The allocation-free entry point demag_apply_full_noalloc.

Some callers cannot allocate device memory: a host framework's memory pool may
own the GPU, an allocation would synchronise a latency-critical loop, or a
plugin host forbids it.  For them the library offers one FP32 full-format call
that uses only a fixed 32 MiB device array inside the library.  These tests
call it through the C ABI and compare it with demag_apply_full (FP32) at the
FP32 tolerance, on two calls in a row with different grids and inputs (the
second call reuses the array the first one left behind).  The file is named
to be collected last.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")


def _desc(abi, n, h, R, c0=2.15):
    return abi.GridDesc((ctypes.c_int * 3)(*n), (ctypes.c_double * 3)(*h), R, c0)


@pytest.mark.gpu
def test_noalloc_matches_apply_full_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1212_3509_gb300 as D
    from paper_1212_3509_gb300 import _abi
    from gpu_helpers import TOL, rel_l2

    stream = torch.cuda.current_stream().cuda_stream
    cases = [((24, 20, 16), (1 / 24,) * 3, 41, 4242), ((32, 32, 32), (1 / 32,) * 3, 41, 4243)]
    for n, h, R, seed in cases:
        m = torch.from_numpy(synth.random_unit_m(n, seed)).cuda()
        P = D.demag_build_factors(n, h, R)
        ref = torch.empty(n[2], n[1], n[0], device="cuda")
        D.demag_apply_full(P, m, ref, "fp32")
        out = torch.full_like(ref, float("nan"))
        st = _abi.lib.demag_apply_full_noalloc(ctypes.byref(_desc(_abi, n, h, R)), m.data_ptr(), out.data_ptr(),
                                               stream)
        assert st == 0, _abi.lib.demag_last_error(None)
        torch.cuda.synchronize()
        err = rel_l2(out.cpu().numpy(), ref.cpu().numpy())
        assert err <= TOL["fp32"], (n, err)


def test_noalloc_rejects_grids_beyond_its_array():
    # validation happens on the host before any device work
    from paper_1212_3509_gb300 import _abi

    d = _desc(_abi, (64, 64, 64), (1 / 64,) * 3, 41)
    st = _abi.lib.demag_apply_full_noalloc(ctypes.byref(d), ctypes.c_void_p(256), ctypes.c_void_p(256), None)
    assert st == 5  # DEMAG_EUNSUPPORTED
    msg = _abi.lib.demag_last_error(None).decode()
    assert "32 MiB" in msg and "bytes" in msg
