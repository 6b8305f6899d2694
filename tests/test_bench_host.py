"""Host-side helpers of bench.py (CPU only): the traffic records keyed to the kernel sources, the
R rule of the energy study and the algorithmic bytes of the 3D FFT passes."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_traffic_is_reported_only_for_the_captured_sources(monkeypatch):
    rec = dict(bench.NCU_TRAFFIC["tc_fused"])
    monkeypatch.setitem(bench.NCU_TRAFFIC, "tc_fused", dict(rec, sha=bench.sources_sha(rec["sources"])))
    per_cell = rec["bytes_per_cell"]
    assert bench.ncu_traffic("tc_fused", 256 ** 3, "bytes_per_cell") == pytest.approx(per_cell * 256 ** 3)
    # a kernel changed since the capture: no traffic figure
    monkeypatch.setitem(bench.NCU_TRAFFIC, "tc_fused", dict(rec, sha="0000000000000000"))
    assert bench.ncu_traffic("tc_fused", 256 ** 3, "bytes_per_cell") is None


def test_sources_sha_depends_on_every_named_file():
    a = bench.sources_sha(("full_tc.cu",))
    b = bench.sources_sha(("full_tc.cu", "tc_ptx.cuh"))
    assert len(a) == len(b) == 16 and a != b


def test_energy_study_terms_grow_with_n():
    # tau_max = sinh(c0 ln M) >= 8 n with M in {64, 128, 256}, else 513
    assert [bench.fig2_terms(n) for n in (64, 128, 256, 512, 1024, 2048, 4096)] == [129, 129, 129, 257, 257,
                                                                                     257, 513]


def test_fft3d_pass_bytes_at_256():
    b = bench.fft3d_pass_bytes((256, 256, 256))
    assert len(b) == 5 and all(x > 0 for x in b)
    assert sum(b) == pytest.approx(3.706e9, rel=2e-3)  # the 3D FFT convolution's algorithmic bytes


def test_single_rank_rate():
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(10, 2.0, 1) == pytest.approx(10 * 1e3 / 2.0)
