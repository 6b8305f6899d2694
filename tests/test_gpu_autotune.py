"""Autotuned launch shapes and grouped FFT launches.

Tuning changes only how work is split over blocks and scheduled (nodes per FFT
block; output-column tile width, operand stages and tile order of the
tensor-core GEMMs); every output element is computed by the same sequence of
operations, so tuned and untuned plans agree bit for bit."""
import numpy as np
import pytest

import synth
from gpu_helpers import dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1212_3509_gb300 as D
    return D


def _fft_length(n):
    """Circulant embedding length: the power of two >= 2n - 1 (at least 2)."""
    L = 2
    while L < 2 * n - 1:
        L *= 2
    return L


def _cp(D, P, n, r, B, tune):
    if tune:
        D.demag_autotune(P, True)
    lam = np.empty((B, 3, r), dtype=np.float32)
    U = np.empty((B, 3 * r * sum(n)), dtype=np.float32)
    for b in range(B):
        lam[b], u = synth.cp_inputs(n, r, 90 + b)
        U[b] = u.ravel()
    w = torch.empty(B * P.M * 3 * r, device="cuda")
    oU = torch.empty(B * P.M * 3 * r * sum(n), device="cuda")
    D.demag_apply_cp_batched(P, B, r, dev(lam), dev(U), w, oU)
    D.demag_apply_cp_batched(P, B, r, dev(lam), dev(U), w, oU)
    torch.cuda.synchronize()
    return w, oU


@pytest.mark.parametrize("n", [(256, 256, 256), (37, 50, 9)])
def test_fft_node_group_tuning_keeps_results(D, n):
    h = (1.0 / max(n),) * 3
    r, B = 4, 8
    P0 = D.demag_build_factors(n, h, 41)
    P1 = D.demag_build_factors(n, h, 41)
    w0, o0 = _cp(D, P0, n, r, B, tune=False)
    w1, o1 = _cp(D, P1, n, r, B, tune=True)
    assert torch.equal(o0, o1) and torch.equal(w0, w1)
    entries = [D.demag_autotune_entry(P1, i) for i in range(D.demag_autotune_count(P1))]
    lengths = {_fft_length(p) for p in n}
    assert len(entries) == len(lengths)  # one tuned launch per distinct FFT length
    for e in entries:
        assert e["kind"] == "fft_node_group" and 1 <= e["value"] <= P1.M and e["ms"] > 0
    assert D.demag_autotune_count(P0) == 0


def test_structured_axes_share_one_launch(D):
    # all three axes of a cube have one FFT length: one FFT launch + the weights
    n, h = (64, 64, 64), (1 / 64,) * 3
    P = D.demag_build_factors(n, h, 21)
    r = 2
    lam, U = synth.cp_inputs(n, r, 5)
    w = torch.empty(P.M * 3 * r, device="cuda")
    oU = torch.empty(P.M * 3 * r * sum(n), device="cuda")
    c0 = D.demag_launch_count(P)
    D.demag_apply_cp(P, r, dev(lam), dev(U.ravel()), w, oU)
    assert D.demag_launch_count(P) - c0 == 2
    # lengths 64, 64, 16 -> two FFT launches
    n2 = (64, 40, 9)
    P2 = D.demag_build_factors(n2, (1 / 64,) * 3, 21)
    lam, U = synth.cp_inputs(n2, r, 5)
    w = torch.empty(P2.M * 3 * r, device="cuda")
    oU = torch.empty(P2.M * 3 * r * sum(n2), device="cuda")
    c0 = D.demag_launch_count(P2)
    D.demag_apply_cp(P2, r, dev(lam), dev(U.ravel()), w, oU)
    torch.cuda.synchronize()
    assert D.demag_launch_count(P2) - c0 == 3


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_tile_width_tuning_keeps_results(D, prec):
    n, h, R = (300, 20, 160), (1 / 300,) * 3, 11
    m = dev(synth.random_unit_m(n, 8))
    out = []
    for tune in (False, True):
        P = D.demag_build_factors(n, h, R)
        if tune:
            D.demag_autotune(P, True)
        phi = torch.empty(n[2], n[1], n[0], device="cuda")
        D.demag_apply_full(P, m, phi, prec)
        y = torch.empty(3, n[2], n[1], n[0], device="cuda")
        D.demag_apply_adjoint(P, phi, y, prec)
        torch.cuda.synchronize()
        D.demag_sync_status(P)
        out.append((phi, y, P))
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
    P = out[1][2]
    entries = [D.demag_autotune_entry(P, i) for i in range(D.demag_autotune_count(P))]
    kind = f"{prec}_tile_width"
    tuned = {e["key"][0]: e for e in entries if e["kind"] == kind}
    # folded axis 1 (n = 300, 150 per half, default width 160) and axis 3 (n = 160,
    # 80 per half, default 80) have narrower candidates: forward and adjoint programs
    assert set(tuned) == {0, 2, 3, 5}
    for e in tuned.values():
        assert e["value"] in (e["key"][1], 128, 64)
    # every tensor-core program also gets its stage count and tile order
    stages = {e["key"][0]: e for e in entries if e["kind"] == f"{prec}_stages"}
    order = {e["key"][0]: e for e in entries if e["kind"] == f"{prec}_tile_order"}
    assert set(stages) == set(order) == set(range(6))
    for e in list(stages.values()) + list(order.values()) + list(tuned.values()):
        assert 0 < e["ms"] <= e["ms_default"]  # the default was a candidate
    assert all(e["value"] in (0, 4, 3, 2) for e in stages.values())
    assert all(e["value"] in (0, 1) for e in order.values())


def test_tuning_cache_round_trip(D, tmp_path):
    """Entries saved by a tuned plan are loaded by a new plan of the same grid on the
    same GPU, which then tunes nothing and gives the same results bit for bit; a plan
    of another grid loads none of them."""
    n, h, R = (96, 80, 64), (1 / 96,) * 3, 21
    m = dev(synth.random_unit_m(n, 31))
    path = str(tmp_path / "tune.jsonl")
    P1 = D.demag_build_factors(n, h, R)
    D.demag_autotune(P1, True)
    a = torch.empty(n[2], n[1], n[0], device="cuda")
    D.demag_apply_full(P1, m, a, "bf16x3")
    count1 = D.demag_autotune_count(P1)
    assert count1 > 0
    D.demag_autotune_save(P1, path)
    P2 = D.demag_build_factors(n, h, R)
    assert D.demag_autotune_load(P2, path) == count1
    D.demag_autotune(P2, True)
    b = torch.empty_like(a)
    D.demag_apply_full(P2, m, b, "bf16x3")
    torch.cuda.synchronize()
    assert D.demag_autotune_count(P2) == count1  # nothing tuned again
    e1 = sorted((e["kind"], tuple(e["key"]), e["value"]) for e in
                (D.demag_autotune_entry(P1, i) for i in range(count1)))
    e2 = sorted((e["kind"], tuple(e["key"]), e["value"]) for e in
                (D.demag_autotune_entry(P2, i) for i in range(count1)))
    assert e1 == e2
    assert torch.equal(a, b)
    P3 = D.demag_build_factors((96, 80, 65), h, R)
    assert D.demag_autotune_load(P3, path) == 0


def test_store_box_tuning_keeps_results(D):
    """At 128^3 every stage's 128-row blocks lie in one outer index, so the tuner also
    times one 128-row store box per chunk against per-warp boxes; whichever it keeps,
    the results equal the untuned plan's bit for bit (forward and adjoint)."""
    n, h, R = (128, 128, 128), (1 / 128,) * 3, 11
    m = dev(synth.random_unit_m(n, 12))
    out = []
    for tune in (False, True):
        P = D.demag_build_factors(n, h, R)
        D.demag_set_fused(P, True)  # the same forward schedule in both plans
        if tune:
            D.demag_autotune(P, True)
        phi = torch.empty(n[2], n[1], n[0], device="cuda")
        D.demag_apply_full(P, m, phi, "bf16x3")
        y = torch.empty(3, n[2], n[1], n[0], device="cuda")
        D.demag_apply_adjoint(P, phi, y, "bf16x3")
        torch.cuda.synchronize()
        D.demag_sync_status(P)
        out.append((phi, y, P))
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
    P = out[1][2]
    entries = [D.demag_autotune_entry(P, i) for i in range(D.demag_autotune_count(P))]
    boxes = {e["key"][0]: e for e in entries if e["kind"] == "bf16x3_store_boxes"}
    # programs 0-5 of the chains and 6, 7, the mode-3 stages of the fused forward
    # and adjoint applications (128^3 has them: every axis folded, 64 entries per half)
    assert set(boxes) == set(range(8)) and all(e["value"] in (0, 1) for e in boxes.values())


def test_forward_schedule_tuning(D):
    """On a grid with the fused schedule the tuner times it against the three-stage
    chain and keeps the faster; the tuned plan's output equals, bit for bit, that of
    a plan forced to the chosen schedule."""
    n, h, R = (128, 128, 64), (1 / 128,) * 3, 21
    m = dev(synth.random_unit_m(n, 41))
    P = D.demag_build_factors(n, h, R)
    D.demag_autotune(P, True)
    a = torch.empty(n[2], n[1], n[0], device="cuda")
    D.demag_apply_full(P, m, a, "bf16x3")
    torch.cuda.synchronize()
    entries = [D.demag_autotune_entry(P, i) for i in range(D.demag_autotune_count(P))]
    sched = [e for e in entries if e["kind"] == "bf16x3_schedule"]
    assert len(sched) == 1 and sched[0]["value"] in (0, 1) and sched[0]["key"] == [0, 1, 0]
    assert 0 < sched[0]["ms"] <= sched[0]["ms_default"]  # ms_default: the fused schedule's time
    Q = D.demag_build_factors(n, h, R)
    D.demag_set_fused(Q, bool(sched[0]["value"]))
    b = torch.empty_like(a)
    D.demag_apply_full(Q, m, b, "bf16x3")
    torch.cuda.synchronize()
    D.demag_sync_status(P)
    assert torch.equal(a, b)
