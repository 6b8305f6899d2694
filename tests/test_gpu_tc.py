"""Tensor-core (tcgen05) split-precision forms against the FP64 oracle.

Shapes cover partial row tiles, contraction lengths that are not multiples of
the 32-wide k-block, output widths below and above the 256-wide N tile, and
thin films."""
import numpy as np
import pytest

import synth
from oracle import full as ofull
from gpu_helpers import assert_close, TOL, dev, host, rel_l2

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
    ((64, 32, 96), (0.02, 0.02, 0.02), 21),
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
    ref_ = ofull.apply_full(m, n, h, R)
    err = rel_l2(host(phi), ref_)
    print(f"{prec} {n}: rel L2 {err:.3e}")
    assert_close(host(phi), ref_, TOL[prec])


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
    ref_ = ofull.apply_adjoint(y, n, h, R)
    err = rel_l2(host(g), ref_)
    print(f"{prec} adjoint {n}: rel L2 {err:.3e}")
    assert_close(host(g), ref_, TOL[prec])


@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("n", [(40, 24, 16), (64, 32, 96), (96, 64, 32)])
def test_bf16x3_repeated_calls_are_identical(D, n, fused):
    # (64, 32, 96) and (96, 64, 32) store every stage of the chain through TMA
    # with an odd number of 32-column chunks per tile; both take the fused
    # schedule when asked ((40, 24, 16) has a short axis: the chain only)
    h, R = (0.05,) * 3, 21
    m = dev(synth.random_unit_m(n, 99))
    P = D.demag_build_factors(n, h, R)
    D.demag_set_fused(P, fused)
    a = torch.empty(n[2], n[1], n[0], device="cuda")
    b = torch.empty_like(a)
    D.demag_apply_full(P, m, a, "bf16x3")
    D.demag_apply_full(P, m, b, "bf16x3")
    torch.cuda.synchronize()
    assert torch.equal(a, b)


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_grouped_batch_equals_single_applies(D, prec):
    """One persistent launch over every stage of grids of different shapes
    (TMA-stored and directly stored epilogues mixed, a plan listed twice, later
    stages waiting for earlier ones through completion counters) gives, bit for
    bit, what separate calls give on grids whose axes all run on the tensor
    cores: every tile runs the same MMA sequence.  A thin last axis (at most 16
    cells) runs on CUDA cores in both, so those grids agree bit for bit too;
    other thin axes run on CUDA cores in a single call but as padded
    tensor-core tiles in the batch, so those grids agree to the split-form
    tolerance.  The batch runs the three-stage chain, so the separate calls are
    held to it too."""
    cases = [TC_SHAPES[0], TC_SHAPES[1], TC_SHAPES[4], TC_SHAPES[7], TC_SHAPES[8]]
    plans, ms, single = [], [], []
    for i, (n, h, R) in enumerate(cases):
        P = D.demag_build_factors(n, h, R)
        D.demag_set_fused(P, False)
        m = dev(synth.random_unit_m(n, 4242 + i))
        phi = torch.empty(n[2], n[1], n[0], device="cuda")
        D.demag_apply_full(P, m, phi, prec)
        plans.append(P)
        ms.append(m)
        single.append(phi)
    # the first plan again, with another input, at the end of the list
    n0 = cases[0][0]
    m_extra = dev(synth.random_unit_m(n0, 777))
    ref_extra = torch.empty(n0[2], n0[1], n0[0], device="cuda")
    D.demag_apply_full(plans[0], m_extra, ref_extra, prec)
    outs = [torch.full_like(p, float("nan")) for p in single] + [torch.full_like(ref_extra, float("nan"))]
    D.demag_apply_full_batched(plans + [plans[0]], ms + [m_extra], outs, prec)
    torch.cuda.synchronize()
    for P in plans:
        D.demag_sync_status(P)
    for (n, _, _), got, ref in zip(cases + [cases[0]], outs, single + [ref_extra]):
        if n[0] > 16 and n[1] > 16:  # a thin last axis runs the single call's CUDA-core stage
            assert torch.equal(got, ref), n
        else:
            assert_close(host(got), host(ref), TOL[prec], n)
    n, h, R = cases[3]
    ref_ = ofull.apply_full(host(ms[3]), n, h, R)
    err = rel_l2(host(outs[3]), ref_)
    assert_close(host(outs[3]), ref_, TOL[prec])


@pytest.mark.parametrize("prec", ["bf16x3", "fp32"])
def test_graph_replay_equals_batched_call(D, prec):
    """The captured graph of a batched apply reproduces the direct call bit for
    bit on replay, picks up new input values, and rejects a repeated plan."""
    cases = [TC_SHAPES[0], TC_SHAPES[1], ((64, 32, 96), (0.02,) * 3, 21)]
    plans, ms, ref, outs = [], [], [], []
    for i, (n, h, R) in enumerate(cases):
        P = D.demag_build_factors(n, h, R)
        D.demag_reserve_workspace(P, prec)
        plans.append(P)
        ms.append(dev(synth.random_unit_m(n, 31 + i)))
        ref.append(torch.empty(n[2], n[1], n[0], device="cuda"))
        outs.append(torch.full_like(ref[-1], float("nan")))
    D.demag_apply_full_batched(plans, ms, ref, prec)
    G = D.demag_graph_create_batched(plans, ms, outs, prec)
    assert G.kernels > 0
    torch.cuda.synchronize()
    assert all(torch.isnan(o).all() for o in outs)  # capture runs nothing
    before = D.demag_launch_count(plans[0])
    for _ in range(2):
        G.launch()
        torch.cuda.synchronize()
        for got, want in zip(outs, ref):
            assert torch.equal(got, want)
    assert D.demag_launch_count(plans[0]) == before + 2 * G.kernels
    # new values in the same buffers
    ms[1].copy_(dev(synth.random_unit_m(cases[1][0], 555)))
    D.demag_apply_full_batched(plans, ms, ref, prec)
    G.launch()
    torch.cuda.synchronize()
    for P in plans:
        D.demag_sync_status(P)
    assert torch.equal(outs[1], ref[1])
    with pytest.raises(D.DemagError):
        D.demag_graph_create_batched([plans[0], plans[0]], [ms[0], ms[0]], [outs[0], outs[0]], prec)
    G.close()


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_unaligned_pointers_take_the_scalar_path(D, prec):
    """m and phi that start 4 bytes past a 16-byte boundary give the same
    result as aligned buffers (the vectorised split and reduce are skipped)."""
    n, h, R = (32, 24, 40), (1 / 40,) * 3, 21
    m = dev(synth.random_unit_m(n, 17))
    P = D.demag_build_factors(n, h, R)
    ref = torch.empty(n[2], n[1], n[0], device="cuda")
    D.demag_apply_full(P, m, ref, prec)
    m_buf = torch.empty(m.numel() + 1, device="cuda")
    m_buf[1:].copy_(m.reshape(-1))
    phi_buf = torch.full((ref.numel() + 1,), float("nan"), device="cuda")
    D.demag_apply_full(P, m_buf[1:].data_ptr(), phi_buf[1:].data_ptr(), prec)
    torch.cuda.synchronize()
    assert torch.equal(phi_buf[1:].reshape(ref.shape), ref)
