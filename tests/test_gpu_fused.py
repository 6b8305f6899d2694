"""Fused mode-1 / mode-2 products (BF16x3) against the FP64 oracle and the three-stage chain.

A grid whose three axes are folded (longer than 16 cells) with ceil(n1 / 2) and
ceil(n2 / 2) at most 128 runs its forward application through the fused kernel
by default; demag_set_fused(plan, False) selects the chain.  Odd extents (63,
127, 255) carry the padding cell of the folded layout; third axes of 17, 33 or
37 cells pad their halves to 16-byte multiples; h1 = 32 leaves three of the four
TMEM lane quadrants of the mode-2 tile without rows.  Halves that are not
multiples of 32 (RAGGED_HALVES) end their contractions inside a k-block, run
tiles of h2 rounded up to 16, pad each half of axes 1 and 2 to a multiple of 8
(h 9 -> 16, 19 -> 24, 115 -> 120) and clip the Z stores to the valid entries."""
import numpy as np
import pytest

import synth
from oracle import full as ofull
from gpu_helpers import assert_close, TOL, dev, host, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FUSED_SHAPES = [
    ((64, 64, 20), (1 / 64,) * 3, 41),
    ((63, 127, 17), (0.02, 0.01, 0.03), 21),
    ((128, 192, 33), (1.0, 1.0, 1.0), 11),
    ((255, 64, 24), (1 / 255, 1 / 64, 1 / 24), 11),
    ((192, 256, 37), (0.5, 0.25, 1.0), 5),
]

RAGGED_HALVES = [
    ((80, 80, 80), (1 / 80,) * 3, 21),                # h 40: k-blocks of 32 + 8, tiles 48 wide
    ((37, 45, 33), (0.03, 0.02, 0.03), 11),           # h 19, 23 (halves padded to 24), tiles 32 wide
    ((17, 18, 17), (1 / 17,) * 3, 11),                # h 9 (padded to 16), tiles 16 wide
    ((160, 100, 21), (0.01, 0.015, 0.05), 11),        # h 80, 50 (odd half at 56), tiles 64 wide
    ((250, 230, 19), (1 / 250, 1 / 230, 1 / 19), 5),  # h 125, 115 (padded to 128, 120), tiles 128 wide
    ((17, 256, 300), (0.02, 0.01, 0.005), 5),         # h 9 / 128 (one k-block against four), 304 slabs, M = 2
    ((256, 17, 33), (0.004, 0.05, 0.03), 5),          # h 128 / 9: 16-wide tiles over four mode-1 k-blocks
]


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1212_3509_gb300 as D
    return D


def _apply(D, P, m, fused):
    n = P.n
    D.demag_set_fused(P, fused)
    phi = torch.empty(n[2], n[1], n[0], device="cuda")
    D.demag_apply_full(P, m, phi, "bf16x3")
    torch.cuda.synchronize()
    D.demag_sync_status(P)
    return host(phi)


@pytest.mark.parametrize("n,h,R", FUSED_SHAPES + RAGGED_HALVES)
def test_fused_vs_oracle_and_chain(D, n, h, R):
    m_h = synth.random_unit_m(n, 3509 + sum(n))
    m = dev(m_h)
    P = D.demag_build_factors(n, h, R)
    fused = _apply(D, P, m, True)
    chain = _apply(D, P, m, False)
    ref_ = ofull.apply_full(m_h, n, h, R)
    ef, ec = rel_l2(fused, ref_), rel_l2(chain, ref_)
    print(f"{n}: fused {ef:.3e} chain {ec:.3e} fused-chain {rel_l2(fused, chain):.3e}")
    assert_close(fused, ref_, TOL["bf16x3"], "fused")
    assert_close(chain, ref_, TOL["bf16x3"], "chain")
    # the same products accumulated in another order
    assert_close(fused, chain, 2 * TOL["bf16x3"], "fused vs chain")


def test_untuned_schedule_follows_grid_size(D):
    """Untuned, a grid of at least 2^20 cells in the folded layout takes the fused
    schedule and a smaller one the chain; demag_set_fused overrides both ways;
    a grid with a short axis has the chain only."""
    for n, want in (((96, 96, 96), 0), ((128, 96, 96), 1), ((128, 128, 12), 0)):
        P = D.demag_build_factors(n, (1 / max(n),) * 3, 11)
        assert D.demag_forward_schedule(P, "bf16x3") == -1  # no tensor-core state yet
        D.demag_reserve_workspace(P, "bf16x3")
        assert D.demag_forward_schedule(P, "bf16x3") == want, n
        D.demag_set_fused(P, True)
        assert D.demag_forward_schedule(P, "bf16x3") == (0 if min(n) <= 16 else 1)
        D.demag_set_fused(P, False)
        assert D.demag_forward_schedule(P, "bf16x3") == 0
        D.demag_set_fused(P, True)
        D.demag_reserve_workspace(P, "tf32x3")
        assert D.demag_forward_schedule(P, "tf32x3") == 0  # the fused kernel is BF16x3 only
        assert D.demag_forward_schedule(P, "fp32") == -1   # not a tensor-core form


def test_fused_repeated_calls_are_identical(D):
    n, h, R = (128, 128, 40), (1 / 128,) * 3, 21
    m = dev(synth.random_unit_m(n, 7))
    P = D.demag_build_factors(n, h, R)
    a = _apply(D, P, m, True)
    b = _apply(D, P, m, True)
    # every output entry is summed by one CTA in a fixed order
    assert np.array_equal(a, b)


def test_fused_and_chain_interleaved_256(D):
    """The bench workload: fused, chain and fused again on one plan (the
    fused kernel's Z fields share the workspace of the chain's stage 1)."""
    n, h, R = (256, 256, 256), (1 / 256,) * 3, 41
    m = dev(synth.vortex_m(n, seed=5))
    P = D.demag_build_factors(n, h, R)
    f1 = _apply(D, P, m, True)
    c = _apply(D, P, m, False)
    f2 = _apply(D, P, m, True)
    assert np.array_equal(f1, f2)
    assert_close(f1, c, 2 * TOL["bf16x3"], "fused vs chain at 256^3")
    # sampled output lines against the oracle: corners, faces and the centre
    lines = [(0, 0), (255, 255), (128, 0), (0, 128), (128, 128), (37, 201)]
    ref = ofull.apply_full_lines(host(m), n, h, R, lines)
    got = np.stack([f1[i3, i2] for i3, i2 in lines])
    assert_close(got, ref, TOL["bf16x3"], "fused 256^3 sampled lines vs oracle")



@pytest.mark.parametrize("n,h,R", [((64, 64, 24), (1 / 64,) * 3, 21), ((128, 64, 19), (0.01, 0.02, 0.03), 11),
                                   ((75, 43, 30), (0.02, 0.03, 0.01), 11)])
def test_fused_stray_field_vs_oracle_and_chain(D, n, h, R):
    """The analytic stray field through the fused schedule (one fused launch per
    direction, with derivative factors along axis 1 or 2, and the mode-3 stage on
    Z, with derivative factors along axis 3 for direction 3) against the oracle
    and against the chain's eight stage launches."""
    from oracle import field as ofield
    m_h = synth.random_unit_m(n, 77 + sum(n))
    m = dev(m_h)
    out = {}
    for fused in (True, False):
        P = D.demag_build_factors(n, h, R)
        D.demag_set_fused(P, fused)
        hd = torch.empty(3, n[2], n[1], n[0], device="cuda")
        D.demag_stray_field_exact(P, m, hd, "bf16x3")
        torch.cuda.synchronize()
        D.demag_sync_status(P)
        out[fused] = host(hd)
    ref = ofield.apply_field(m_h, n, h, R)
    print(f"{n}: fused {rel_l2(out[True], ref):.3e} chain {rel_l2(out[False], ref):.3e}")
    assert_close(out[True], ref, TOL["bf16x3"], "fused field")
    assert_close(out[False], ref, TOL["bf16x3"], "chain field")
    assert_close(out[True], out[False], 2 * TOL["bf16x3"], "fused vs chain field")


@pytest.mark.parametrize("n,h,R", FUSED_SHAPES[:3] + RAGGED_HALVES[:2])
def test_fused_adjoint_vs_oracle_and_chain(D, n, h, R):
    """The adjoint through the fused schedule (the transposed chain's first two
    mode products in one kernel, Za, Zb, Zc per node read MN-major by the
    mode-3 stage) against the oracle's explicit transpose and the chain."""
    rng = np.random.default_rng(5 + sum(n))
    y_h = rng.standard_normal((n[2], n[1], n[0])).astype(np.float32)
    y = dev(y_h)
    out = {}
    for fused in (True, False):
        P = D.demag_build_factors(n, h, R)
        D.demag_set_fused(P, fused)
        g = torch.empty(3, n[2], n[1], n[0], device="cuda")
        D.demag_apply_adjoint(P, y, g, "bf16x3")
        torch.cuda.synchronize()
        D.demag_sync_status(P)
        out[fused] = host(g)
    ref = ofull.apply_adjoint(y_h, n, h, R)
    print(f"{n}: fused {rel_l2(out[True], ref):.3e} chain {rel_l2(out[False], ref):.3e}")
    assert_close(out[True], ref, TOL["bf16x3"], "fused adjoint")
    assert_close(out[False], ref, TOL["bf16x3"], "chain adjoint")
    assert_close(out[True], out[False], 2 * TOL["bf16x3"], "fused vs chain adjoint")


def test_fused_forward_and_adjoint_graph_capturable(D):
    """The fused schedule's launches (split, fused kernel, mode-3 stage, node-sum
    reduction; the same for the adjoint) capture into a CUDA graph and replay to
    the direct calls' bits."""
    n, h, R = (128, 64, 40), (1 / 128,) * 3, 21
    m = dev(synth.random_unit_m(n, 21))
    P = D.demag_build_factors(n, h, R)
    D.demag_set_fused(P, True)
    a = torch.empty(n[2], n[1], n[0], device="cuda")
    ga = torch.empty(3, n[2], n[1], n[0], device="cuda")
    D.demag_apply_full(P, m, a, "bf16x3")  # the first calls build the tensor-core state
    D.demag_apply_adjoint(P, a, ga, "bf16x3")
    torch.cuda.synchronize()
    b = torch.zeros_like(a)
    gb = torch.zeros_like(ga)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            D.demag_apply_full(P, m, b, "bf16x3", stream=s)
            D.demag_apply_adjoint(P, b, gb, "bf16x3", stream=s)
    g.replay()
    torch.cuda.synchronize()
    D.demag_sync_status(P)
    assert torch.equal(a, b) and torch.equal(ga, gb)


def test_fused_batch_equals_single_applies(D):
    """A batch mixing both schedules: one fused mode-1 / mode-2 launch over the
    grids with the fused schedule (largest first; halves of 40, 64 / 32 and
    19 / 23 entries), whose mode-3 stages run inside the persistent launch
    beside the chain grids' three stages, and the thin last stage of a film on
    CUDA cores after it.  Every tile runs the MMA sequence of the grid's own
    call and the film's thin stage the same CUDA-core kernel, so each output
    equals that call bit for bit; the captured graph of the batch replays the
    same bits."""
    cases = [((80, 80, 80), (1 / 80,) * 3, 21, True),
             ((48, 40, 37), (1 / 48,) * 3, 21, False),
             ((128, 64, 40), (1 / 128,) * 3, 21, True),
             ((37, 45, 33), (0.03, 0.02, 0.03), 11, True),
             ((96, 64, 8), (1 / 96,) * 3, 21, True)]   # axis 3 not folded: the chain
    plans, ms, single = [], [], []
    for i, (n, h, R, fused) in enumerate(cases):
        P = D.demag_build_factors(n, h, R)
        D.demag_set_fused(P, fused)
        m = dev(synth.random_unit_m(n, 9100 + i))
        phi = torch.empty(n[2], n[1], n[0], device="cuda")
        D.demag_apply_full(P, m, phi, "bf16x3")
        plans.append(P)
        ms.append(m)
        single.append(phi)
    assert [D.demag_forward_schedule(P, "bf16x3") for P in plans] == [1, 0, 1, 1, 0]
    before = D.demag_launch_count(plans[0])
    outs = [torch.full_like(p, float("nan")) for p in single]
    D.demag_apply_full_batched(plans, ms, outs, "bf16x3")
    torch.cuda.synchronize()
    for P in plans:
        D.demag_sync_status(P)
    # split, fused mode-1 / mode-2 products, persistent launch, the film's thin stage, reduction
    assert D.demag_launch_count(plans[0]) - before == 5
    for (n, _, _, _), got, ref in zip(cases, outs, single):
        if n[0] > 16 and n[1] > 16:  # a thin last axis runs the single call's CUDA-core stage
            assert torch.equal(got, ref), n
        else:
            assert_close(host(got), host(ref), TOL["bf16x3"], n)
    n, h, R, _ = cases[3]
    assert_close(host(outs[3]), ofull.apply_full(host(ms[3]), n, h, R), TOL["bf16x3"], "ragged halves in the batch")
    gouts = [torch.full_like(p, float("nan")) for p in single]
    G = D.demag_graph_create_batched(plans, ms, gouts, "bf16x3")
    assert G.kernels == 5
    G.launch()
    torch.cuda.synchronize()
    for got, want in zip(gouts, outs):
        assert torch.equal(got, want)
    G.close()
