"""The bounded-wait failure path of the tensor-core kernels, made to happen.

Every device-side wait of the tcgen05 pipeline (mbarriers between its roles,
completion counters between tiles of one launch) gives up after the plan's
wait limit, sets DEMAG_ETIMEOUT in the plan's status word, lets every copy and
MMA it issued land, releases its tensor memory and returns.  A zero limit makes
the first wait that is not already satisfied give up; the status must say so,
and the same plan with the default limit must then give the oracle's result.
No fault, trap or endless loop is involved: the kernel returns on its own.
"""
import numpy as np
import pytest

import synth
from oracle import full as ofull
from gpu_helpers import TOL, assert_close, dev, host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1212_3509_gb300 as D
    return D


# every axis > 16 cells: all stages on tcgen05, through the three-stage chain
# (its kernel's abort path) or the fused schedule (the fused kernel's abort
# path, then the mode-3 stage's)
@pytest.mark.parametrize("n,fused", [((48, 40, 37), False), ((48, 40, 37), True), ((64, 64, 20), True)])
def test_zero_wait_limit_reports_timeout_then_plan_recovers(D, n, fused):
    h, R = (1 / max(n),) * 3, 21
    m = synth.random_unit_m(n, 1230)
    P = D.demag_build_factors(n, h, R)
    D.demag_set_fused(P, fused)
    phi = torch.empty(n[2], n[1], n[0], device="cuda")
    D.demag_apply_full(P, dev(m), phi, "bf16x3")  # prepares the tensor-core state
    D.demag_sync_status(P)
    D.demag_set_wait_limit(P, 0.0)
    D.demag_apply_full(P, dev(m), phi, "bf16x3")
    with pytest.raises(D.DemagError) as ei:
        D.demag_sync_status(P)
    assert ei.value.status == 4  # DEMAG_ETIMEOUT
    D.demag_set_wait_limit(P, 2.0)
    phi.fill_(float("nan"))
    D.demag_apply_full(P, dev(m), phi, "bf16x3")
    D.demag_sync_status(P)
    assert_close(host(phi), ofull.apply_full(m, n, h, R), TOL["bf16x3"])


def test_zero_wait_limit_in_a_batch_with_fused_grids(D):
    """The batched application (one fused mode-1 / mode-2 launch over two fused grids,
    then the persistent launch with their mode-3 stages and a chain grid's stages)
    with the first plan's limit at zero: the status on that plan says DEMAG_ETIMEOUT;
    with the limit restored the same batch gives the single calls' bits."""
    cases = [((64, 64, 20), True), ((48, 40, 37), False), ((37, 45, 33), True)]
    plans, ms, single = [], [], []
    for i, (n, fused) in enumerate(cases):
        P = D.demag_build_factors(n, (1 / max(n),) * 3, 21)
        D.demag_set_fused(P, fused)
        m = dev(synth.random_unit_m(n, 1240 + i))
        phi = torch.empty(n[2], n[1], n[0], device="cuda")
        D.demag_apply_full(P, m, phi, "bf16x3")
        plans.append(P)
        ms.append(m)
        single.append(phi)
    outs = [torch.empty_like(p) for p in single]
    D.demag_apply_full_batched(plans, ms, outs, "bf16x3")  # builds the grouped descriptors
    torch.cuda.synchronize()
    D.demag_sync_status(plans[0])
    D.demag_set_wait_limit(plans[0], 0.0)
    D.demag_apply_full_batched(plans, ms, outs, "bf16x3")
    with pytest.raises(D.DemagError) as ei:
        D.demag_sync_status(plans[0])
    assert ei.value.status == 4  # DEMAG_ETIMEOUT
    D.demag_set_wait_limit(plans[0], 2.0)
    for o in outs:
        o.fill_(float("nan"))
    D.demag_apply_full_batched(plans, ms, outs, "bf16x3")
    torch.cuda.synchronize()
    for P in plans:
        D.demag_sync_status(P)
    for got, want in zip(outs, single):
        assert torch.equal(got, want)


def test_wait_limit_is_validated(D):
    P = D.demag_build_factors((8, 8, 8), (1 / 8,) * 3, 11)
    for bad in (-1.0, 61.0, float("nan")):
        with pytest.raises(D.DemagError) as ei:
            D.demag_set_wait_limit(P, bad)
        assert ei.value.status == 1
