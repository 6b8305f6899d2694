"""Parity at the full sizes of the benchmark configurations, in the launch
configuration bench.py times (sampled outputs where the oracle cannot do all).

C2: full format 256^3 (sampled output lines) and 128^3 (every output), R = 41,
    vortex state + 5% noise, every form.
C3: CP n = 4096, rank 4 per component, R = 61, batched launch; the first and
    last batch items compared element by element.
C4: Tucker n = 1024 ranks (8,8,8) and TT n = 1024 ranks (8,8), R = 61.
C5: mixed grid shapes (cubes and thin films) with random unit m in one
    batched call (BF16x3), and the energy gradient at 16^3 against central
    finite differences of the FP64 oracle energy (step 1e-4).
"""
import numpy as np
import pytest

import synth
from oracle import energy as oen
from oracle import full as ofull
from oracle import structured as ost
from gpu_helpers import assert_close, TOL, dev, host, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1212_3509_gb300 as D
    return D


def _lines(n3):
    n = n3[0]
    return [(0, 0), (n // 2, n // 3), (n - 1, n - 1), (n // 4, n - 7), (7, 1)]


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3", "fp32"])
def test_c2_full_256_sampled_lines(D, prec):
    n3, h, R = (256, 256, 256), (1 / 256,) * 3, 41
    m = synth.vortex_m(n3, 1213)
    P = D.demag_build_factors(n3, h, R)
    phi = torch.empty(256, 256, 256, device="cuda")
    D.demag_apply_full(P, dev(m), phi, prec)
    torch.cuda.synchronize()
    D.demag_sync_status(P)
    lines = _lines(n3)
    ref = ofull.apply_full_lines(m, n3, h, R, lines)
    got = host(phi)
    err = rel_l2(np.stack([got[i3, i2] for i3, i2 in lines]), ref)
    print(f"C2 256^3 {prec}: sampled rel L2 {err:.3e}")
    assert_close(np.stack([got[i3, i2] for i3, i2 in lines]), ref, TOL[prec])


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3", "fp32", "fp64"])
def test_c2_full_128_every_output(D, prec):
    n3, h, R = (128, 128, 128), (1 / 128,) * 3, 41
    m = synth.vortex_m(n3, 1213)
    P = D.demag_build_factors(n3, h, R)
    phi = torch.empty(128, 128, 128, device="cuda")
    D.demag_apply_full(P, dev(m), phi, prec)
    torch.cuda.synchronize()
    ref_ = ofull.apply_full(m, n3, h, R)
    err = rel_l2(host(phi), ref_)
    print(f"C2 128^3 {prec}: rel L2 {err:.3e}")
    assert_close(host(phi), ref_, TOL[prec])


def test_c3_cp_4096_batched(D):
    n, r, R, B = 4096, 4, 61, 6
    n3, h = (n, n, n), (1 / n,) * 3
    P = D.demag_build_factors(n3, h, R)
    M = P.M
    lam = np.empty((B, 3, r), dtype=np.float32)
    U = np.empty((B, 9 * r * n), dtype=np.float32)
    for b in range(B):
        lam[b], u = synth.cp_inputs(n3, r, 1214 + b)
        U[b] = u.ravel()
    w = torch.empty(B * M * 3 * r, device="cuda")
    oU = torch.empty(B * M * 3 * r * 3 * n, device="cuda")
    D.demag_apply_cp_batched(P, B, r, dev(lam), dev(U), w, oU)
    torch.cuda.synchronize()
    per = M * 3 * r * 3 * n
    for b in (0, B - 1):
        rw, rU = ost.apply_cp(lam[b], U[b], n3, h, R)
        ref = np.concatenate([rU[p].ravel() for p in range(3)])
        err = rel_l2(host(oU[b * per:(b + 1) * per]), ref)
        print(f"C3 CP n=4096 item {b}: rel L2 {err:.3e}")
        assert_close(host(oU[b * per:(b + 1) * per]), ref, TOL["fp32"])
        assert rel_l2(host(w[b * M * 3 * r:(b + 1) * M * 3 * r]), rw.ravel()) < 1e-6


def test_c4_tucker_1024(D):
    n3, h, R, ranks = (1024,) * 3, (1 / 1024,) * 3, 61, (8, 8, 8)
    core, V = synth.tucker_inputs(n3, ranks, 1215)
    P = D.demag_build_factors(n3, h, R)
    M = P.M
    tot = sum(ranks[p] * n3[p] for p in range(3))
    w = torch.empty(M * 3, device="cuda")
    oV = torch.empty(M * 3 * tot, device="cuda")
    D.demag_apply_tucker(P, ranks, dev(V), w, oV)
    torch.cuda.synchronize()
    rw, rV = ost.apply_tucker(core, V, n3, ranks, h, R)
    ref_ = np.concatenate([rV[p].ravel() for p in range(3)])
    err = rel_l2(host(oV), ref_)
    print(f"C4 Tucker n=1024: rel L2 {err:.3e}")
    assert_close(host(oV), ref_, TOL["fp32"])


def test_c4_tt_1024(D):
    n3, h, R, ranks = (1024,) * 3, (1 / 1024,) * 3, 61, (8, 8)
    G1, G2, G3 = synth.tt_inputs(n3, ranks, 1216)
    P = D.demag_build_factors(n3, h, R)
    M = P.M
    w = torch.empty(M * 3, device="cuda")
    o1 = torch.empty(M * 3 * 8 * 1024, device="cuda")
    o2 = torch.empty(M * 3 * 64 * 1024, device="cuda")
    o3 = torch.empty(M * 3 * 8 * 1024, device="cuda")
    D.demag_apply_tt(P, ranks, dev(G1), dev(G2), dev(G3), w, o1, o2, o3)
    torch.cuda.synchronize()
    rw, r1, r2, r3 = ost.apply_tt(G1, G2, G3, n3, ranks, h, R)
    for got, ref in ((o1, r1), (o2, r2), (o3, r3)):
        ref_ = ref.ravel()
        err = rel_l2(host(got), ref_)
        print(f"C4 TT n=1024: rel L2 {err:.3e}")
        assert_close(host(got), ref_, TOL["fp32"])


def test_c5_mixed_grids_batched(D):
    # every shape of the 64-grid uneven workload (cubes 32^3..192^3 in steps of
    # 16 and both films), in one batched call: one persistent launch runs all
    # stages of all grids; large grids are checked on sampled output lines
    shapes = sorted(set(synth.uneven_batch_shapes(64, 1215)), key=lambda s: s[0] * s[1] * s[2])
    assert len(shapes) >= 13 and (512, 512, 4) in shapes and (256, 64, 8) in shapes
    plans, ms, phis = [], [], []
    for i, n3 in enumerate(shapes):
        h = (1.0 / max(n3),) * 3
        P = D.demag_build_factors(n3, h, 41)
        D.demag_reserve_workspace(P, "bf16x3")
        plans.append(P)
        ms.append(synth.random_unit_m(n3, 1217 + i))
        phis.append(torch.empty(n3[2], n3[1], n3[0], device="cuda"))
    D.demag_apply_full_batched(plans, [dev(m) for m in ms], phis, "bf16x3")
    torch.cuda.synchronize()
    for P, m, phi, n3 in zip(plans, ms, phis, shapes):
        h = (1.0 / max(n3),) * 3
        if P.N <= 100_000:
            ref, got = ofull.apply_full(m, n3, h, 41), host(phi)
        else:
            lines = [(0, 0), (n3[2] - 1, n3[1] // 2), (n3[2] // 2, n3[1] - 1)]
            ref = ofull.apply_full_lines(m, n3, h, 41, lines)
            g = host(phi)
            got = np.stack([g[i3, i2] for i3, i2 in lines])
        err = rel_l2(got, ref)
        print(f"C5 {n3} bf16x3: rel L2 {err:.3e}")
        assert_close(got, ref, TOL["bf16x3"])


def test_c5_gradient_vs_fp64_finite_differences(D):
    n3, h, R = (16, 16, 16), (1 / 16,) * 3, 41
    m = synth.random_unit_m(n3, 1218)
    P = D.demag_build_factors(n3, h, R)
    E = torch.empty((), dtype=torch.float64, device="cuda")
    grad = torch.empty(3, 16, 16, 16, device="cuda")
    D.demag_energy(P, dev(m), E, grad, "fp32")
    torch.cuda.synchronize()
    g = host(grad)
    m64 = m.astype(np.float64)
    rng = np.random.default_rng(5)
    eps = 1e-4
    # E is quadratic in m, so the central difference is exact up to FP64 rounding;
    # the FP32 gradient is compared relative to the gradient's scale.
    gscale = np.abs(g).max()
    errs = []
    for _ in range(6):
        idx = (rng.integers(3), rng.integers(16), rng.integers(16), rng.integers(16))
        mp, mm = m64.copy(), m64.copy()
        mp[idx] += eps
        mm[idx] -= eps
        fd = (oen.energy_from_m(mp, n3, h, R) - oen.energy_from_m(mm, n3, h, R)) / (2 * eps)
        errs.append(abs(g[idx] - fd) / gscale)
    v = rng.standard_normal(m.shape)
    fd = (oen.energy_from_m(m64 + eps * v, n3, h, R) - oen.energy_from_m(m64 - eps * v, n3, h, R)) / (2 * eps)
    dir_err = abs((g * v).sum() - fd) / abs(fd)
    print(f"C5 gradient vs FD: max pointwise err / max|g| {max(errs):.2e}, directional rel {dir_err:.2e}")
    assert max(errs) < 1e-5 and dir_err < 1e-5
    assert float(E) == pytest.approx(oen.energy_from_m(m64, n3, h, R), rel=1e-5)


def test_c4_batched_and_graph_captured(D):
    """C4 as a batch: Tucker and TT items in one launch equal single applies,
    and the batched calls replay from a captured CUDA graph."""
    n3, h, R = (1024,) * 3, (1 / 1024,) * 3, 61
    P = D.demag_build_factors(n3, h, R)
    M, B = P.M, 3
    rt, rr = (8, 8, 8), (8, 8)
    tot = sum(rt[p] * 1024 for p in range(3))
    V = torch.cat([dev(synth.tucker_inputs(n3, rt, 1300 + b)[1].ravel()) for b in range(B)])
    wB = torch.empty(B * M * 3, device="cuda")
    oB = torch.empty(B * M * 3 * tot, device="cuda")
    tts = [synth.tt_inputs(n3, rr, 1400 + b) for b in range(B)]
    G = [torch.cat([dev(t[i].ravel()) for t in tts]) for i in range(3)]
    sizes = [8 * 1024, 64 * 1024, 8 * 1024]
    tw = torch.empty(B * M * 3, device="cuda")
    tO = [torch.empty(B * M * 3 * s, device="cuda") for s in sizes]

    def run():
        D.demag_apply_tucker_batched(P, B, rt, V, wB, oB)
        D.demag_apply_tt_batched(P, B, rr, G[0], G[1], G[2], tw, *tO)

    run()
    torch.cuda.synchronize()
    for b in range(B):
        w1 = torch.empty(M * 3, device="cuda")
        o1 = torch.empty(M * 3 * tot, device="cuda")
        D.demag_apply_tucker(P, rt, V[b * 3 * tot:(b + 1) * 3 * tot], w1, o1)
        t1 = [torch.empty(M * 3 * s, device="cuda") for s in sizes]
        D.demag_apply_tt(P, rr, *[G[i][b * 3 * sizes[i]:(b + 1) * 3 * sizes[i]] for i in range(3)], w1, *t1)
        torch.cuda.synchronize()
        assert torch.equal(oB[b * M * 3 * tot:(b + 1) * M * 3 * tot], o1)
        for i in range(3):
            assert torch.equal(tO[i][b * M * 3 * sizes[i]:(b + 1) * M * 3 * sizes[i]], t1[i])
    ref = [oB.clone()] + [t.clone() for t in tO]
    oB.fill_(float("nan"))
    for t in tO:
        t.fill_(float("nan"))
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            run()
    torch.cuda.current_stream().wait_stream(s)
    g.replay()
    torch.cuda.synchronize()
    for got, want in zip([oB] + tO, ref):
        assert torch.equal(got, want)
    # spot check against the oracle: first Tucker item
    core, Vh = synth.tucker_inputs(n3, rt, 1300)
    rw, rV = ost.apply_tucker(core, Vh, n3, rt, h, R)
    assert_close(host(oB[:M * 3 * tot]), np.concatenate([rV[p].ravel() for p in range(3)]), TOL["fp32"])
