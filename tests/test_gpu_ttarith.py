"""GPU parity of the TT conversions and Hadamard product of App. C (demag_tucker_to_tt,
demag_cp_to_tt, demag_tt_hadamard) against the oracle (oracle/ttround.py), through the C ABI."""
import numpy as np
import pytest

import synth
from oracle import structured as ost
from oracle import ttround as otr
from gpu_helpers import dev, host, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1212_3509_gb300 as D
    return D


def _blocks(flat, n, ranks):
    out, off = [], 0
    for q in range(3):
        row = []
        for p in range(3):
            size = ranks[p] * n[p]
            row.append(np.asarray(flat[off:off + size], dtype=np.float64).reshape(ranks[p], n[p]))
            off += size
        out.append(row)
    return out


def _empty_tt(n, r1, r2):
    return (torch.empty(3 * r1 * n[0], device="cuda"), torch.empty(3 * r1 * r2 * n[1], device="cuda"),
            torch.empty(3 * r2 * n[2], device="cuda"))


@pytest.mark.parametrize("n,ranks", [((12, 10, 8), (2, 3, 4)), ((1, 7, 33), (1, 1, 2))])
def test_tucker_to_tt(D, n, ranks):
    core, V = synth.tucker_inputs(n, ranks, 91)
    P = D.demag_build_factors(n, (1.0 / max(n),) * 3, 21)
    G = _empty_tt(n, ranks[0], ranks[2])
    D.demag_tucker_to_tt(P, ranks, dev(core.ravel()), dev(V), *G)
    torch.cuda.synchronize()
    Vb = _blocks(V, n, ranks)
    for q in range(3):
        ref = otr.tucker_to_tt(core[q], *Vb[q])
        for i, g in enumerate(G):
            got = host(g).astype(np.float64).reshape(3, -1)[q]
            assert rel_l2(got, ref[i].ravel()) <= 1e-6


def test_cp_to_tt(D):
    n, r = (9, 11, 6), 3
    lam, U = synth.cp_inputs(n, r, 92)
    lam = (lam * np.array([1.0, 0.5, -2.0], dtype=np.float32)).astype(np.float32)
    P = D.demag_build_factors(n, (1.0 / 11,) * 3, 21)
    G = _empty_tt(n, r, r)
    D.demag_cp_to_tt(P, r, dev(lam), dev(np.ascontiguousarray(U).ravel()), *G)
    torch.cuda.synchronize()
    Ub = _blocks(np.ascontiguousarray(U).ravel(), n, (r, r, r))
    for q in range(3):
        ref = otr.cp_to_tt(lam[q], *Ub[q])
        for i, g in enumerate(G):
            got = host(g).astype(np.float64).reshape(3, -1)[q]
            assert rel_l2(got, ref[i].ravel()) <= 1e-7


def test_hadamard_small_and_dense(D):
    n, ra, rb = (10, 7, 9), (2, 3), (3, 2)
    A = synth.tt_inputs(n, ra, 93)
    B = synth.tt_inputs(n, rb, 94)
    P = D.demag_build_factors(n, (0.1,) * 3, 21)
    C = _empty_tt(n, ra[0] * rb[0], ra[1] * rb[1])
    D.demag_tt_hadamard(P, ra, [dev(x) for x in A], rb, [dev(x) for x in B], C)
    torch.cuda.synchronize()
    for q in range(3):
        ref = otr.tt_hadamard([x[q] for x in A], ra, [x[q] for x in B], rb)
        got = [host(c).astype(np.float64).reshape(3, -1)[q] for c in C]
        for g, r_ in zip(got, ref):
            assert rel_l2(g, r_.ravel()) <= 1e-7
        dense = ost.tt_to_full(*[g.reshape(r_.shape) for g, r_ in zip(got, ref)], (ra[0] * rb[0], ra[1] * rb[1]))
        prod = ost.tt_to_full(*[x[q] for x in A], ra) * ost.tt_to_full(*[x[q] for x in B], rb)
        assert rel_l2(dense, prod) <= 1e-6


def test_tucker_to_tt_then_apply_matches_the_tucker_application(D):
    # App. C end to end: the TT form of a Tucker magnetization gives the same potential
    n, ranks, R = (14, 12, 10), (2, 2, 3), 21
    h = (1.0 / 14,) * 3
    core, V = synth.tucker_inputs(n, ranks, 95)
    P = D.demag_build_factors(n, h, R)
    G = _empty_tt(n, ranks[0], ranks[2])
    D.demag_tucker_to_tt(P, ranks, dev(core.ravel()), dev(V), *G)
    M, t = P.M, (ranks[0], ranks[2])
    w = torch.empty(M * 3, device="cuda")
    o = [torch.empty(M * 3 * s, device="cuda") for s in (t[0] * n[0], t[0] * t[1] * n[1], t[1] * n[2])]
    D.demag_apply_tt(P, t, *G, w, *o)
    torch.cuda.synchronize()
    phi_tt = ost.tt_output_to_full(host(w).astype(np.float64).reshape(M, 3),
                                   host(o[0]).astype(np.float64).reshape(M, 3, t[0], n[0]),
                                   host(o[1]).astype(np.float64).reshape(M, 3, t[0] * t[1], n[1]),
                                   host(o[2]).astype(np.float64).reshape(M, 3, t[1], n[2]), t)
    rw, rV = ost.apply_tucker(core, V, n, ranks, h, R)
    ref = ost.tucker_output_to_full(core.astype(np.float64), rw, rV)
    assert rel_l2(phi_tt, ref) <= 1e-5


def test_hadamard_1024_sampled(D):
    n, ra, rb = (1024, 1024, 1024), (8, 8), (8, 8)
    A = synth.tt_inputs(n, ra, 96)
    B = synth.tt_inputs(n, rb, 97)
    P = D.demag_build_factors(n, (1.0 / 1024,) * 3, 21)
    C = _empty_tt(n, 64, 64)
    D.demag_tt_hadamard(P, ra, [dev(x) for x in A], rb, [dev(x) for x in B], C)
    torch.cuda.synchronize()
    C1 = host(C[0]).astype(np.float64).reshape(3, 64, 1024)
    C2 = host(C[1]).astype(np.float64).reshape(3, 64, 64, 1024)
    C3 = host(C[2]).astype(np.float64).reshape(3, 64, 1024)
    A64 = [x.astype(np.float64) for x in A]
    B64 = [x.astype(np.float64) for x in B]
    pts = np.random.default_rng(3).integers(0, 1024, size=(32, 3))
    for q in range(3):
        for i1, i2, i3 in pts:
            got = C1[q, :, i1] @ C2[q, :, :, i2] @ C3[q, :, i3]
            scale = np.abs(C1[q, :, i1]) @ np.abs(C2[q, :, :, i2]) @ np.abs(C3[q, :, i3])
            a = A64[0][q][:, i1] @ A64[1][q].reshape(8, 8, 1024)[:, :, i2] @ A64[2][q][:, i3]
            b = B64[0][q][:, i1] @ B64[1][q].reshape(8, 8, 1024)[:, :, i2] @ B64[2][q][:, i3]
            assert abs(got - a * b) <= 1e-6 * scale
