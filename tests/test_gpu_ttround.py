"""GPU parity of the TT rounding of the potential (demag_round_tt, App. C) against
the oracle's dense TT-SVD (oracle/ttround.py), through the C ABI."""
import numpy as np
import pytest

import synth
from oracle import structured as ost
from oracle import ttround
from gpu_helpers import dev, host, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1212_3509_gb300 as D
    return D


def _apply(D, P, n, ranks, G1, G2, G3):
    M = P.M
    r1, r2 = ranks
    w = torch.empty(M * 3, device="cuda")
    o1 = torch.empty(M * 3 * r1 * n[0], device="cuda")
    o2 = torch.empty(M * 3 * r1 * r2 * n[1], device="cuda")
    o3 = torch.empty(M * 3 * r2 * n[2], device="cuda")
    D.demag_apply_tt(P, ranks, dev(G1), dev(G2), dev(G3), w, o1, o2, o3)
    torch.cuda.synchronize()
    return w, o1, o2, o3


def _dense_of(P, n, ranks, w, o1, o2, o3):
    M = P.M
    r1, r2 = ranks
    return ost.tt_output_to_full(host(w).astype(np.float64).reshape(M, 3),
                                 host(o1).astype(np.float64).reshape(M, 3, r1, n[0]),
                                 host(o2).astype(np.float64).reshape(M, 3, r1 * r2, n[1]),
                                 host(o3).astype(np.float64).reshape(M, 3, r2, n[2]), ranks)


CASES = [
    # (n, TT ranks, R, tol, smooth inputs)
    ((14, 12, 10), (3, 3), 21, 1e-3, False),   # full ranks: exact after the first samples
    ((24, 20, 16), (2, 3), 21, 1e-4, True),
    ((40, 36, 32), (2, 3), 21, 1e-4, False),   # needs 64 samples on the first unfolding
    ((64, 64, 64), (2, 2), 41, 1e-6, True),
    ((33, 17, 5), (1, 1), 21, 1e-5, True),     # rank-1 input, odd sizes, thin third axis
    ((1, 9, 7), (1, 2), 21, 1e-4, True),       # a single cell along the first axis
]


@pytest.mark.parametrize("n,ranks,R,tol,smooth", CASES)
def test_round_vs_oracle(D, n, ranks, R, tol, smooth):
    h = (1.0 / max(n),) * 3
    gen = synth.tt_smooth_inputs if smooth else synth.tt_inputs
    G1, G2, G3 = gen(n, ranks, 5)
    P = D.demag_build_factors(n, h, R)
    w, o1, o2, o3 = _apply(D, P, n, ranks, G1, G2, G3)
    phi = _dense_of(P, n, ranks, w, o1, o2, o3)
    (q1, q2), T1, T2, T3, err = D.demag_round_tt(P, ranks, w, o1, o2, o3, tol)
    T1h, T2h, T3h = (host(x).astype(np.float64) for x in (T1, T2, T3))
    approx = ost.tt_to_full(T1h, T2h, T3h, (q1, q2))
    true = rel_l2(approx, phi)
    # the bound, and the reported error is the error reached (FP32 outputs add ~1e-7)
    assert true <= tol * 1.001 + 2e-7, (true, tol)
    assert err <= tol
    assert abs(true - err) <= 0.01 * tol + 2e-7, (true, err)
    # left-orthonormal cores: G1 rows, and G2 as the [(a1 i2), a2] matrix
    assert np.allclose(T1h @ T1h.T, np.eye(q1), atol=1e-5)
    L = T2h.reshape(q1, q2, n[1]).transpose(0, 2, 1).reshape(q1 * n[1], q2)
    assert np.allclose(L.T @ L, np.eye(q2), atol=1e-5)
    # ranks: those of the oracle's TT-SVD (the sketch and the budget split may cost one or two)
    _, _, _, ref = ttround.tt_round_dense(phi, tol)
    assert all(ref[i] <= (q1, q2)[i] <= ref[i] + 2 for i in range(2)), ((q1, q2), ref)


def test_round_1024(D):
    # the full-size TT workload (1024^3, R = 61): the rounded train against the 3M input
    # trains at sampled points
    n, ranks, R, tol = (1024, 1024, 1024), (2, 2), 61, 1e-5
    G1, G2, G3 = synth.tt_smooth_inputs(n, ranks, 9)
    P = D.demag_build_factors(n, (1.0 / 1024,) * 3, R)
    w, o1, o2, o3 = _apply(D, P, n, ranks, G1, G2, G3)
    (q1, q2), T1, T2, T3, err = D.demag_round_tt(P, ranks, w, o1, o2, o3, tol)
    assert err <= tol and max(q1, q2) <= 64
    M = P.M
    r1, r2 = ranks
    wh = host(w).astype(np.float64).reshape(3 * M)
    A = host(o1).astype(np.float64).reshape(3 * M, r1, 1024)
    B = host(o2).astype(np.float64).reshape(3 * M, r1, r2, 1024)
    C = host(o3).astype(np.float64).reshape(3 * M, r2, 1024)
    T1h = host(T1).astype(np.float64)
    T2h = host(T2).astype(np.float64).reshape(q1, q2, 1024)
    T3h = host(T3).astype(np.float64)
    pts = np.random.default_rng(2).integers(0, 1024, size=(64, 3))
    num = den = 0.0
    for i1, i2, i3 in pts:
        a = float(np.einsum("t,ta,tab,tb->", wh, A[:, :, i1], B[:, :, :, i2], C[:, :, i3]))
        b = float(T1h[:, i1] @ T2h[:, :, i2] @ T3h[:, i3])
        num += (a - b) ** 2
        den += a ** 2
    assert (num / den) ** 0.5 <= 10 * tol


def test_round_rejects_zero_potential_and_bad_tol(D):
    n, ranks = (12, 10, 8), (2, 2)
    P = D.demag_build_factors(n, (1.0 / 12,) * 3, 21)
    zeros = [np.zeros_like(x) for x in synth.tt_inputs(n, ranks, 1)]
    w, o1, o2, o3 = _apply(D, P, n, ranks, *zeros)
    with pytest.raises(RuntimeError, match="zero"):
        D.demag_round_tt(P, ranks, w, o1, o2, o3, 1e-4)
    G1, G2, G3 = synth.tt_inputs(n, ranks, 1)
    w, o1, o2, o3 = _apply(D, P, n, ranks, G1, G2, G3)
    for bad in (0.0, 1.0, -1e-3):
        with pytest.raises(RuntimeError, match="tol"):
            D.demag_round_tt(P, ranks, w, o1, o2, o3, bad)
