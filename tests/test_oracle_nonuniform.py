"""Pins of the oracle's operator on non-uniform tensor grids (oracle/nonuniform.py).

1. On uniform edges it is the uniform operator of oracle.full (to rounding).
2. On graded grids it matches the O(N^2) exact collocation sum (cell integrals of
   x_q/|x|^3 over boxes with the true, unequal cell limits) within the
   sinc-quadrature error, for random and for uniform magnetization.
3. Its transpose form is the transpose of the dense operator (unit vectors), and
   on a graded grid that transpose is not -P (the uniform-grid identity).
4. Plausible mistakes (collocation at a cell edge, F's sign, factor rows and
   columns swapped, F on the wrong axis) each break pin 2.
"""
import numpy as np
import pytest

from oracle import exact, full, nonuniform as nu


def _graded(n, length, ratio, rng=None):
    """n cells on [0, length] whose widths grow geometrically by `ratio` (plus jitter)."""
    w = ratio ** np.arange(n, dtype=np.float64)
    if rng is not None:
        w *= 1.0 + 0.3 * rng.random(n)
    return np.concatenate([[0.0], np.cumsum(w)]) * (length / w.sum())


def _brute(m, edges):
    """phi_i = (1/4pi) sum_q sum_j m_j^(q) int_{cell j} (xi_i - y)_q / |xi_i - y|^3 dy."""
    n = [len(e) - 1 for e in edges]
    xi = [0.5 * (e[:-1] + e[1:]) for e in edges]
    # all (i, j) pairs per axis: box of x = xi_i - y over cell j
    lo, hi = [], []
    for p in range(3):
        lo.append(xi[p][:, None] - edges[p][None, 1:])
        hi.append(xi[p][:, None] - edges[p][None, :-1])
    phi = np.zeros((n[2], n[1], n[0]))
    for q in range(3):
        # broadcast to [i3, i2, i1, j3, j2, j1]
        L = [lo[0][None, None, :, None, None, :], lo[1][None, :, None, None, :, None], lo[2][:, None, None, :, None, None]]
        H = [hi[0][None, None, :, None, None, :], hi[1][None, :, None, None, :, None], hi[2][:, None, None, :, None, None]]
        shape = (n[2], n[1], n[0], n[2], n[1], n[0])
        G = exact.box_G(q, [np.broadcast_to(x, shape) for x in L], [np.broadcast_to(x, shape) for x in H])
        phi += np.tensordot(G, m[q], axes=([3, 4, 5], [0, 1, 2]))
    return phi / (4.0 * np.pi)


def _edges():
    rng = np.random.default_rng(5)
    return [_graded(5, 1.0, 1.3, rng), _graded(4, 0.8, 0.7, rng), _graded(6, 1.2, 1.15, rng)]


def test_uniform_edges_reduce_to_the_uniform_operator():
    n, h = (6, 5, 4), (0.1, 0.15, 0.2)
    edges = [np.arange(n[p] + 1) * h[p] for p in range(3)]
    m = np.random.default_rng(1).standard_normal((3, n[2], n[1], n[0]))
    ref = full.apply_full(m, n, h, 21)
    got = nu.apply_full(m, edges, 21)
    assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)


@pytest.mark.parametrize("kind", ["random", "uniform"])
def test_graded_grid_matches_exact_collocation(kind):
    edges = _edges()
    n = [len(e) - 1 for e in edges]
    rng = np.random.default_rng(2)
    if kind == "random":
        m = rng.standard_normal((3, n[2], n[1], n[0]))
    else:
        m = np.zeros((3, n[2], n[1], n[0]))
        m[2] = 1.0
    ref = _brute(m, edges)
    got = nu.apply_full(m, edges, 41)
    assert np.linalg.norm(got - ref) < 2e-5 * np.linalg.norm(ref)


def test_transpose_is_the_dense_transpose():
    edges = [_graded(3, 1.0, 1.5), _graded(2, 0.5, 0.6), _graded(4, 0.9, 1.2)]
    n = [len(e) - 1 for e in edges]
    N = n[0] * n[1] * n[2]
    A = np.zeros((N, 3 * N))
    for col in range(3 * N):
        e = np.zeros(3 * N)
        e[col] = 1.0
        A[:, col] = nu.apply_full(e.reshape(3, n[2], n[1], n[0]), edges, 11).ravel()
    y = np.random.default_rng(4).standard_normal((n[2], n[1], n[0]))
    got = nu.apply_full(y, edges, 11, transpose=True)
    assert np.allclose(got.ravel(), A.T @ y.ravel(), rtol=0, atol=1e-13 * np.abs(A).max() * N)
    # on a graded grid the uniform identity P^T = -P fails
    neg = -np.stack([(A[:, q * N:(q + 1) * N]) @ y.ravel() for q in range(3)])
    assert np.linalg.norm(neg - got.reshape(3, -1)) > 1e-3 * np.linalg.norm(got)


def test_planted_mistakes_are_caught(monkeypatch):
    edges = _edges()
    n = [len(e) - 1 for e in edges]
    m = np.random.default_rng(2).standard_normal((3, n[2], n[1], n[0]))
    ref = _brute(m, edges)

    def err():
        got = nu.apply_full(m, edges, 41)
        return np.linalg.norm(got - ref) / np.linalg.norm(ref)

    assert err() < 2e-5
    orig_fm, orig_F, orig_kind = nu.factor_matrices, nu._F, nu.factor_kind

    def left_edge(edges_p, s, tau):  # collocation at the left cell edge
        y = np.asarray(edges_p, dtype=np.float64) / s
        xi = y[:-1] + 1e-3 * (y[1:] - y[:-1])
        a, b = xi[:, None] - y[None, 1:], xi[:, None] - y[None, :-1]
        return nu._E(tau, a, b), orig_F(tau, a, b)

    def swapped(edges_p, s, tau):
        E, F = orig_fm(edges_p, s, tau)
        return E.T, F.T

    for name, fn in [("factor_matrices", left_edge), ("factor_matrices", swapped),
                     ("_F", lambda tau, a, b: -orig_F(tau, a, b)),
                     ("factor_kind", lambda p, q: orig_kind(2 - p, q))]:
        with monkeypatch.context() as mp:
            mp.setattr(nu, name, fn)
            assert err() > 1e-3, name


def test_line_sampler_equals_the_full_application():
    edges = _edges()
    n = [len(e) - 1 for e in edges]
    m = np.random.default_rng(8).standard_normal((3, n[2], n[1], n[0]))
    full_phi = nu.apply_full(m, edges, 21)
    lines = [(0, 0), (5, 3), (2, 1)]
    got = nu.apply_full_lines(m, edges, 21, lines)
    for (i3, i2), row in zip(lines, got):
        assert np.allclose(row, full_phi[i3, i2], rtol=1e-13, atol=1e-15 * np.abs(full_phi).max())
