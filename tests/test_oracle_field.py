"""Pins of the oracle's analytic stray field (oracle/field.py).

1. It is the derivative of the potential: the Kronecker potential evaluated at
   collocation points shifted by +-delta along one axis (cell integrals with
   shifted limits, written here from erf and exp directly) and differenced
   centrally agrees with -h_d.
2. It is the field of a uniformly magnetized box: central differences of the
   closed-form potential (charged-rectangle integrals) at the cell centres,
   up to the sinc-quadrature error.
3. -D phi with the second-order difference stencils converges to it at
   second order in h on a smooth magnetization.
"""
import numpy as np
import pytest
from scipy import special

import synth
from oracle import exact, field, full
from oracle import energy as En
from oracle.generators import scaled_spacing, toeplitz
from oracle.quadrature import sinc_nodes


def _shifted_potential(m, n, h, R, axis, delta, c0=2.15):
    """phi at the cell centres shifted by delta (scaled units) along `axis`."""
    M = (R - 1) // 2
    s, hh = scaled_spacing(n, h)
    _, _, tau, omega = sinc_nodes(M, c0)
    phi = np.zeros((n[2], n[1], n[0]))
    for k in range(M):
        t = tau[k]
        mats = {}
        for p in range(3):
            d = np.arange(-(n[p] - 1), n[p], dtype=np.float64)
            sh = delta if p == axis else 0.0
            a, b = (d - 0.5) * hh[p] + sh, (d + 0.5) * hh[p] + sh
            E = 0.5 * np.sqrt(np.pi) / t * (special.erf(t * b) - special.erf(t * a))
            F = (np.exp(-t * t * a * a) - np.exp(-t * t * b * b)) / (2.0 * t * t)
            mats[(p, "E")], mats[(p, "F")] = toeplitz(E, n[p]), toeplitz(F, n[p])
        for q in range(3):
            X = m[q]
            for p in range(3):
                X = full.mode_product(X, mats[(p, full.factor_kind(p, q))], p + 1)
            phi += omega[k] * X
    return full.C_POT * s * phi


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_field_is_the_derivative_of_the_potential(axis):
    n, h, R = (6, 5, 7), (0.11, 0.09, 0.13), 11
    rng = np.random.default_rng(3)
    m = rng.standard_normal((3, n[2], n[1], n[0]))
    s, hh = scaled_spacing(n, h)
    delta = 1e-4 * hh[axis]
    fd = (_shifted_potential(m, n, h, R, axis, delta) - _shifted_potential(m, n, h, R, axis, -delta)) / (
        2.0 * delta * s)
    hd = field.apply_field(m, n, h, R)
    assert np.max(np.abs(-fd - hd[axis])) < 1e-7 * np.max(np.abs(hd[axis]))


def _box_potential_at(n, h, q, shift):
    """Closed-form potential of the box magnetized along q at shifted cell centres."""
    L = [n[p] * h[p] for p in range(3)]
    c = [(np.arange(n[p]) + 0.5) * h[p] + shift[p] for p in range(3)]
    X3, X2, X1 = np.meshgrid(c[2], c[1], c[0], indexing="ij")
    X = (X1, X2, X3)
    u, v = [p for p in range(3) if p != q]
    top = exact.rect_integral(X[u] - L[u], X[u], X[v] - L[v], X[v], X[q] - L[q])
    bottom = exact.rect_integral(X[u] - L[u], X[u], X[v] - L[v], X[v], X[q])
    return (top - bottom) / (4.0 * np.pi)


@pytest.mark.parametrize("q", [0, 2])
def test_uniform_box_field_closed_form(q):
    n, h, R = (10, 8, 12), (0.1, 0.1, 0.1), 41
    m = synth.uniform_m(n, q).astype(np.float64)
    hd = field.apply_field(m, n, h, R)
    for p in range(3):
        d = 1e-6
        e = np.zeros(3)
        e[p] = d
        ref = -(_box_potential_at(n, h, q, e) - _box_potential_at(n, h, q, -e)) / (2.0 * d)
        assert np.max(np.abs(hd[p] - ref)) < 2e-4 * np.max(np.abs(ref)), (q, p)
    # inside a body magnetized along q the field points against m on average
    assert hd[q].mean() < 0


def test_finite_differences_converge_to_the_field_at_second_order():
    # -D phi (second-order stencils) differs from the analytic field by O(h^2)
    # in the interior of a smooth magnetization
    errs = []
    for nn in (10, 20):
        n, h = (nn, nn, nn), (1.0 / nn,) * 3
        m = synth.smooth_m(n).astype(np.float64)
        hd = field.apply_field(m, n, h, 21)
        fd = En.stray_field(full.apply_full(m, n, h, 21), h)
        c = nn // 5
        inner = (slice(None), slice(c, -c), slice(c, -c), slice(c, -c))
        errs.append(np.linalg.norm(hd[inner] - fd[inner]) / np.linalg.norm(hd[inner]))
    order = np.log2(errs[0] / errs[1])
    assert errs[1] < 1e-2 and 1.5 < order < 2.6, (errs, order)


def test_derivative_generators_parity():
    # dE is odd, dF even; dE = -2 tau^2 F by the closed form of F
    for tau in (0.3, 4.0, 60.0):
        dE = field.gen_dE(tau, 0.05, 9)
        dF = field.gen_dF(tau, 0.05, 9)
        assert np.allclose(dE, -dE[::-1], rtol=0, atol=1e-15)
        assert np.allclose(dF, dF[::-1], rtol=1e-13, atol=0)
        d = np.arange(-8, 9) * 0.05
        a, b = d - 0.025, d + 0.025
        direct = b * np.exp(-tau * tau * b * b) - a * np.exp(-tau * tau * a * a)
        assert np.allclose(dF, direct, rtol=1e-10, atol=1e-300)


def test_cube_demagnetizing_factor_one_third():
    # N_x + N_y + N_z = 1 and a cube is symmetric, so the volume average of the
    # field inside a uniformly magnetized cube is -m/3 along m and 0 across it
    n, h = (12, 12, 12), (1 / 12,) * 3
    for q in range(3):
        m = synth.uniform_m(n, q).astype(np.float64)
        hd = field.apply_field(m, n, h, 41)
        assert abs(hd[q].mean() + 1.0 / 3.0) < 1e-5
        for p in range(3):
            if p != q:
                assert abs(hd[p].mean()) < 1e-12


def test_field_operator_is_symmetric_so_the_energy_gradient_is_minus_v_h():
    # h_d = -A m with A symmetric (real, even Fourier kernels K_pq = K_qp): then
    # E = -1/2 V sum m . h_d has gradient -V h_d; checked by central differences
    n, h, R = (5, 4, 3), (0.2, 0.25, 0.3), 11
    rng = np.random.default_rng(21)
    a, b = rng.standard_normal((2, 3, n[2], n[1], n[0]))
    ha = field.apply_field(a, n, h, R)
    hb = field.apply_field(b, n, h, R)
    assert abs(np.sum(a * hb) - np.sum(b * ha)) <= 1e-12 * np.abs(np.sum(a * hb))
    V = h[0] * h[1] * h[2]

    def energy(m):
        return -0.5 * V * np.sum(m * field.apply_field(m, n, h, R))

    grad = -V * ha
    for _ in range(3):
        d = rng.standard_normal(a.shape)
        eps = 1e-4
        fd = (energy(a + eps * d) - energy(a - eps * d)) / (2 * eps)
        assert abs(fd - np.sum(grad * d)) <= 1e-8 * abs(fd)
