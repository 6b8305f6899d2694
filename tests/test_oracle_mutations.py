"""Plant plausible mistakes in the oracle (CPU only) and check that the
independent pins catch every one: a dropped term, a wrong sign, a transposed
operand, a wrong axis assignment and a wrong scale."""
import numpy as np
import pytest

import synth
from oracle import exact, full, generators, quadrature

N, H = (7, 5, 6), (2e-9, 3e-9, 2.5e-9)


def _kron_vs_exact_error(R=41):
    rng = np.random.default_rng(3)
    m = rng.standard_normal((3, N[2], N[1], N[0]))
    ref = exact.collocation_exact(m, N, H)
    got = full.apply_full(m, N, H, R)
    return np.linalg.norm(got - ref) / np.linalg.norm(ref)


def test_unmutated_is_accurate():
    assert _kron_vs_exact_error() < 1e-5


def _mutations():
    orig_F, orig_E = generators.gen_F, generators.gen_E
    orig_nodes, orig_kind = quadrature.sinc_nodes, full.factor_kind
    orig_mp, orig_scale = full.mode_product, generators.scaled_spacing

    def F_sign(tau, hh, n):
        return -orig_F(tau, hh, n)

    def E_half(tau, hh, n):  # dropped factor 1/2 on the off-centre cells
        e = orig_E(tau, hh, n)
        e[np.arange(e.size) != n - 1] *= 2.0
        return e

    def nodes_no_theta(M, c0=2.15):
        th, t, tau, om = orig_nodes(M, c0)
        return th, t, tau, om / th

    def kind_wrong_axis(p, q):
        return "F" if p == (q + 1) % 3 else "E"

    def mp_transposed(X, U, mode):
        return orig_mp(X, U.T, mode)

    def no_scaling(n, h):
        s, hh = orig_scale(n, h)
        return 1.0, hh

    return [
        ("gen_F", generators, F_sign),
        ("gen_E", generators, E_half),
        ("sinc_nodes", quadrature, nodes_no_theta),
        ("factor_kind", full, kind_wrong_axis),
        ("mode_product", full, mp_transposed),
        ("scaled_spacing", generators, no_scaling),
    ]


@pytest.mark.parametrize("name,mod,fn", _mutations(), ids=lambda x: x if isinstance(x, str) else "")
def test_mutation_is_caught(monkeypatch, name, mod, fn):
    monkeypatch.setattr(mod, name, fn)
    # modules that imported the symbol by name get the mutation too
    for other in (full,):
        if hasattr(other, name):
            monkeypatch.setattr(other, name, fn)
    assert _kron_vs_exact_error() > 1e-3


# ---- the analytic stray field (oracle/field.py): plant mistakes in its
# derivative generators and scale, and check that the closed-form box field
# or the derivative of the shifted potential catches each one
from oracle import field  # noqa: E402


def _field_pin_errors():
    import test_oracle_field as T
    errs = []
    n, h, R = (6, 5, 7), (0.11, 0.09, 0.13), 11
    rng = np.random.default_rng(3)
    m = rng.standard_normal((3, n[2], n[1], n[0]))
    s, hh = generators.scaled_spacing(n, h)
    for axis in range(3):
        d = 1e-4 * hh[axis]
        fd = (T._shifted_potential(m, n, h, R, axis, d) - T._shifted_potential(m, n, h, R, axis, -d)) / (2 * d * s)
        hd = field.apply_field(m, n, h, R)
        errs.append(np.max(np.abs(-fd - hd[axis])) / np.max(np.abs(hd[axis])))
    n, h = (10, 8, 12), (0.1, 0.1, 0.1)
    mu = synth.uniform_m(n, 2).astype(np.float64)
    hd = field.apply_field(mu, n, h, 41)
    for p in range(3):
        e = np.zeros(3)
        e[p] = 1e-6
        ref = -(T._box_potential_at(n, h, 2, e) - T._box_potential_at(n, h, 2, -e)) / 2e-6
        errs.append(np.max(np.abs(hd[p] - ref)) / np.max(np.abs(ref)))
    return max(errs)


def test_field_unmutated_is_accurate():
    assert _field_pin_errors() < 2e-4


def _field_mutations():
    orig_dE, orig_dF, orig_c = field.gen_dE, field.gen_dF, field.C_POT

    def dE_sign(tau, hh, n):
        return -orig_dE(tau, hh, n)

    def dF_one_face(tau, hh, n):  # only the upper cell face
        d = np.abs(np.arange(-(n - 1), n, dtype=np.float64))
        b = (d + 0.5) * hh
        return b * np.exp(-tau * tau * b * b)

    def dE_no_tau2(tau, hh, n):  # the factor 2 tau^2 dropped
        return orig_dE(tau, hh, n) / (2.0 * tau * tau)

    return [
        ("gen_dE", dE_sign),
        ("gen_dF", dF_one_face),
        ("gen_dE", dE_no_tau2),
        ("C_POT", orig_c * 1.2),  # the domain scale s = 1.2 of the box grid kept in the field
    ]


@pytest.mark.parametrize("name,fn", _field_mutations(), ids=lambda x: x if isinstance(x, str) else "")
def test_field_mutation_is_caught(monkeypatch, name, fn):
    monkeypatch.setattr(field, name, fn)
    assert _field_pin_errors() > 1e-3
