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
