"""Pins of the oracle's sinc quadrature and 1D generators against closed forms,
high-precision arithmetic and independent numerical integration."""
import json
import os

import numpy as np
import pytest
from scipy import integrate

from oracle import quadrature as Q
from oracle import generators as G

FACTS = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_facts.json")))
C0 = FACTS["sinc_c0"]["value"]


def test_gauss_transform_identity_exact():
    # Eq. gauss_trans, checked by numerical integration (no sinc rule involved).
    for rho in [1e-3, 0.1, 1.0, 3.0]:
        val, _ = integrate.quad(lambda t: t * t * np.exp(-t * t * rho), -np.inf, np.inf)
        assert abs(2 / np.sqrt(np.pi) * val * rho ** 1.5 - 1) < 1e-10


def test_nodes_definition():
    theta, t, tau, om = Q.sinc_nodes(20, C0)
    assert theta == pytest.approx(C0 * np.log(20) / 20, rel=1e-15)
    assert np.allclose(t, theta * np.arange(1, 21), rtol=1e-15)
    # the folded weight equals the two symmetric trapezoid weights theta*cosh*sinh^2
    assert np.allclose(om, 2 * theta * np.cosh(t) * np.sinh(t) ** 2, rtol=1e-14)
    with pytest.raises(ValueError):
        Q.sinc_nodes(1)


def test_folded_rule_equals_symmetric_trapezoid():
    # sum_{k=-M..M} theta * cosh(t_k) sinh(t_k)^2 e^{-sinh^2 rho} equals the folded sum
    M, rho = 12, 0.37
    theta = C0 * np.log(M) / M
    k = np.arange(-M, M + 1)
    t = k * theta
    sym = theta * (np.cosh(t) * np.sinh(t) ** 2 * np.exp(-np.sinh(t) ** 2 * rho)).sum()
    _, _, tau, om = Q.sinc_nodes(M, C0)
    assert sym == pytest.approx((om * np.exp(-tau ** 2 * rho)).sum(), rel=1e-14)


def test_quadrature_error_decays_exponentially_in_rank():
    # Thm. 1 / Fig. 1: log of the max relative error on [3h^2/4, 3] is a
    # decreasing (roughly affine) function of the rank, for fixed h.
    rho_min = FACTS["rho_min_factor"]["value"] * (1 / 16) ** 2
    Ms = np.arange(8, 41, 4)
    errs = np.array([Q.max_rel_error(int(M), rho_min, 3.0, C0) for M in Ms])
    assert np.all(np.diff(np.log(errs)) < 0)
    slope, icpt = np.polyfit(Ms, np.log(errs), 1)
    resid = np.log(errs) - (slope * Ms + icpt)
    assert slope < -0.3
    assert np.max(np.abs(resid)) < 1.0
    assert errs[-1] < 1e-8


def test_quadrature_not_uniform_in_h():
    # Remark after Lemma 2: for fixed rank the error grows as h -> 0.
    e = [Q.max_rel_error(20, 0.75 * hh ** 2, 3.0, C0) for hh in (1 / 16, 1 / 256, 1 / 1024)]
    assert e[0] < e[1] < e[2]


# ---------------------------------------------------------------- generators

def _E_quad(d, tau, hh):
    a, b = (d - 0.5) * hh, (d + 0.5) * hh
    return integrate.quad(lambda x: np.exp(-tau * tau * x * x), a, b, epsabs=0, epsrel=1e-13, limit=200)[0]


def _F_quad(d, tau, hh):
    a, b = (d - 0.5) * hh, (d + 0.5) * hh
    return integrate.quad(lambda x: x * np.exp(-tau * tau * x * x), a, b, epsabs=0, epsrel=1e-13, limit=200)[0]


@pytest.mark.parametrize("hh", [1 / 16, 1 / 256])
def test_generators_vs_numerical_integration(hh):
    # Eq. sep_integrands integrated numerically, independent of the erf forms.
    _, _, tau, _ = Q.sinc_nodes(20, C0)
    n = 40
    for k in (0, 7, 19):
        E = G.gen_E(tau[k], hh, n)
        F = G.gen_F(tau[k], hh, n)
        for d in (-39, -5, -1, 0, 1, 2, 9, 39):
            e = _E_quad(d, tau[k], hh)
            f = _F_quad(d, tau[k], hh)
            assert abs(E[d + n - 1] - e) <= 1e-10 * abs(e) + 1e-300
            assert abs(F[d + n - 1] - f) <= 1e-10 * abs(f) + 1e-300


def test_generators_vs_high_precision():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    _, _, tau, _ = Q.sinc_nodes(30, C0)
    worst = 0.0
    for k in (0, 5, 15, 29):
        for hh in (1 / 16, 1 / 256, 1 / 4096):
            n = 64
            E = G.gen_E(tau[k], hh, n)
            F = G.gen_F(tau[k], hh, n)
            for d in (-63, -10, -1, 0, 1, 2, 7, 30, 63):
                T = mp.mpf(float(tau[k]))
                a = mp.mpf(d) * hh - mp.mpf(hh) / 2
                b = a + hh
                e = float(mp.sqrt(mp.pi) / (2 * T) * (mp.erf(T * b) - mp.erf(T * a)))
                f = float((mp.exp(-T * T * a * a) - mp.exp(-T * T * b * b)) / (2 * T * T))
                if e > 1e-290:
                    worst = max(worst, abs(E[d + n - 1] - e) / e)
                if abs(f) > 1e-290:
                    worst = max(worst, abs(F[d + n - 1] - f) / abs(f))
    assert worst < 1e-11


def test_generator_symmetries_and_telescoping():
    _, _, tau, _ = Q.sinc_nodes(20, C0)
    n, hh = 100, 1 / 100
    for k in range(20):
        E = G.gen_E(tau[k], hh, n)
        F = G.gen_F(tau[k], hh, n)
        assert np.array_equal(E, E[::-1])  # even
        assert np.array_equal(F, -F[::-1])  # odd
        assert F[n - 1] == 0.0  # self term vanishes
        # telescoping: the cells tile [-(n-1/2)h, (n-1/2)h]
        tot = np.sqrt(np.pi) / tau[k] * __import__("scipy").special.erf(tau[k] * (n - 0.5) * hh)
        assert E.sum() == pytest.approx(tot, rel=1e-12)
        right = (np.exp(-tau[k] ** 2 * (hh / 2) ** 2) - np.exp(-tau[k] ** 2 * ((n - 0.5) * hh) ** 2)) / (2 * tau[k] ** 2)
        assert F[n:].sum() == pytest.approx(right, rel=1e-12)


def test_scaled_spacing():
    s, hh = G.scaled_spacing((64, 32, 4), (1e-9, 2e-9, 3e-9))
    assert s == pytest.approx(6.4e-8)
    assert np.allclose(hh, np.array([1e-9, 2e-9, 3e-9]) / 6.4e-8)


def test_toeplitz_layout():
    gen = np.arange(-3, 4, dtype=float)  # d = -3..3 for n = 4
    T = G.toeplitz(gen, 4)
    assert T[2, 0] == 2 and T[0, 2] == -2 and T[3, 0] == 3 and T[1, 1] == 0
