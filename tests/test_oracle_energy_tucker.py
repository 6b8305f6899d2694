"""Pins of the oracle's energy of a Tucker magnetization (oracle/energy.py: energy_tucker).

1. The structured route (Eq. kron_eval_tuck per node and component, then the
   second-order energy) gives the energy of the full-format route on the same
   dense magnetization.
2. Uniform magnetization of the unit cube, the case of the energy study after
   Alg. 2: the Tucker-route energy equals the energy of the closed-form exact
   collocation potential (charged-rectangle integrals), up to the sinc
   quadrature error, which vanishes as R grows.
3. The TT route (oracle/energy.py: energy_tt) gives the full-format energy of
   the formed TT magnetization.
"""
import numpy as np
import pytest

import synth
from oracle import energy as oe
from oracle import exact


def test_tucker_energy_equals_the_full_format_energy():
    n, ranks, h, R = (9, 7, 6), (2, 3, 2), (0.11, 0.11, 0.11), 21
    core, V = synth.tucker_inputs(n, ranks, 41)
    E = oe.energy_tucker(core, V, n, ranks, h, R)
    m = oe.tucker_magnetization(core, V, n, ranks)
    ref = oe.energy_from_m(m, n, h, R)
    assert abs(E - ref) <= 1e-12 * abs(ref)


@pytest.mark.parametrize("n", [16, 32])
def test_uniform_cube_energy_is_the_exact_collocation_energy(n):
    h = (1.0 / n,) * 3
    core = np.zeros((3, 1, 1, 1))
    core[2] = 1.0
    V = np.ones(3 * 3 * n)
    m = synth.uniform_m((n, n, n), 2).astype(np.float64)
    exact_E = oe.energy(m, exact.uniform_box_potential((n, n, n), h, 2), h)
    errs = [abs(oe.energy_tucker(core, V, (n, n, n), (1, 1, 1), h, R) - exact_E) / exact_E for R in (21, 41, 129)]
    assert errs[2] <= 1e-10
    assert errs[0] > errs[1] > errs[2] or errs[1] <= 1e-10
    # and the discretisation error itself, near 1/6 (the text after Fig. 2)
    assert abs(exact_E - 1.0 / 6.0) < 3e-3


def test_tt_energy_equals_the_full_format_energy():
    from oracle import structured as ost
    n, ranks, h, R = (8, 7, 6), (2, 3), (0.12, 0.12, 0.12), 21
    G1, G2, G3 = synth.tt_inputs(n, ranks, 42)
    E = oe.energy_tt(G1, G2, G3, n, ranks, h, R)
    m = np.stack([ost.tt_to_full(G1[q], G2[q], G3[q], ranks) for q in range(3)])
    ref = oe.energy_from_m(m, n, h, R)
    assert abs(E - ref) <= 1e-12 * abs(ref)


def test_fd_column_sums_match_the_stencil_matrix():
    for n, hp in ((1, 0.3), (2, 0.5), (3, 0.25), (7, 0.1), (40, 1 / 40)):
        assert np.allclose(oe.fd_column_sums(n, hp), oe.fd_matrix(n, hp).sum(axis=0), rtol=0, atol=1e-12 / hp)


@pytest.mark.parametrize("n,R", [(8, 21), (12, 41), (17, 129)])
def test_uniform_cube_energy_by_1d_sums_equals_the_tucker_route(n, R):
    """The factorised energy of the study's cube equals the dense Tucker route."""
    h = (1.0 / n,) * 3
    core = np.zeros((3, 1, 1, 1))
    core[2] = 1.0
    V = np.ones(3 * 3 * n)
    ref = oe.energy_tucker(core, V, (n, n, n), (1, 1, 1), h, R)
    assert abs(oe.uniform_cube_energy(n, R) - ref) <= 1e-12 * abs(ref)


def test_uniform_cube_energy_converges_to_one_sixth():
    """The text after Fig. 2: the relative energy error falls with n, at an order
    near 1.5 (R large enough that the quadrature error is far below it)."""
    import json
    import os
    facts = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_facts.json")))
    order = facts["energy_error_order"]["value"]
    E0 = facts["uniform_cube_energy"]["value"]
    errs = [abs(oe.uniform_cube_energy(n, 257) - E0) / E0 for n in (64, 128, 256, 512)]
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert all(abs(o - order) <= 0.3 for o in orders), orders
    assert errs[-1] < 1e-5
