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


# ---- App. C TT arithmetic and the structured energies: plant mistakes and check that the
# dense comparisons of their pins catch each one
from oracle import energy as oen  # noqa: E402
from oracle import structured as ost  # noqa: E402
from oracle import ttround  # noqa: E402


def _tt_pin_errors():
    rng = np.random.default_rng(9)
    errs = []
    r, n = (2, 3, 4), (7, 6, 5)
    C = rng.standard_normal((r[2], r[1], r[0]))
    V = [rng.standard_normal((r[p], n[p])) for p in range(3)]
    G = ttround.tucker_to_tt(C, *V)
    ref = ost.tucker_to_full(C, V)
    errs.append(np.linalg.norm(ost.tt_to_full(*G, (r[0], r[2])) - ref) / np.linalg.norm(ref))
    lam = rng.standard_normal(3) + 2.0
    U = [rng.standard_normal((3, n[p])) for p in range(3)]
    G = ttround.cp_to_tt(lam, *U)
    ref = np.einsum("l,li,lj,lk->kji", lam, U[0], U[1], U[2])
    errs.append(np.linalg.norm(ost.tt_to_full(*G, (3, 3)) - ref) / np.linalg.norm(ref))
    ra, rb = (2, 3), (3, 2)
    A = (rng.standard_normal((2, n[0])), rng.standard_normal((6, n[1])), rng.standard_normal((3, n[2])))
    B = (rng.standard_normal((3, n[0])), rng.standard_normal((6, n[1])), rng.standard_normal((2, n[2])))
    Cc = ttround.tt_hadamard(A, ra, B, rb)
    ref = ost.tt_to_full(*A, ra) * ost.tt_to_full(*B, rb)
    errs.append(np.linalg.norm(ost.tt_to_full(*Cc, (6, 6)) - ref) / np.linalg.norm(ref))
    return max(errs)


def _energy_pin_error():
    n, ranks, h, R = (6, 5, 4), (2, 2, 1), (0.15, 0.15, 0.15), 11
    core, V = synth.tucker_inputs(n, ranks, 43)
    E = oen.energy_tucker(core, V, n, ranks, h, R)
    ref = oen.energy_from_m(oen.tucker_magnetization(core, V, n, ranks), n, h, R)
    errs = [abs(E - ref) / abs(ref)]
    G1, G2, G3 = synth.tt_inputs(n, (2, 2), 44)
    E = oen.energy_tt(G1, G2, G3, n, (2, 2), h, R)
    m = np.stack([ost.tt_to_full(G1[q], G2[q], G3[q], (2, 2)) for q in range(3)])
    ref = oen.energy_from_m(m, n, h, R)
    errs.append(abs(E - ref) / abs(ref))
    return max(errs)


def test_tt_and_energy_unmutated_are_exact():
    assert _tt_pin_errors() < 1e-12
    assert _energy_pin_error() < 1e-12


def _tt_mutations():
    orig_t2t, orig_c2t, orig_had = ttround.tucker_to_tt, ttround.cp_to_tt, ttround.tt_hadamard

    def t2t_rows_swapped(core, V1, V2, V3):  # middle-core rows (a3, a1) instead of (a1, a3)
        G1, G2, G3 = orig_t2t(core, V1, V2, V3)
        r1, r3 = G1.shape[0], G3.shape[0]
        return G1, G2.reshape(r1, r3, -1).transpose(1, 0, 2).reshape(r1 * r3, -1), G3

    def c2t_no_lambda(lam, U1, U2, U3):
        return orig_c2t(np.ones_like(np.asarray(lam, dtype=np.float64)), U1, U2, U3)

    def had_first_core_b_major(A, ra, B, rb):  # Kronecker order of the first core flipped
        C1, C2, C3 = orig_had(A, ra, B, rb)
        n1 = C1.shape[1]
        return C1.reshape(ra[0], rb[0], n1).transpose(1, 0, 2).reshape(-1, n1), C2, C3

    return [("tucker_to_tt", t2t_rows_swapped), ("cp_to_tt", c2t_no_lambda), ("tt_hadamard", had_first_core_b_major)]


@pytest.mark.parametrize("name,fn", _tt_mutations(), ids=lambda x: x if isinstance(x, str) else "")
def test_tt_mutation_is_caught(monkeypatch, name, fn):
    monkeypatch.setattr(ttround, name, fn)
    assert _tt_pin_errors() > 1e-3


def _energy_mutations():
    orig_apply_tucker, orig_apply_tt = ost.apply_tucker, ost.apply_tt

    def tucker_wrong_component(core, V, n, ranks, h, R, c0=2.15):  # outputs of component q + 1 for q
        w, outV = orig_apply_tucker(core, V, n, ranks, h, R, c0)
        return w, [np.roll(o, 1, axis=1) for o in outV]

    def tt_no_weights(G1, G2, G3, n, ranks, h, R, c0=2.15):  # c s omega_k dropped
        w, o1, o2, o3 = orig_apply_tt(G1, G2, G3, n, ranks, h, R, c0)
        return np.ones_like(w), o1, o2, o3

    return [("apply_tucker", tucker_wrong_component), ("apply_tt", tt_no_weights)]


@pytest.mark.parametrize("name,fn", _energy_mutations(), ids=lambda x: x if isinstance(x, str) else "")
def test_energy_mutation_is_caught(monkeypatch, name, fn):
    monkeypatch.setattr(ost, name, fn)
    assert _energy_pin_error() > 1e-3


def _cube_pin_error(n=12, R=41):
    """The study's 1D-sum cube energy against the dense Tucker route."""
    from oracle import energy as oen
    h = (1.0 / n,) * 3
    core = np.zeros((3, 1, 1, 1))
    core[2] = 1.0
    V = np.ones(9 * n)
    ref = oen.energy_tucker(core, V, (n, n, n), (1, 1, 1), h, R)
    return abs(oen.uniform_cube_energy(n, R) - ref) / abs(ref)


def test_cube_energy_unmutated_is_exact():
    assert _cube_pin_error() < 1e-12


def _cube_mutations():
    from oracle import energy as oen
    orig_cs = oen.fd_column_sums

    def central_only(n, hp):  # the one-sided end stencils replaced by the central one
        cs = np.zeros(n)
        i = np.arange(n)
        np.add.at(cs, np.clip(i - 1, 0, n - 1), -0.5 / hp)
        np.add.at(cs, np.clip(i + 1, 0, n - 1), 0.5 / hp)
        return cs

    def halved(n, hp):  # a dropped factor 1/2 h_p -> 1/h_p on one end
        cs = orig_cs(n, hp)
        cs[0] *= 2.0
        return cs

    return [("central_only", central_only), ("halved", halved)]


@pytest.mark.parametrize("name,fn", _cube_mutations(), ids=lambda x: x if isinstance(x, str) else "")
def test_cube_energy_mutation_is_caught(monkeypatch, name, fn):
    from oracle import energy as oen
    monkeypatch.setattr(oen, "fd_column_sums", fn)
    assert _cube_pin_error() > 1e-3
