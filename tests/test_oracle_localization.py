"""Pins of the oracle's Jacobi-sweep Pipek-Mezey localization (Algorithm 2,
Eq. loc_theta) against facts fixed by the functional itself:

* two orbitals: one rotation reaches the maximum of L(theta), found here by a
  brute-force scan of the rotated orbitals' charges plus a golden-section
  refinement (this fixes the 1/4 and the branch of the angle, reading R19);
* at convergence every pair is stationary (b_ij ~ 0) at a maximum (a_ij <= 0),
  U is orthogonal and L does not decrease from sweep to sweep;
* the result does not depend on how the input orbitals were mixed: two
  different mixings of the same space localize to the same L and orbital set;
* the orbitals the synthetic input was mixed from are recovered;
* the single-argument arctan or a dropped 1/4 fails the two-orbital pin.
"""
import numpy as np
import pytest

import oracle
from oracle import pm_localization as pm
import synth


def _L_of(C, atom_ao):
    return oracle.pm_functional(oracle.charge_tensor(C, atom_ao))


def _two_orbital_case(seed):
    ls = synth.make_loc_system(6, seed=seed)
    return ls.C[:, [1, 4]].copy(), ls.atom_ao


def _best_rotation(C, atom_ao):
    f = lambda t: _L_of(C @ np.array([[np.cos(t), -np.sin(t)], [np.sin(t), np.cos(t)]]), atom_ao)
    ts = np.linspace(-np.pi / 4, np.pi / 4, 4001)
    v = np.array([f(t) for t in ts])
    k = int(np.argmax(v))
    lo, hi = ts[max(k - 1, 0)], ts[min(k + 1, len(ts) - 1)]
    g = (np.sqrt(5.0) - 1.0) / 2.0
    for _ in range(100):
        a, b = hi - g * (hi - lo), lo + g * (hi - lo)
        if f(a) > f(b):
            hi = b
        else:
            lo = a
    return f(0.5 * (lo + hi))


@pytest.mark.parametrize("seed", [2, 5, 9])
def test_two_orbitals_reach_the_brute_force_maximum(seed):
    C, atom_ao = _two_orbital_case(seed)
    r = oracle.pm_localize(C, atom_ao, l_loc=1e-14)
    assert abs(r.L - _best_rotation(C, atom_ao)) < 1e-10 * r.L
    assert np.allclose(r.U.T @ r.U, np.eye(2), atol=1e-14)


@pytest.mark.parametrize("slip", ["arctan", "no quarter"])
def test_planted_angle_mistakes_fail_the_two_orbital_pin(monkeypatch, slip):
    fails = 0
    for seed in (2, 5, 9):
        C, atom_ao = _two_orbital_case(seed)
        best = _best_rotation(C, atom_ao)
        atan2 = np.arctan2
        if slip == "arctan":
            monkeypatch.setattr(pm.np, "arctan2", lambda y, x: np.arctan(y / x))
        else:
            monkeypatch.setattr(pm.np, "arctan2", lambda y, x: 4.0 * atan2(y, x))
        r = oracle.pm_localize(C, atom_ao, l_loc=1e-14, max_sweeps=5)
        monkeypatch.undo()
        fails += abs(r.L - best) > 1e-8 * best
    assert fails >= 1


def test_converged_pairs_are_stationary_maxima():
    ls = synth.make_loc_system(16, seed=3)
    r = oracle.pm_localize(ls.C, ls.atom_ao, l_loc=1e-12, max_sweeps=200)
    assert r.converged
    assert np.allclose(r.U.T @ r.U, np.eye(16), atol=1e-12)
    P = oracle.charge_tensor(ls.C @ r.U, ls.atom_ao)
    for i in range(16):
        for j in range(i + 1, 16):
            Pij, Pii, Pjj = P[:, i, j], P[:, i, i], P[:, j, j]
            a = np.sum(Pij * Pij - 0.25 * (Pii - Pjj) ** 2)
            b = np.sum(Pij * (Pii - Pjj))
            assert abs(b) < 1e-5 and a < 1e-5
    assert r.L >= _L_of(ls.C, ls.atom_ao)


def test_result_is_independent_of_the_input_mixing_and_recovers_the_target():
    ls = synth.make_loc_system(12, seed=4)
    rng = np.random.default_rng(0)
    R, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    r1 = oracle.pm_localize(ls.C, ls.atom_ao, l_loc=1e-10, max_sweeps=200)
    r2 = oracle.pm_localize(ls.C @ R, ls.atom_ao, l_loc=1e-10, max_sweeps=200)
    assert abs(r1.L - r2.L) < 1e-8 * r1.L
    C1, C2 = ls.C @ r1.U, ls.C @ R @ r2.U
    ov = np.abs(C1.T @ C2)
    assert np.all(np.abs(ov.max(axis=1) - 1.0) < 1e-5)
    assert np.all(np.abs(ls.L.T @ C1).max(axis=0) > 0.98)
