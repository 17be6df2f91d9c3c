"""Pins of the oracle's pair screening and weak-pair branch (Eqs. s2b, s3b,
osv_weak_k, res_weak; Algorithm 7, weak pairs) against facts fixed by the
mathematics rather than by the oracle itself.

* s2b of complete OSV bases is 1 for every pair (the overlap of two orthogonal
  matrices has Frobenius norm^2 = n), and 0 for OSVs on disjoint virtuals.
* Untruncated, two orbitals: with the diagonal amplitudes of the full
  two-orbital solve, the single-block weak-pair equation is the full pair
  equation, so the weak amplitude equals the full solve's T_ij.
* Untruncated with a diagonal occupied Fock block: the weak-pair energy is the
  direct (Coulomb-like) part of the canonical pair energy,
  4 sum_ab (ia|jb)^2 / (f_ii + f_jj - e_a - e_b) for both orders.
* With every pair close and every triple kept, the screened cluster list is the
  all-inclusive MBE(3) list (whose inclusion-exclusion identity is pinned
  elsewhere); weights sum to one over the clusters containing any cluster.
* The printed form of Eq. res_weak (T F_(j,i), (f_ij + f_ii)) fails these pins.
"""
import itertools

import numpy as np
import pytest

import oracle
import synth


def _full_space(P, T):
    return P @ T @ P.T


def test_s2b_closed_forms():
    s = synth.make_system(3, 12, 30, seed=2, lam=2.0)
    o = oracle.OSVSystem(s.B_block, 3, s.e_vir, s.f_occ, l_osv=0.0)
    M = oracle.s2b_matrix(o.Q)
    assert np.allclose(M, 1.0, atol=1e-13)
    Q = [np.eye(6)[:, :3], np.eye(6)[:, 3:], np.eye(6)[:, [0, 4]]]
    assert oracle.s2b_metric(Q, 0, 1) == 0.0
    assert abs(oracle.s2b_metric(Q, 0, 2) - 1.0 / np.sqrt(6.0)) < 1e-15
    assert abs(oracle.s3b_metric(np.array([[1, .3, .6], [.3, 1, .9], [.6, .9, 1]]), 0, 1, 2) - 0.6) < 1e-15


def _two_orbital_full(f_off, seed=41):
    s = synth.make_system(2, 12, 36, seed=seed, lam=2.5, f_off=f_off)
    o = oracle.OSVSystem(s.B_block, 2, s.e_vir, s.f_occ, l_osv=0.0)
    r = o.solve((0, 1), tol=1e-14, e_tol=1e-16, max_iter=400)
    assert r.converged
    return s, o, r


def test_weak_amplitude_equals_full_pair_amplitude_untruncated():
    s, o, r = _two_orbital_full(f_off=5e-2)
    fr = o.fragment((0, 1))
    T_full = _full_space(fr.P[(0, 1)], r.T[(0, 1)])
    w = oracle.weak_pair(o.Q, o.B, s.f_occ, s.e_vir, 0, 1, r.T[(0, 0)], r.T[(1, 1)])
    T_weak = o.Q[0] @ w.T @ o.Q[1].T
    assert np.abs(T_weak - T_full).max() < 1e-11 * np.abs(T_full).max()
    # and it zeroes its own residual
    R = oracle.weak_residual(o.Q, o.B, s.f_occ, s.e_vir, 0, 1, w.T, r.T[(0, 0)], r.T[(1, 1)])
    assert np.abs(R).max() < 1e-12 * np.abs(w.T).max()


def test_weak_energy_is_the_direct_canonical_term_for_diagonal_fock():
    s = synth.make_system(2, 12, 36, seed=43, lam=2.5, f_off=0.0)
    o = oracle.OSVSystem(s.B_block, 2, s.e_vir, s.f_occ, l_osv=0.0)
    zero = [np.zeros((12, 12))] * 2
    w = oracle.weak_pair(o.Q, o.B, s.f_occ, s.e_vir, 0, 1, *zero)
    K = s.B_block(0) @ s.B_block(1).T
    D = s.f_occ[0, 0] + s.f_occ[1, 1] - s.e_vir[:, None] - s.e_vir[None, :]
    want = 4.0 * float(np.sum(K * K / D))
    assert abs(w.energy - want) < 1e-12 * abs(want)


@pytest.mark.parametrize("slip", ["F_(j,i)", "(f_ij + f_ii)"])
def test_printed_form_of_res_weak_fails_the_pins(slip):
    """The equation as printed (a garbled F_(j,i), a (f_ij + f_ii) shift) does not
    reproduce the full pair amplitude, so reading R17 is the one the pins fix."""
    s, o, r = _two_orbital_full(f_off=5e-2)
    fr = o.fragment((0, 1))
    T_full = _full_space(fr.P[(0, 1)], r.T[(0, 1)])
    Q, f, e = o.Q, s.f_occ, s.e_vir
    i, j = 0, 1
    K = (Q[i].T @ o.B(i)) @ (Q[j].T @ o.B(j)).T
    S = Q[i].T @ Q[j]
    Fii = Q[i].T @ (e[:, None] * Q[i])
    Fjj_ok = Q[j].T @ (e[:, None] * Q[j])
    Fjj = Fjj_ok if slip != "F_(j,i)" else Q[j].T @ (e[:, None] * Q[i])
    shift = f[i, i] + f[j, j] if slip != "(f_ij + f_ii)" else f[i, j] + f[i, i]
    # solve the linear single-block equation by brute force (Kronecker form)
    n = Fii.shape[0]
    rhs = -(K - f[i, j] * (r.T[(0, 0)] @ S + S @ r.T[(1, 1)]))
    A = np.kron(Fii, np.eye(n)) + np.kron(np.eye(n), Fjj.T) - shift * np.eye(n * n)
    T_bad = np.linalg.solve(A, rhs.ravel()).reshape(n, n)
    assert np.abs(Q[i] @ T_bad @ Q[j].T - T_full).max() > 1e-4 * np.abs(T_full).max()
    # while the same brute force with reading R17 reproduces it
    A = np.kron(Fii, np.eye(n)) + np.kron(np.eye(n), Fjj_ok.T) - (f[i, i] + f[j, j]) * np.eye(n * n)
    T_good = np.linalg.solve(A, rhs.ravel()).reshape(n, n)
    assert np.abs(Q[i] @ T_good @ Q[j].T - T_full).max() < 1e-10 * np.abs(T_full).max()


def test_screened_lists_are_subset_closed_and_reduce_to_the_full_list():
    s = synth.make_system(4, 12, 30, seed=19, lam=2.0, f_off=3e-2)
    o = oracle.OSVSystem(s.B_block, 4, s.e_vir, s.f_occ, l_osv=1e-3)
    M = oracle.s2b_matrix(o.Q)
    every = oracle.Screen(s2b_distant=0.0, s2b_close=0.0, s3b_min=0.0)
    frags, weak = oracle.screened_fragments(M, every)
    assert weak == []
    assert frags == oracle.mbe3_fragments(s.r_occ, 1e3, 1e3)
    # the paper's cuts on a larger synthetic box
    b = synth.make_system(24, 60, 80, seed=5, lam=1.0)
    ob = oracle.OSVSystem(b.B_block, 24, b.e_vir, b.f_occ, l_osv=1e-4)
    Mb = oracle.s2b_matrix(ob.Q)
    frags, weak = oracle.screened_fragments(Mb, oracle.Screen())
    kept = {o_ for o_, _ in frags}
    for o_, _ in frags:
        for r in range(1, len(o_)):
            for sub in itertools.combinations(o_, r):
                assert sub in kept
        assert sum(c for S, c in frags if set(o_) <= set(S)) == 1
    for (i, j) in weak:
        assert 1e-7 <= Mb[i, j] < 1e-2 and (i, j) not in kept


def test_diagonal_amplitudes_follow_the_mbe_expansion():
    """Eq. tmbediag written out term by term for a 3-orbital all-kept list equals the
    weighted sum over clusters."""
    s = synth.make_system(3, 10, 24, seed=17, lam=2.0, f_off=3e-2)
    o = oracle.OSVSystem(s.B_block, 3, s.e_vir, s.f_occ, l_osv=1e-3)
    frags = oracle.mbe3_fragments(s.r_occ, 1e3, 1e3)
    res = [o.solve(orbs) for orbs, _ in frags]
    Td = oracle.mbe3_diagonal_amplitudes(res, frags)
    T = {orbs: r.T for (orbs, _), r in zip(frags, res)}
    t1 = T[(0,)][(0, 0)]
    d01 = T[(0, 1)][(0, 0)] - t1
    d02 = T[(0, 2)][(0, 0)] - t1
    d012 = T[(0, 1, 2)][(0, 0)] - d01 - d02 - t1
    assert np.abs(Td[0] - (t1 + d01 + d02 + d012)).max() < 1e-14 * np.abs(t1).max()
