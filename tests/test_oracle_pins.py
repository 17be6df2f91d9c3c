"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: published
generator vectors, the canonical RI-MP2 closed form (Eq. mp2_tmat with the
Section-2 energy), orbital invariance of the Hylleraas solution, a dense LU
solve of the same linear equations, the full-virtual-space definition of the
projected residual, the inclusion-exclusion identity behind Eqs.
(tmbediag)-(deltaoff), and central finite differences for the gradient.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- generator
def test_splitmix64_published_vectors():
    want = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_state0.txt"))
            if l.strip() and not l.startswith("#")]
    got = synth.draws(0, np.arange(4, dtype=np.uint64))
    assert [int(x) for x in got] == want
    # scalar and vector finalisers agree
    z = [synth.mix64_int(0x1234567 + k * 977) for k in range(50)]
    zv = synth.mix64(np.array([0x1234567 + k * 977 for k in range(50)], dtype=np.uint64))
    assert z == [int(v) for v in zv]


def test_irwin_hall_normal_moments():
    z = synth.normal_ih12(synth.stream_key(7, synth.S_B), np.arange(1_000_000, dtype=np.uint64))
    n = z.size
    assert abs(z.mean()) < 5.0 / np.sqrt(n)
    assert abs(z.var() - 1.0) < 5.0 * np.sqrt(2.0 / n)
    assert z.min() >= -6.0 and z.max() <= 6.0
    # values are exact multiples of 2^-16
    assert np.all(z * 65536.0 == np.round(z * 65536.0))


def test_system_recipe_ranges():
    s = synth.make_system(20, 100, 40, seed=3, lam=3.0)
    assert s.e_occ.min() >= -1.5 and s.e_occ.max() <= -0.3
    assert s.e_vir.min() >= 0.1 and s.e_vir.max() <= 5.0
    assert np.allclose(s.f_occ, s.f_occ.T)
    assert np.all(np.diag(s.f_occ) == s.e_occ)
    assert s.r_occ.min() >= 0 and s.r_occ.max() <= 10.0
    B = s.B_block(3)
    assert B[5, 7] == s.B_entry(3, 5, 7)
    c = synth.make_system(10, 30, 8, geometry="chain", lam=1.0)
    assert np.all(c.r_occ[:, 0] == 1.5 * np.arange(10))


# ---------------------------------------------------------------- OSVs
@pytest.mark.parametrize("l_osv", [0.0, 1e-3])
def test_osv_diagonalises_tii(l_osv):
    s = synth.make_system(3, 16, 40, seed=2, lam=2.0)
    for i in range(3):
        T = oracle.semicanonical_tii(s.B_block(i), s.e_vir, s.f_occ[i, i])
        w_all = np.linalg.eigvalsh(T)
        assert w_all.min() > -1e-14 * w_all.max()          # PSD (Schur product theorem)
        Q, w = oracle.osv_from_tii(T, l_osv)
        assert np.allclose(Q.T @ Q, np.eye(Q.shape[1]), atol=1e-13)
        assert np.allclose(Q.T @ T @ Q, np.diag(w), atol=1e-13 * w_all.max())
        assert np.all(np.diff(w) <= 0)
        if l_osv > 0:
            assert np.all(w >= l_osv) and np.sum(w_all >= l_osv) == len(w)
        else:
            assert Q.shape == (16, 16)
        big = np.argmax(np.abs(Q), axis=0)
        assert np.all(Q[big, np.arange(Q.shape[1])] > 0)


def test_semicanonical_tii_is_the_single_orbital_amplitude():
    """Eq. mp2_tmat at i = j: the amplitude of a one-orbital cluster (Eq. res_close with
    k = i only, which keeps f_ii alone even for a non-diagonal Fock block) is
    T_ii^ab = K_ii^ab / (2 f_ii - e_a - e_b).  Obtained here from the untruncated
    iterative solve (pinned to the closed form, and independent of the OSVs' T_ii once
    they span the whole space), its negative must be the semi-canonical T_ii of
    Eq. mp2_tkk under reading R4."""
    s = synth.make_system(3, 14, 40, seed=37, lam=2.0, f_off=3e-2)
    o = oracle.OSVSystem(s.B_block, 3, s.e_vir, s.f_occ, l_osv=0.0)
    for i in range(3):
        r = o.solve((i,), tol=1e-14, e_tol=1e-16, max_iter=200)
        T_full = o.Q[i] @ r.T[(i, i)] @ o.Q[i].T
        Ts = oracle.semicanonical_tii(s.B_block(i), s.e_vir, s.f_occ[i, i])
        assert np.abs(-T_full - Ts).max() < 1e-11 * np.abs(Ts).max()


@pytest.mark.parametrize("slip", ["f_ii for 2 f_ii", "sign of the denominator"])
def test_planted_tii_mistakes_fail_the_amplitude_pin(monkeypatch, slip):
    """A dropped factor 2 on f_ii, or the opposite sign of Eq. mp2_tkk's literal form,
    fails the one-orbital amplitude pin above."""
    s = synth.make_system(2, 14, 40, seed=37, lam=2.0, f_off=3e-2)
    o = oracle.OSVSystem(s.B_block, 2, s.e_vir, s.f_occ, l_osv=0.0)
    r = o.solve((0,), tol=1e-14, e_tol=1e-16, max_iter=200)
    T_full = o.Q[0] @ r.T[(0, 0)] @ o.Q[0].T
    if slip == "f_ii for 2 f_ii":
        bad = lambda B, e, f: (B @ B.T) / (e[:, None] + e[None, :] - f)
    else:
        bad = lambda B, e, f: (B @ B.T) / (2.0 * f - e[:, None] - e[None, :])
    monkeypatch.setattr(oracle, "semicanonical_tii", bad)
    Ts = oracle.semicanonical_tii(s.B_block(0), s.e_vir, s.f_occ[0, 0])
    assert np.abs(-T_full - Ts).max() > 1e-3 * np.abs(Ts).max()


def test_preconditioner_invariants():
    s = synth.make_system(3, 14, 30, seed=4, lam=3.0)
    o = oracle.OSVSystem(s.B_block, 3, s.e_vir, s.f_occ, l_osv=1e-4)
    fr = o.fragment((0, 1, 2))
    for p in fr.pairs:
        X, e = fr.X[p], fr.Et[p]
        assert np.allclose(X.T @ fr.S(p, p) @ X, np.eye(len(e)), atol=1e-11)
        assert np.allclose(X.T @ fr.F(p, p) @ X, np.diag(e), atol=1e-10)


# ---------------------------------------------------------------- residual
def test_residual_matches_full_space_definition():
    """Eq. (res_close) in the OSV basis equals P^T R_full P with
    R_full = K + F T + T F - sum_k (f_ik T_kj + f_kj T_ik) in the full virtual space."""
    s = synth.make_system(3, 12, 30, seed=5, lam=2.5)
    o = oracle.OSVSystem(s.B_block, 3, s.e_vir, s.f_occ, l_osv=1e-4)
    fr = o.fragment((0, 1, 2))
    rng = np.random.default_rng(0)
    T = {p: rng.standard_normal((fr.P[p].shape[1],) * 2) for p in fr.pairs}
    for (i, j) in fr.pairs:            # T_ii = T_ii^T: diagonal-pair amplitudes are symmetric
        if i == j:
            T[(i, j)] = T[(i, j)] + T[(i, j)].T
    Tfull = {}
    for (i, j) in fr.pairs:
        Tfull[(i, j)] = fr.P[(i, j)] @ T[(i, j)] @ fr.P[(i, j)].T
        Tfull[(j, i)] = Tfull[(i, j)].T
    Fv = np.diag(s.e_vir)
    f = s.f_occ
    for (i, j) in fr.pairs:
        Kf = s.B_block(i) @ s.B_block(j).T
        Rf = Kf + Fv @ Tfull[(i, j)] + Tfull[(i, j)] @ Fv
        for k in fr.orbs:
            Rf -= f[i, k] * Tfull[(k, j)] + f[k, j] * Tfull[(i, k)]
        P = fr.P[(i, j)]
        want = P.T @ Rf @ P
        got = fr.residual(T, (i, j))
        assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())


# ---------------------------------------------------------------- closed form
@pytest.mark.parametrize("f_off", [0.0, 1e-2, 5e-2])
def test_untruncated_solve_equals_canonical_closed_form(f_off):
    s = synth.make_system(5, 14, 40, seed=11, lam=3.0, f_off=f_off)
    o = oracle.OSVSystem(s.B_block, 5, s.e_vir, s.f_occ, l_osv=0.0)
    r = o.solve(range(5))
    assert r.converged
    e_cf = oracle.canonical_mp2_energy(s.B_block, 5, s.f_occ, s.e_vir)
    assert abs(r.energy - e_cf) < 1e-12 * abs(e_cf)


def test_closed_form_at_first_workload_shape():
    """The 20-orbital untruncated case (n_vir=100, n_aux=400) against the closed form."""
    s = synth.workload("canonical_n20", seed=0)
    o = oracle.OSVSystem(s.B_block, s.n_occ, s.e_vir, s.f_occ, l_osv=0.0)
    r = o.solve(range(s.n_occ))
    e_cf = oracle.canonical_mp2_energy(s.B_block, s.n_occ, s.f_occ, s.e_vir)
    assert r.converged
    assert abs(r.energy - e_cf) < 1e-9       # absolute Eh
    assert abs(r.energy - e_cf) < 1e-11 * abs(e_cf)


def test_occupied_rotation_invariance():
    s = synth.make_system(4, 12, 30, seed=13, lam=3.0)
    o = oracle.OSVSystem(s.B_block, 4, s.e_vir, s.f_occ, l_osv=0.0)
    e0 = o.solve(range(4)).energy
    rng = np.random.default_rng(1)
    U, _ = np.linalg.qr(rng.standard_normal((4, 4)))
    Bs = np.stack([s.B_block(i) for i in range(4)])
    Br = np.einsum("ik,iaP->kaP", U, Bs)
    fr = U.T @ s.f_occ @ U
    o2 = oracle.OSVSystem(lambda i: Br[i], 4, s.e_vir, fr, l_osv=0.0)
    e1 = o2.solve(range(4)).energy
    assert abs(e1 - e0) < 1e-10 * abs(e0)


def test_iteration_matches_dense_lu_truncated():
    s = synth.make_system(3, 10, 24, seed=17, lam=2.0, f_off=3e-2)
    o = oracle.OSVSystem(s.B_block, 3, s.e_vir, s.f_occ, l_osv=1e-3)
    for orbs in [(0,), (0, 2), (0, 1, 2)]:
        fr = o.fragment(orbs)
        a = oracle.solve_fragment(fr)
        b = oracle.solve_fragment_dense(fr)
        assert a.converged
        assert abs(a.energy - b.energy) < 1e-12 * abs(b.energy)
        for p in fr.pairs:
            Pa = fr.P[p] @ a.T[p] @ fr.P[p].T
            Pb = fr.P[p] @ b.T[p] @ fr.P[p].T
            assert np.allclose(Pa, Pb, atol=1e-12 * np.abs(Pb).max())


# ---------------------------------------------------------------- MBE(3)
def _subset_energy(o, S):
    return o.solve(S).energy


def test_mbe3_plus_four_body_equals_full_solve():
    s = synth.make_system(4, 12, 30, seed=19, lam=2.0, f_off=3e-2)
    o = oracle.OSVSystem(s.B_block, 4, s.e_vir, s.f_occ, l_osv=1e-3)
    e_mbe3, per = o.mbe3_energy(s.r_occ, 1e3, 1e3)
    assert len(per) == 4 + 6 + 4
    full = _subset_energy(o, (0, 1, 2, 3))
    d4 = 0.0
    for r in range(1, 5):
        for S in itertools.combinations(range(4), r):
            d4 += (-1) ** (4 - r) * _subset_energy(o, S)
    assert abs(e_mbe3 + d4 - full) < 1e-13 * abs(full)
    # three orbitals: MBE(3) is the full solve
    e3, _ = oracle.OSVSystem(s.B_block, 3, s.e_vir, s.f_occ[:3, :3], l_osv=1e-3).mbe3_energy(s.r_occ[:3], 1e3, 1e3)
    assert abs(e3 - _subset_energy(o, (0, 1, 2))) < 1e-13 * abs(e3)


def test_fragment_weights_are_inclusion_exclusion():
    s = synth.make_system(40, 10, 4, seed=23)
    frags = oracle.mbe3_fragments(s.r_occ, 4.0, 3.0)
    sets = [(set(o), c) for o, c in frags]
    kept = {o for o, _ in frags}
    for o, _ in frags:
        # every subset of a kept cluster is kept
        for r in range(1, len(o)):
            for sub in itertools.combinations(o, r):
                assert sub in kept
        # weights of the clusters containing it sum to one
        assert sum(c for S, c in sets if set(o) <= S) == 1


def test_fragment_list_on_chain_with_exact_ties():
    """Chain of 1.5 A spacing: 8 A keeps |i-j| <= 5, 6 A keeps triples spanning <= 4 steps (tie included)."""
    n = 12
    r = np.zeros((n, 3))
    r[:, 0] = 1.5 * np.arange(n)
    frags = oracle.mbe3_fragments(r, 8.0, 6.0)
    pairs = [o for o, _ in frags if len(o) == 2]
    triples = [o for o, _ in frags if len(o) == 3]
    assert len(pairs) == sum(1 for i in range(n) for j in range(i + 1, n) if j - i <= 5)
    assert len(triples) == sum(1 for i in range(n) for k in range(i + 2, n) if k - i <= 4
                               for j in range(i + 1, k))
    assert (0, 2, 4) in [t for t in triples]


# ---------------------------------------------------------------- gradient
def _fd_system():
    s = synth.make_system(4, 10, 16, seed=29, lam=2.0, f_off=3e-2)
    Bs = np.stack([s.B_block(i) for i in range(4)])
    return s, Bs


def _energy(Bs, s, Q, e_vir, f_occ, r2, r3):
    o = oracle.OSVSystem.__new__(oracle.OSVSystem)
    o._B, o._Bsrc, o.cache = {}, (lambda i: Bs[i]), True
    o.n_occ, o.e_vir, o.f_occ, o.tau_s = 4, e_vir, f_occ, 1e-10
    o.Q = Q
    return o.mbe3_energy(s.r_occ, r2, r3, tol=1e-15, e_tol=1e-17)[0]


def test_gradient_matches_central_differences():
    s, Bs = _fd_system()
    r2, r3 = 4.0, 3.5
    o = oracle.OSVSystem(lambda i: Bs[i], 4, s.e_vir, s.f_occ, l_osv=1e-3)
    frags = oracle.mbe3_fragments(s.r_occ, r2, r3)
    assert any(len(f) == 2 for f, _ in frags)
    E, dB, de, df = oracle.mbe3_energy_gradient(o, s.r_occ, r2, r3, 10, 16, tol=1e-15, e_tol=1e-17)
    h = 1e-5
    rng = np.random.default_rng(3)
    scale = np.abs(dB).max()
    for _ in range(200):
        i, a, p = rng.integers(4), rng.integers(10), rng.integers(16)
        Bp, Bm = Bs.copy(), Bs.copy()
        Bp[i, a, p] += h
        Bm[i, a, p] -= h
        fd = (_energy(Bp, s, o.Q, s.e_vir, s.f_occ, r2, r3) - _energy(Bm, s, o.Q, s.e_vir, s.f_occ, r2, r3)) / (2 * h)
        assert abs(fd - dB[i, a, p]) < 1e-6 * scale
    for a in range(0, 10, 3):
        ep, em = s.e_vir.copy(), s.e_vir.copy()
        ep[a] += h
        em[a] -= h
        fd = (_energy(Bs, s, o.Q, ep, s.f_occ, r2, r3) - _energy(Bs, s, o.Q, em, s.f_occ, r2, r3)) / (2 * h)
        assert abs(fd - de[a]) < 1e-6 * np.abs(de).max()
    for (k, l) in [(0, 0), (0, 1), (1, 3), (2, 2)]:
        fp, fm = s.f_occ.copy(), s.f_occ.copy()
        fp[k, l] += h
        fm[k, l] -= h
        if k != l:
            fp[l, k] += h
            fm[l, k] -= h
        fd = (_energy(Bs, s, o.Q, s.e_vir, fp, r2, r3) - _energy(Bs, s, o.Q, s.e_vir, fm, r2, r3)) / (2 * h)
        want = df[k, l] * (1.0 if k == l else 2.0)
        assert abs(fd - want) < 1e-6 * np.abs(df).max()


# ---------------------------------------------------------------- the pins bite
def test_planted_mistakes_fail_the_closed_form(monkeypatch):
    """A dropped term or a missing transpose in the oracle breaks the closed-form pin."""
    s = synth.make_system(4, 12, 30, seed=31, lam=3.0, f_off=5e-2)
    e_cf = oracle.canonical_mp2_energy(s.B_block, 4, s.f_occ, s.e_vir)

    def run():
        o = oracle.OSVSystem(s.B_block, 4, s.e_vir, s.f_occ, l_osv=0.0)
        return o.solve(range(4), max_iter=200).energy

    assert abs(run() - e_cf) < 1e-12 * abs(e_cf)
    orig_amp = oracle.Fragment.ordered_amp
    monkeypatch.setattr(oracle.Fragment, "ordered_amp",
                        lambda self, T, i, k: T[(i, k)] if i <= k else oracle.swap_blocks(T[(k, i)], self.n[k]))
    assert abs(run() - e_cf) > 1e-8 * abs(e_cf)
    monkeypatch.setattr(oracle.Fragment, "ordered_amp", orig_amp)
    orig_pe = oracle.Fragment.pair_energy
    monkeypatch.setattr(oracle.Fragment, "pair_energy",
                        lambda self, T, p: float(np.sum(self.K[p] * (2 * T[p] - T[p].T))))
    assert abs(run() - e_cf) > 1e-6 * abs(e_cf)
    monkeypatch.setattr(oracle.Fragment, "pair_energy", orig_pe)
