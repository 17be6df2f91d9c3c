"""Pins of the oracle's OSV-relaxed gradient (the response of the OSVs of Eq. osv_gen
to T_ii of Eq. mp2_tkk, added to the frozen-OSV derivative of the Hylleraas
functional), each against something other than the oracle itself:

* dE/dQ against central differences of the MBE(3) energy in the entries of Q
  (the fragment solver takes any, even non-orthonormal, Q), and the symmetry of
  Q^T dE/dQ that invariance of E under rotations within span(Q) demands;
* the eigenvector response alone against central differences of a
  rotation-invariant function of the kept eigenvectors of a symmetric matrix;
* the whole gradient against central differences of the energy with the OSVs
  rebuilt from the perturbed B, e and f (200 entries of B), with a check that
  the frozen-OSV gradient misses by far more than the tolerance;
* untruncated OSVs: nothing is discarded, so the relaxed and frozen gradients
  are identical;
* planted mistakes (a flipped response sign, a dropped factor) fail the pins.
"""
import numpy as np
import pytest

import oracle
import oracle.osv_mp2 as om
import synth

R2, R3, L_OSV = 4.0, 3.5, 1e-3
KW = dict(tol=1e-15, e_tol=1e-17)


@pytest.fixture(scope="module")
def fd_system():
    s = synth.make_system(4, 10, 16, seed=29, lam=2.0, f_off=3e-2)
    Bs = np.stack([s.B_block(i) for i in range(4)])
    o = oracle.OSVSystem(lambda i: Bs[i], 4, s.e_vir, s.f_occ, l_osv=L_OSV)
    return s, Bs, o


def _energy(s, Bs, e_vir, f_occ, Q=None, n_osv=None):
    """MBE(3) energy; with Q None the OSVs are rebuilt (and their counts checked)."""
    if Q is None:
        o = oracle.OSVSystem(lambda i: Bs[i], 4, e_vir, f_occ, l_osv=L_OSV)
        assert [q.shape[1] for q in o.Q] == n_osv
    else:
        o = oracle.OSVSystem.__new__(oracle.OSVSystem)
        o._B, o._Bsrc, o.cache = {}, (lambda i: Bs[i]), True
        o.n_occ, o.e_vir, o.f_occ, o.tau_s = 4, e_vir, f_occ, 1e-10
        o.Q = Q
    return o.mbe3_energy(s.r_occ, R2, R3, **KW)[0]


def _dE_dQ(o, r_occ):
    GQ = {}
    for orbs, c in oracle.mbe3_fragments(r_occ, R2, R3):
        if c == 0:
            continue
        fr = o.fragment(orbs)
        res = oracle.solve_fragment(fr, **KW)
        for x, g in oracle.fragment_dE_dQ(fr, res, o.B, o.e_vir).items():
            GQ[x] = GQ.get(x, 0.0) + c * g
    return GQ


def test_dE_dQ_matches_central_differences(fd_system):
    s, Bs, o = fd_system
    GQ = _dE_dQ(o, s.r_occ)
    scale = max(np.abs(g).max() for g in GQ.values())
    for x, g in GQ.items():
        M = o.Q[x].T @ g
        assert np.abs(M - M.T).max() < 1e-12 * scale
    h = 1e-6
    rng = np.random.default_rng(1)
    for _ in range(40):
        x = int(rng.integers(4))
        a, k = int(rng.integers(10)), int(rng.integers(o.Q[x].shape[1]))
        Qp = [q.copy() for q in o.Q]
        Qm = [q.copy() for q in o.Q]
        Qp[x][a, k] += h
        Qm[x][a, k] -= h
        fd = (_energy(s, Bs, s.e_vir, s.f_occ, Qp) - _energy(s, Bs, s.e_vir, s.f_occ, Qm)) / (2 * h)
        assert abs(fd - GQ[x][a, k]) < 1e-7 * scale


def test_eigenvector_response_matches_central_differences():
    """E(Q) = tr(Q^T A Q) over the 3 largest eigenvectors of a symmetric T is invariant
    under rotations within span(Q); its derivative in T is <Z, dT> with Z from
    osv_response(T, Q, 2 A Q)."""
    rng = np.random.default_rng(5)
    n, k = 9, 3
    M = rng.standard_normal((n, n))
    T = M @ M.T
    A = rng.standard_normal((n, n))
    A = A + A.T

    def top(Tm):
        w, V = np.linalg.eigh(Tm)
        return V[:, np.argsort(-w)[:k]]

    Q = top(T)
    Z, gap = oracle.osv_response(T, Q, 2.0 * A @ Q)
    assert gap > 0.05 and np.abs(Z - Z.T).max() == 0.0
    h = 1e-6
    for _ in range(20):
        D = rng.standard_normal((n, n))
        D = D + D.T
        fp = np.trace(top(T + h * D).T @ A @ top(T + h * D))
        fm = np.trace(top(T - h * D).T @ A @ top(T - h * D))
        assert abs((fp - fm) / (2 * h) - float(np.sum(Z * D))) < 1e-7 * np.abs(Z).max() * n


@pytest.fixture(scope="module")
def relaxed(fd_system):
    s, Bs, o = fd_system
    return oracle.mbe3_energy_gradient_relaxed(o, s.r_occ, R2, R3, 10, 16, **KW)


def test_relaxed_gradient_matches_central_differences(fd_system, relaxed):
    s, Bs, o = fd_system
    n_osv = [q.shape[1] for q in o.Q]
    E, dB, de, df, gap = relaxed
    assert 1e-4 < gap and min(n_osv) >= 1 and max(n_osv) < 10
    _, dB0, de0, df0 = oracle.mbe3_energy_gradient(o, s.r_occ, R2, R3, 10, 16, **KW)
    h = 1e-5
    rng = np.random.default_rng(3)
    scale = np.abs(dB).max()
    miss = 0.0
    for _ in range(200):
        i, a, p = int(rng.integers(4)), int(rng.integers(10)), int(rng.integers(16))
        Bp, Bm = Bs.copy(), Bs.copy()
        Bp[i, a, p] += h
        Bm[i, a, p] -= h
        fd = (_energy(s, Bp, s.e_vir, s.f_occ, n_osv=n_osv) - _energy(s, Bm, s.e_vir, s.f_occ, n_osv=n_osv)) / (2 * h)
        assert abs(fd - dB[i, a, p]) < 1e-6 * scale
        miss = max(miss, abs(fd - dB0[i, a, p]))
    assert miss > 1e-3 * scale           # the OSV response is not negligible here
    for a in range(0, 10, 3):
        ep, em = s.e_vir.copy(), s.e_vir.copy()
        ep[a] += h
        em[a] -= h
        fd = (_energy(s, Bs, ep, s.f_occ, n_osv=n_osv) - _energy(s, Bs, em, s.f_occ, n_osv=n_osv)) / (2 * h)
        assert abs(fd - de[a]) < 1e-6 * np.abs(de).max()
    for (k, l) in [(0, 0), (0, 1), (1, 3), (2, 2)]:
        fp, fm = s.f_occ.copy(), s.f_occ.copy()
        fp[k, l] += h
        fm[k, l] -= h
        if k != l:
            fp[l, k] += h
            fm[l, k] -= h
        fd = (_energy(s, Bs, s.e_vir, fp, n_osv=n_osv) - _energy(s, Bs, s.e_vir, fm, n_osv=n_osv)) / (2 * h)
        want = df[k, l] * (1.0 if k == l else 2.0)
        assert abs(fd - want) < 1e-6 * np.abs(df).max()


def test_untruncated_relaxed_equals_frozen(fd_system):
    s, Bs, _ = fd_system
    o = oracle.OSVSystem(lambda i: Bs[i], 4, s.e_vir, s.f_occ, l_osv=0.0)
    E, dB, de, df, gap = oracle.mbe3_energy_gradient_relaxed(o, s.r_occ, R2, R3, 10, 16)
    E0, dB0, de0, df0 = oracle.mbe3_energy_gradient(o, s.r_occ, R2, R3, 10, 16)
    assert gap == np.inf and E == E0
    assert np.array_equal(dB, dB0) and np.array_equal(de, de0) and np.array_equal(df, df0)


@pytest.mark.parametrize("slip", ["response_sign", "dQ_factor", "tii_B_factor"])
def test_planted_mistakes_fail_the_relaxed_pin(fd_system, monkeypatch, slip):
    s, Bs, o = fd_system
    if slip == "response_sign":
        f0 = om.osv_response
        monkeypatch.setattr(om, "osv_response", lambda T, Q, G: (lambda r: (-r[0], r[1]))(f0(T, Q, G)))
    elif slip == "dQ_factor":
        f0 = om.fragment_dE_dQ
        monkeypatch.setattr(om, "fragment_dE_dQ",
                            lambda *a: {x: 0.5 * g for x, g in f0(*a).items()})
    else:
        f0 = om.tii_adjoint
        monkeypatch.setattr(om, "tii_adjoint", lambda Z, B, e, f: (lambda r: (0.5 * r[0],) + r[1:])(f0(Z, B, e, f)))
    _, dB, _, _, _ = om.mbe3_energy_gradient_relaxed(o, s.r_occ, R2, R3, 10, 16, **KW)
    n_osv = [q.shape[1] for q in o.Q]
    h = 1e-5
    rng = np.random.default_rng(3)
    worst = 0.0
    for _ in range(12):
        i, a, p = int(rng.integers(4)), int(rng.integers(10)), int(rng.integers(16))
        Bp, Bm = Bs.copy(), Bs.copy()
        Bp[i, a, p] += h
        Bm[i, a, p] -= h
        fd = (_energy(s, Bp, s.e_vir, s.f_occ, n_osv=n_osv) - _energy(s, Bm, s.e_vir, s.f_occ, n_osv=n_osv)) / (2 * h)
        worst = max(worst, abs(fd - dB[i, a, p]))
    assert worst > 1e-6 * np.abs(dB).max()
