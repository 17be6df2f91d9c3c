"""Pair screening (Eqs. s2b, s3b) and weak pairs (Eq. res_weak, Algorithm 7) on the
GPU through the C ABI, against the FP64 oracle: s2b values and the class lists
(bit-exact, with the distance of every s2b from the cuts checked first), the
cluster list and weights, per-cluster and per-weak-pair energies, and totals
(1e-9 Eh FP64 form, 1 uEh mixed form)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _t(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device=DEV)


def _setup(n, nv, nx, seed, box, osv_prec="fp64"):
    from paper_2603_16575_gb300 import Context
    s = synth.make_system(n, nv, nx, seed=seed, lam=1.0, box_edge=box)
    ctx = Context(0, osv_prec=osv_prec)
    n_osv = ctx.build_osv(_t(s.f_occ), _t(s.e_vir), 1e-4, env=_t(s.env), seed=s.seed, n_aux=s.n_aux, r_occ=s.r_occ)
    o = oracle.OSVSystem(s.B_block, n, s.e_vir, s.f_occ, l_osv=1e-4)
    assert list(n_osv) == [q.shape[1] for q in o.Q]
    return s, ctx, o


@pytest.fixture(scope="module")
def ref20():
    s = synth.make_system(20, 80, 200, seed=7, lam=1.0, box_edge=12.0)
    o = oracle.OSVSystem(s.B_block, 20, s.e_vir, s.f_occ, l_osv=1e-4)
    return oracle.mbe3_screened_energy(o, oracle.Screen())


def test_s2b_and_pair_classes_match_oracle(ref20):
    from paper_2603_16575_gb300 import osvmp2
    _, _, _, _, M = ref20
    s, ctx, o = _setup(20, 80, 200, 7, 12.0)
    s2b, cls, cnt = ctx.pair_screening(osvmp2.Screen())
    assert np.allclose(s2b, M, rtol=1e-12, atol=1e-15)
    iu = np.triu_indices(20, 1)
    v = M[iu]
    # no s2b within rounding of a cut, so the class decisions are well defined
    assert min(np.min(np.abs(v - 1e-2) / 1e-2), np.min(np.abs(v - 1e-7) / 1e-7)) > 1e-9
    want = np.where(M >= 1e-2, 2, np.where(M >= 1e-7, 1, 0))
    np.fill_diagonal(want, 2)
    assert np.array_equal(cls, want)
    assert cnt == (int((v >= 1e-2).sum()), int(((v >= 1e-7) & (v < 1e-2)).sum()), int((v < 1e-7).sum()))
    ctx.close()


def test_screened_mbe3_fp64_matches_oracle(ref20):
    E_ref, Ew_ref, per, wres, _ = ref20
    s, ctx, o = _setup(20, 80, 200, 7, 12.0)
    E, Ew, st = ctx.mbe3_energy_screened("fp64")
    orbs, w, ef = ctx.fragment_results()
    assert len(orbs) == len(per)
    for (ob, c, e_ref), og, cg, eg in zip(per, orbs, w, ef):
        assert tuple(int(x) for x in og if x >= 0) == ob and int(cg) == c
        assert abs(eg - e_ref) < 1e-10
    pairs, ew = ctx.weak_results()
    assert [tuple(int(x) for x in p) for p in pairs] == [r.pair for r in wres]
    assert st["n_weak"] == len(wres) > 0
    for g, r in zip(ew, wres):
        assert abs(g - r.energy) < 1e-12 + 1e-10 * abs(r.energy)
    assert abs(Ew - Ew_ref) < 1e-11
    assert abs(E - E_ref) < 1e-9
    assert st["n_unconverged"] == 0
    ctx.close()


@pytest.mark.parametrize("osv_prec", ["fp64", "mixed"])
def test_screened_mbe3_mixed_within_one_microhartree(ref20, osv_prec):
    E_ref, Ew_ref, per, wres, _ = ref20
    s, ctx, o = _setup(20, 80, 200, 7, 12.0, osv_prec=osv_prec)
    E, Ew, st = ctx.mbe3_energy_screened("mixed")
    assert st["n_unconverged"] == 0 and st["n_weak"] == len(wres)
    _, ew = ctx.weak_results()
    for g, r in zip(ew, wres):
        assert abs(g - r.energy) < 1e-7 * max(abs(r.energy), 1e-6)
    assert abs(Ew - Ew_ref) < 1e-8
    assert abs(E - E_ref) < 1e-6
    ctx.close()


def test_all_weak_and_all_close_limits():
    """s2b_close above 1: no close pair, every non-distant pair is weak and its
    diagonal amplitudes are the single-orbital ones.  s2b_close = s2b_distant = 0 and
    s3b_min = 0: every pair and triple is a cluster, no weak pair, and the energy is
    the distance-rule MBE(3) energy with every cluster kept."""
    from paper_2603_16575_gb300 import osvmp2
    s, ctx, o = _setup(16, 80, 200, 5, 11.0)
    E, Ew, st = ctx.mbe3_energy_screened("fp64", osvmp2.Screen(1e-7, 2.0, 0.2))
    M = oracle.s2b_matrix(o.Q)
    frags, weak = oracle.screened_fragments(M, oracle.Screen(1e-7, 2.0, 0.2))
    assert len(frags) == 16 and st["n_pair"] == 0 and st["n_weak"] == len(weak)
    res = [o.solve(orbs) for orbs, _ in frags]
    Td = oracle.mbe3_diagonal_amplitudes(res, frags)
    want = sum(oracle.weak_pair(o.Q, o.B, s.f_occ, s.e_vir, i, j, Td[i], Td[j]).energy for (i, j) in weak)
    assert abs(Ew - want) < 1e-11
    assert abs(E - (want + sum(r.energy for r in res))) < 1e-9
    E_all, Ew_all, st = ctx.mbe3_energy_screened("fp64", osvmp2.Screen(0.0, 0.0, 0.0))
    E_dist, _ = ctx.mbe3_energy(1e3, 1e3, "fp64")
    assert Ew_all == 0.0 and st["n_weak"] == 0
    assert abs(E_all - E_dist) < 1e-12
    ctx.close()
