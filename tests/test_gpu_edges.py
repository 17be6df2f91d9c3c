"""Edge cases of the GPU path against the oracle: one orbital, singles only (zero
cutoffs), an orbital with a single OSV, ragged pair orders within one launch, the
screening with no weak pair, and an orbital left without any OSV (an error)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _t(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda:0")


def _ctx_build(s, l_osv, **kw):
    from paper_2603_16575_gb300 import Context
    ctx = Context(0, **kw)
    n = ctx.build_osv(_t(s.f_occ), _t(s.e_vir), l_osv, env=_t(s.env), seed=s.seed, n_aux=s.n_aux, r_occ=s.r_occ)
    return ctx, n


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_single_orbital(prec):
    s = synth.make_system(1, 30, 50, seed=3, lam=1.5)
    ctx, n = _ctx_build(s, 1e-4)
    E, st = ctx.mbe3_energy(8.0, 6.0, prec)
    o = oracle.OSVSystem(s.B_block, 1, s.e_vir, s.f_occ, l_osv=1e-4)
    assert st["n_single"] == 1 and st["n_pair"] == 0 and st["n_triple"] == 0
    assert abs(E - o.solve((0,)).energy) < (1e-10 if prec == "fp64" else 1e-7 * abs(E))
    ctx.close()


def test_singles_only_and_ragged_orders():
    """Zero cutoffs keep the singles only; OSV counts from 1 to tens in one launch."""
    s = synth.make_system(8, 60, 100, seed=11, lam=1.2)
    ctx, n_osv = _ctx_build(s, 1e-3)
    o = oracle.OSVSystem(s.B_block, 8, s.e_vir, s.f_occ, l_osv=1e-3)
    assert list(n_osv) == [q.shape[1] for q in o.Q]
    assert min(n_osv) <= 3 < max(n_osv)
    E, st = ctx.mbe3_energy(0.0, 0.0, "fp64")
    assert st["n_pair"] == 0
    assert abs(E - sum(o.solve((i,)).energy for i in range(8))) < 1e-10
    E, st = ctx.mbe3_energy(5.0, 4.0, "fp64")
    E_ref, _ = o.mbe3_energy(s.r_occ, 5.0, 4.0)
    assert abs(E - E_ref) < 1e-10
    ctx.close()


def test_orbital_with_one_osv():
    """The cut between the two largest omega of the orbital whose largest omega is the
    smallest: that orbital keeps one OSV, every other keeps at least one."""
    s = synth.make_system(3, 40, 60, seed=5, lam=1.0)
    o = oracle.OSVSystem(s.B_block, 3, s.e_vir, s.f_occ, l_osv=1e-4)
    i1 = int(np.argmin([w.max() for w in o.omega]))
    w1 = np.sort(o.omega[i1])
    l_osv = float(0.5 * (w1[-1] + w1[-2]))
    o2 = oracle.OSVSystem(s.B_block, 3, s.e_vir, s.f_occ, l_osv=l_osv)
    counts = [q.shape[1] for q in o2.Q]
    assert counts[i1] == 1 and min(counts) >= 1
    ctx, n_osv = _ctx_build(s, l_osv)
    assert list(n_osv) == counts
    for prec, tol in (("fp64", 1e-10), ("mixed", 1e-7)):
        E, st = ctx.mbe3_energy(8.0, 6.0, prec)
        E_ref, _ = o2.mbe3_energy(s.r_occ, 8.0, 6.0)
        assert abs(E - E_ref) < tol * max(1.0, abs(E_ref))
    ctx.close()


def test_orbital_without_osv_is_an_error():
    from paper_2603_16575_gb300 import osvmp2
    s = synth.make_system(3, 40, 60, seed=5, lam=1.0)
    from paper_2603_16575_gb300 import Context
    ctx = Context(0)
    with pytest.raises(osvmp2.OSVMP2Error) as ei:
        ctx.build_osv(_t(s.f_occ), _t(s.e_vir), 1e3, env=_t(s.env), seed=s.seed, n_aux=s.n_aux, r_occ=s.r_occ)
    assert ei.value.code == osvmp2.STATUS_CODES["E_NUMERIC"]
    ctx.close()


def test_screening_with_every_pair_distant():
    from paper_2603_16575_gb300 import osvmp2
    s = synth.make_system(5, 40, 80, seed=9, lam=1.2)
    ctx, _ = _ctx_build(s, 1e-4)
    o = oracle.OSVSystem(s.B_block, 5, s.e_vir, s.f_occ, l_osv=1e-4)
    E, Ew, st = ctx.mbe3_energy_screened("fp64", osvmp2.Screen(2.0, 2.0, 0.2))
    assert st["n_pair"] == 0 and st["n_weak"] == 0 and Ew == 0.0
    assert abs(E - sum(o.solve((i,)).energy for i in range(5))) < 1e-10
    ctx.close()
