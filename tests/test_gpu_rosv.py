"""Randomized OSV generation (Algorithm 3) on the GPU through the C ABI against
the oracle's randomized_osv with the same Gaussian draws (each side generates
them from the same counter-based definition): OSV counts exact, singular values
and kept spaces close, MBE(3) energies from those OSVs to 1e-9 Eh (FP64 form) /
1 uEh (mixed form), and a row budget that is too small is reported."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _t(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device=DEV)


def _build(ctx, s, l_osv):
    return ctx.build_osv(_t(s.f_occ), _t(s.e_vir), l_osv, env=_t(s.env), seed=s.seed, n_aux=s.n_aux, r_occ=s.r_occ)


def _oracle(s, l_osv):
    gauss = lambda i, k: synth.gauss_row(s.seed, i, k, s.n_vir)
    return oracle.build_osv_randomized(s.B_block, s.n_occ, s.e_vir, s.f_occ, l_osv, gauss)


@pytest.mark.parametrize("osv_prec,tol_w,tol_p", [("fp64", 1e-10, 1e-8), ("mixed", 1e-8, 1e-6)])
def test_randomized_osvs_match_oracle(osv_prec, tol_w, tol_p):
    from paper_2603_16575_gb300 import Context
    s = synth.make_system(6, 220, 330, seed=4, lam=1.0)
    Q, W, R = _oracle(s, 1e-4)
    ctx = Context(0, osv_prec=osv_prec, osv_method="randomized")
    n_osv = _build(ctx, s, 1e-4)
    assert list(n_osv) == [q.shape[1] for q in Q]
    for i in range(6):
        Qg, wg = (x.cpu().numpy() for x in ctx.get_osv(i))
        assert np.abs(wg - W[i]).max() < tol_w * W[i].max()
        assert np.allclose(Qg.T @ Qg, np.eye(Qg.shape[1]), atol=1e-10)
        assert np.abs(Qg @ Qg.T - Q[i] @ Q[i].T).max() < tol_p
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_mbe3_energy_from_randomized_osvs(prec):
    from paper_2603_16575_gb300 import Context
    s = synth.make_system(10, 64, 120, seed=21, lam=1.2)
    Q, W, _ = _oracle(s, 1e-4)
    o = oracle.OSVSystem(s.B_block, 10, s.e_vir, s.f_occ, l_osv=1e-4)
    o.Q, o.omega = Q, W
    E_ref, per = o.mbe3_energy(s.r_occ, 4.0, 3.5)
    ctx = Context(0, osv_prec=prec, osv_method="randomized")
    _build(ctx, s, 1e-4)
    E, st = ctx.mbe3_energy(4.0, 3.5, prec)
    assert st["n_unconverged"] == 0
    assert abs(E - E_ref) < (1e-9 if prec == "fp64" else 1e-6)
    ctx.close()


def test_too_few_rows_is_reported():
    from paper_2603_16575_gb300 import Context, osvmp2
    s = synth.make_system(4, 160, 240, seed=6, lam=1.0)
    ctx = Context(0, osv_method="randomized", rosv_max_rows=12)
    with pytest.raises(osvmp2.OSVMP2Error) as ei:
        _build(ctx, s, 1e-4)
    assert ei.value.code == osvmp2.STATUS_CODES["E_NUMERIC"] and "rows" in str(ei.value)
    ctx.set_opts(rosv_max_rows=0)
    assert _build(ctx, s, 1e-4).min() > 0
    ctx.close()


def test_chain_800_randomized_osv_build_samples_match_oracle():
    """The 800-orbital chain (6000 virtuals, 16000 aux, B regenerated, never stored) at its full
    size, the randomized OSV build in the mixed form as bench.py times it: orbitals 0 and 400
    against the oracle's randomized OSVs with the same Gaussian rows (counts exact, values and
    kept-space projectors to the split-precision T_ii's accuracy)."""
    from paper_2603_16575_gb300 import Context
    s = synth.workload("chain_n800", seed=0)
    ctx = Context(0, osv_prec="mixed", osv_method="randomized")
    n_osv = ctx.build_osv(_t(s.f_occ), _t(s.e_vir), 1e-4, env=_t(s.env), seed=s.seed, n_aux=s.n_aux,
                          r_occ=s.r_occ)
    assert len(n_osv) == 800 and min(n_osv) > 0
    for i in (0, 400):
        Qg, wg = (x.cpu().numpy() for x in ctx.get_osv(i))
        T = oracle.semicanonical_tii(s.B_block(i), s.e_vir, s.f_occ[i, i])
        ro = oracle.randomized_osv(T, 1e-4, lambda k, i=i: synth.gauss_row(s.seed, i, k, s.n_vir))
        assert Qg.shape[1] == ro.Q.shape[1]
        assert np.abs(wg - ro.omega).max() < 1e-8 * ro.omega.max()
        assert np.abs(Qg @ Qg.T - ro.Q @ ro.Q.T).max() < 1e-6
    ctx.close()
