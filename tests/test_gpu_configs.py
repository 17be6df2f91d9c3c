"""GPU path at the stated workload shapes, and its failure statuses.

* The 20-orbital untruncated system (n_vir = 100, n_aux = 400) through
  osvmp2_solve against the canonical RI-MP2 closed form (Eq. mp2_tmat with the
  Section-2 energy).  Its pairs have order 200, so the CTA-per-pair FP64
  preconditioner (orders above the one-warp limit of 192) runs here.
* The 128-orbital MBE(3) workload that bench.py times: every fragment among the
  10 orbitals nearest orbital 0 (the bench's oracle sample) is solved by the
  oracle and compared fragment by fragment with the GPU's fragment energies.
* Failure statuses made on the host: max_iter = 1 -> E_NOCONV with the failing
  fragment reported, a device-memory cap -> E_NOMEM, calls out of order ->
  E_STATE.  None of them faults or stalls the GPU.
"""
import ctypes

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


def test_first_config_untruncated_solve_equals_closed_form():
    from paper_2603_16575_gb300 import Context
    s = synth.workload("canonical_n20", seed=0)
    ctx = Context(0)
    n_osv = _build(ctx, s, 0.0)
    assert list(n_osv) == [s.n_vir] * s.n_occ
    E, pe, it = ctx.solve(range(s.n_occ))
    e_cf = oracle.canonical_mp2_energy(s.B_block, s.n_occ, s.f_occ, s.e_vir)
    assert abs(E - e_cf) < 1e-9, (E, e_cf)
    assert np.isclose(pe.sum(), E, rtol=1e-13, atol=0.0)
    ctx.close()


@pytest.fixture(scope="module")
def bench_sample():
    """Oracle energies of every fragment among the 10 orbitals nearest orbital 0
    of the 128-orbital workload (the sample bench.py's CPU baseline times)."""
    s = synth.workload("mbe3_n128", seed=0)
    d = np.linalg.norm(s.r_occ - s.r_occ[0], axis=1)
    near = sorted(np.argsort(d, kind="stable")[:10].tolist())
    frags = [o for o, _ in oracle.mbe3_fragments(s.r_occ, 8.0, 6.0) if set(o) <= set(near)]
    osys = oracle.OSVSystem(s.B_block, s.n_occ, s.e_vir, s.f_occ, l_osv=1e-4, orbitals=near)
    ref = {o: osys.solve(o).energy for o in frags}
    counts = {i: osys.Q[i].shape[1] for i in near}
    return s, ref, counts


def _gpu_fragment_energies(ctx):
    orbs, _, e = ctx.fragment_results()
    return {tuple(int(x) for x in o if x >= 0): float(v) for o, v in zip(orbs, e)}


@pytest.mark.parametrize("osv_prec,prec", [("fp64", "fp64"), ("mixed", "mixed"), ("fp64", "mixed")])
def test_bench_workload_fragments_match_oracle(bench_sample, osv_prec, prec):
    from paper_2603_16575_gb300 import Context
    s, ref, counts = bench_sample
    ctx = Context(0, osv_prec=osv_prec)
    n_osv = _build(ctx, s, 1e-4)
    assert all(int(n_osv[i]) == c for i, c in counts.items())
    E, st = ctx.mbe3_energy(8.0, 6.0, prec)
    assert st["n_unconverged"] == 0
    got = _gpu_fragment_energies(ctx)
    assert len(ref) > 100
    worst_abs = max(abs(got[o] - e) for o, e in ref.items())
    worst_rel = max(abs(got[o] - e) / abs(e) for o, e in ref.items())
    if prec == "fp64":
        assert worst_abs < 1e-9, worst_abs
    else:
        # split-precision contractions: per-fragment error bounded as in the small-case test
        assert worst_rel < 1e-7, worst_rel
    ctx.close()


# ---------------------------------------------------------------- failure statuses
def test_max_iter_one_reports_noconv_and_the_failing_fragment():
    from paper_2603_16575_gb300 import Context, osvmp2
    s = synth.make_system(8, 48, 90, seed=3, lam=1.2, f_off=3e-2)
    ctx = Context(0, max_iter=1)
    _build(ctx, s, 1e-4)
    for prec in ("fp64", "mixed"):
        e = ctypes.c_double(0.0)
        st = osvmp2.MbeStats()
        code = osvmp2.lib().osvmp2_mbe3_energy(ctx._h, 4.5, 3.8, osvmp2.PREC[prec], ctypes.addressof(e),
                                               ctypes.byref(st))
        assert code == osvmp2.STATUS_CODES["E_NOCONV"], code
        assert st.n_unconverged > 0 and 0 <= st.worst_fragment < st.n_single + st.n_pair + st.n_triple
        assert st.max_iter_used == 1
        assert b"did not converge" in osvmp2.lib().osvmp2_last_error(ctx._h)
    with pytest.raises(osvmp2.OSVMP2Error) as ei:
        ctx.solve([0, 1, 2])
    assert ei.value.code == osvmp2.STATUS_CODES["E_NOCONV"]
    # the ctx stays usable: with the default limit the same call converges
    ctx.set_opts(max_iter=100)
    E, st = ctx.mbe3_energy(4.5, 3.8, "fp64")
    assert st["n_unconverged"] == 0 and np.isfinite(E)
    ctx.close()


def test_memory_cap_gives_nomem_and_the_ctx_recovers():
    from paper_2603_16575_gb300 import Context, osvmp2
    s = synth.make_system(6, 200, 300, seed=5, lam=1.2)
    ctx = Context(0, mem_cap_mib=1)          # the T_ii batch alone needs ~2 MB
    with pytest.raises(osvmp2.OSVMP2Error) as ei:
        _build(ctx, s, 1e-4)
    assert ei.value.code == osvmp2.STATUS_CODES["E_NOMEM"]
    ctx.set_opts(mem_cap_mib=0)
    n_osv = _build(ctx, s, 1e-4)
    assert n_osv.min() > 0
    # a cap that admits the OSV build but not the pair store
    ctx.set_opts(mem_cap_mib=64)
    _build(ctx, s, 1e-4)
    ctx.set_opts(mem_cap_mib=2)
    with pytest.raises(osvmp2.OSVMP2Error) as ei:
        ctx.mbe3_energy(8.0, 6.0, "fp64")
    assert ei.value.code == osvmp2.STATUS_CODES["E_NOMEM"]
    ctx.set_opts(mem_cap_mib=0)
    E, st = ctx.mbe3_energy(8.0, 6.0, "fp64")
    assert st["n_unconverged"] == 0
    ctx.close()


def test_calls_out_of_order_give_state_errors():
    from paper_2603_16575_gb300 import Context, osvmp2
    ctx = Context(0)
    L = osvmp2.lib()
    pairs = np.array([[0, 1]], dtype=np.int32)
    e = ctypes.c_double(0.0)
    orbs = np.array([0, 1], dtype=np.int32)
    E_STATE = osvmp2.STATUS_CODES["E_STATE"]
    assert L.osvmp2_pair_integrals(ctx._h, pairs.ctypes.data, 1, 0) == E_STATE
    assert L.osvmp2_solve(ctx._h, orbs.ctypes.data, 2, 0, ctypes.addressof(e), None, None) == E_STATE
    assert L.osvmp2_mbe3_energy(ctx._h, 8.0, 6.0, 0, ctypes.addressof(e), None) == E_STATE
    assert L.osvmp2_get_osv(ctx._h, 0, None, None) == E_STATE
    s = synth.make_system(4, 30, 60, seed=2, lam=1.5)
    _build(ctx, s, 1e-4)
    # a pair that was never built
    assert L.osvmp2_get_pair_blocks(ctx._h, 0, 3, None, None, None) == E_STATE
    assert L.osvmp2_get_precond(ctx._h, 0, 3, None, None, None) == E_STATE
    ctx.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("mixed", 3e-6)])
def test_gradient_rows_at_the_gradient_workload_shape(prec, tol):
    """64 orbitals / 320 virtuals / 1200 aux: the frozen-OSV dE/dB rows of orbital 0,
    which only the fragments containing it feed, against the oracle (relative to their
    largest entry).  The mixed form's back-projection dB = U (W~ G) runs in FP32, so its
    bound is a few FP32 ulps (measured 1.1e-6) rather than the FP64 form's 1e-9."""
    from paper_2603_16575_gb300 import Context
    s = synth.workload("grad_n64", seed=0)
    ctx = Context(0, osv_prec="fp64")
    _build(ctx, s, 1e-4)
    E, dB, df, de, st = ctx.energy_grad(8.0, 6.0, prec)
    assert st["n_unconverged"] == 0
    frags = [(o, c) for o, c in oracle.mbe3_fragments(s.r_occ, 8.0, 6.0) if 0 in o and c != 0]
    orbs = sorted({x for o, _ in frags for x in o})
    osys = oracle.OSVSystem(s.B_block, s.n_occ, s.e_vir, s.f_occ, l_osv=1e-4, orbitals=orbs)
    ref = np.zeros((s.n_vir, s.n_aux))
    for o, c in frags:
        fr = osys.fragment(o)
        gB, _, _ = oracle.fragment_gradient(fr, oracle.solve_fragment(fr), osys.B, s.n_occ, s.n_vir, s.n_aux)
        ref += c * gB[0]
    got = dB[0].cpu().numpy()
    assert np.abs(got - ref).max() < tol * np.abs(ref).max()
    ctx.close()


@pytest.mark.parametrize("osv_method,prec", [("exact", "fp64"), ("exact", "mixed"), ("randomized", "mixed")])
def test_second_config_fragments_match_oracle(osv_method, prec):
    """256 orbitals / 1200 virtuals / 4800 aux (the second workload's full size): the
    fragments among the 6 orbitals nearest orbital 0, solved inside the whole MBE(3)
    launch, against the oracle with the same OSV rule."""
    from paper_2603_16575_gb300 import Context
    s = synth.workload("osv_n256", seed=0)
    d = np.linalg.norm(s.r_occ - s.r_occ[0], axis=1)
    near = sorted(np.argsort(d, kind="stable")[:6].tolist())
    frags = [o for o, _ in oracle.mbe3_fragments(s.r_occ, 8.0, 6.0) if set(o) <= set(near)]
    if osv_method == "randomized":
        osys = oracle.OSVSystem(s.B_block, s.n_occ, s.e_vir, s.f_occ, l_osv=1e-4, orbitals=[])
        gauss = lambda i, k: synth.gauss_row(s.seed, i, k, s.n_vir)
        osys.Q, osys.omega, _ = oracle.build_osv_randomized(osys.B, s.n_occ, s.e_vir, s.f_occ, 1e-4, gauss,
                                                            orbitals=near)
    else:
        osys = oracle.OSVSystem(s.B_block, s.n_occ, s.e_vir, s.f_occ, l_osv=1e-4, orbitals=near)
    ctx = Context(0, osv_prec="fp64" if prec == "fp64" else "mixed", osv_method=osv_method)
    n_osv = _build(ctx, s, 1e-4)
    assert all(int(n_osv[i]) == osys.Q[i].shape[1] for i in near)
    E, st = ctx.mbe3_energy(8.0, 6.0, prec)
    assert st["n_unconverged"] == 0
    got = _gpu_fragment_energies(ctx)
    assert len(frags) >= 10
    for o in frags:
        e_ref = osys.solve(o).energy
        if prec == "fp64":
            assert abs(got[o] - e_ref) < 1e-9, (o, got[o], e_ref)
        else:
            assert abs(got[o] - e_ref) < 1e-7 * abs(e_ref), (o, got[o], e_ref)
    ctx.close()
