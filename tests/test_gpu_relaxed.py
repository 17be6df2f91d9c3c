"""OSV-relaxed gradient (frozen-OSV derivative plus the response of the OSVs of
Eq. osv_gen to T_ii of Eq. mp2_tkk) on the GPU through the C ABI, against the FP64
oracle: all of dE/dB, dE/de, dE/df and the eigenvalue gap at the OSV cut on small
systems (virtual spaces below and above the shared-memory limit of the full
eigen-solver), and the dE/dB rows of orbital 0 at the gradient workload's full
size.  The relaxed term is checked to matter (far above the tolerance)."""
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


@pytest.mark.parametrize("n,nv,nx,seed,r2,r3", [(8, 48, 90, 3, 4.5, 3.8), (5, 200, 260, 11, 6.0, 5.0)])
def test_relaxed_gradient_matches_oracle(n, nv, nx, seed, r2, r3):
    from paper_2603_16575_gb300 import Context
    s = synth.make_system(n, nv, nx, seed=seed, lam=1.2, f_off=3e-2)
    ctx = Context(0)
    _build(ctx, s, 1e-4)
    E, dB, df, de, st, gap = ctx.energy_grad_relaxed(r2, r3)
    assert st["n_unconverged"] == 0
    o = oracle.OSVSystem(s.B_block, n, s.e_vir, s.f_occ, l_osv=1e-4)
    E_r, dB_r, de_r, df_r, gap_r = oracle.mbe3_energy_gradient_relaxed(o, s.r_occ, r2, r3, nv, nx)
    _, dB_f, de_f, df_f = oracle.mbe3_energy_gradient(o, s.r_occ, r2, r3, nv, nx)
    assert abs(E - E_r) < 1e-10
    assert abs(gap - gap_r) < 1e-9 * abs(gap_r)
    sB = np.abs(dB_r).max()
    assert np.abs(dB_r - dB_f).max() > 1e-4 * sB          # the OSV response is not negligible
    assert np.abs(dB.cpu().numpy() - dB_r).max() < 1e-9 * sB
    assert np.abs(de.cpu().numpy() - de_r).max() < 1e-9 * np.abs(de_r).max()
    assert np.abs(df.cpu().numpy() - df_r).max() < 1e-9 * np.abs(df_r).max()
    ctx.close()


def test_relaxed_needs_exact_osvs():
    from paper_2603_16575_gb300 import Context, osvmp2
    s = synth.make_system(6, 60, 100, seed=4, lam=1.2)
    ctx = Context(0, osv_method="randomized")
    _build(ctx, s, 1e-4)
    with pytest.raises(osvmp2.OSVMP2Error) as ei:
        ctx.energy_grad_relaxed(4.5, 3.8)
    assert ei.value.code == osvmp2.STATUS_CODES["E_ARG"]
    ctx.close()


def test_relaxed_rows_at_the_gradient_workload_shape():
    """64 orbitals / 320 virtuals / 1200 aux: the relaxed dE/dB rows of orbital 0 (fed by
    the fragments containing it, through both the frozen term and the response of Q_0)
    against the oracle, relative to their largest entry."""
    from paper_2603_16575_gb300 import Context
    s = synth.workload("grad_n64", seed=0)
    ctx = Context(0)
    _build(ctx, s, 1e-4)
    E, dB, df, de, st, gap = ctx.energy_grad_relaxed(8.0, 6.0)
    assert st["n_unconverged"] == 0 and gap > 0
    frags = [(o, c) for o, c in oracle.mbe3_fragments(s.r_occ, 8.0, 6.0) if 0 in o and c != 0]
    orbs = sorted({x for o, _ in frags for x in o})
    osys = oracle.OSVSystem(s.B_block, s.n_occ, s.e_vir, s.f_occ, l_osv=1e-4, orbitals=orbs)
    frozen = np.zeros((s.n_vir, s.n_aux))
    G0 = 0.0
    for o, c in frags:
        fr = osys.fragment(o)
        res = oracle.solve_fragment(fr)
        gB, _, _ = oracle.fragment_gradient(fr, res, osys.B, s.n_occ, s.n_vir, s.n_aux)
        frozen += c * gB[0]
        G0 = G0 + c * oracle.fragment_dE_dQ(fr, res, osys.B, s.e_vir)[0]
    T00 = oracle.semicanonical_tii(osys.B(0), s.e_vir, s.f_occ[0, 0])
    Z, _ = oracle.osv_response(T00, osys.Q[0], G0)
    ref = frozen + oracle.tii_adjoint(Z, osys.B(0), s.e_vir, s.f_occ[0, 0])[0]
    got = dB[0].cpu().numpy()
    assert np.abs(got - ref).max() < 1e-9 * np.abs(ref).max()
    assert np.abs(ref - frozen).max() > 1e-6 * np.abs(ref).max()
    ctx.close()


def test_autograd_function_relaxed_backward():
    from paper_2603_16575_gb300 import Context, osvmp2
    s = synth.make_system(5, 36, 70, seed=31, lam=1.5)
    ctx = Context(0)
    B = _t(s.B_full()).requires_grad_(True)
    f = _t(s.f_occ).requires_grad_(True)
    e = _t(s.e_vir).requires_grad_(True)
    Fn = osvmp2.mbe3_energy_function()
    E = Fn.apply(ctx, B, f, e, s.r_occ, 4.5, 4.0, "fp64", 1e-3, True)
    (2.0 * E).backward()
    E2, dB, df, de, _, _ = ctx.energy_grad_relaxed(4.5, 4.0)
    _, dB0, _, _, _ = ctx.energy_grad(4.5, 4.0)
    assert float(E.detach()) == E2
    assert torch.allclose(B.grad, 2.0 * dB) and torch.allclose(f.grad, 2.0 * df) and torch.allclose(e.grad, 2.0 * de)
    assert not torch.allclose(dB, dB0)
    ctx.close()


def test_untruncated_relaxed_equals_frozen_bit_for_bit():
    """l_osv = 0 keeps every eigenvector: nothing is discarded, the response vanishes, and the
    relaxed outputs are the frozen ones exactly, with no gap at the cut."""
    from paper_2603_16575_gb300 import Context
    s = synth.make_system(5, 30, 60, seed=2, lam=1.2, f_off=3e-2)
    ctx = Context(0)
    n_osv = _build(ctx, s, 0.0)
    assert list(n_osv) == [30] * 5
    E, dB, df, de, st, gap = ctx.energy_grad_relaxed(4.5, 3.8)
    E0, dB0, df0, de0, _ = ctx.energy_grad(4.5, 3.8)
    assert gap == float("inf") and E == E0
    assert torch.equal(dB, dB0) and torch.equal(df, df0) and torch.equal(de, de0)
    ctx.close()


def test_relaxed_failure_statuses_and_recovery():
    """Made on the host: the call before any OSV build is E_STATE; max_iter = 1 makes the
    fragment solve fail with E_NOCONV; the ctx then gives the gradient with the default limit."""
    from paper_2603_16575_gb300 import Context, osvmp2
    ctx = Context(0)
    with pytest.raises(osvmp2.OSVMP2Error) as ei:
        ctx.energy_grad_relaxed(4.5, 3.8)
    assert ei.value.code == osvmp2.STATUS_CODES["E_STATE"]
    s = synth.make_system(6, 40, 80, seed=9, lam=1.2, f_off=3e-2)
    _build(ctx, s, 1e-4)
    ctx.set_opts(max_iter=1)
    with pytest.raises(osvmp2.OSVMP2Error) as ei:
        ctx.energy_grad_relaxed(4.5, 3.8)
    assert ei.value.code == osvmp2.STATUS_CODES["E_NOCONV"]
    ctx.set_opts(max_iter=100)
    E, dB, df, de, st, gap = ctx.energy_grad_relaxed(4.5, 3.8)
    assert st["n_unconverged"] == 0 and np.isfinite(E) and gap > 0
    assert bool(torch.isfinite(dB).all()) and bool(torch.isfinite(de).all()) and bool(torch.isfinite(df).all())
    ctx.close()
