"""GPU path (through the C ABI) against the FP64 CPU oracle."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _ctx(**kw):
    from paper_2603_16575_gb300 import Context
    return Context(0, **kw)


def _t(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device=DEV)


def _build(ctx, s, l_osv, stored=False):
    if stored:
        return ctx.build_osv(_t(s.f_occ), _t(s.e_vir), l_osv, B=_t(s.B_full()), r_occ=s.r_occ)
    return ctx.build_osv(_t(s.f_occ), _t(s.e_vir), l_osv, env=_t(s.env), seed=s.seed, n_aux=s.n_aux, r_occ=s.r_occ)


# ---------------------------------------------------------------- generator
@pytest.mark.parametrize("shape", [(3, 17, 45), (2, 64, 130)])
def test_generator_bit_exact(shape):
    from paper_2603_16575_gb300 import generate_B
    s = synth.make_system(*shape, seed=9, lam=2.0)
    B = generate_B(s.n_occ, s.n_vir, s.n_aux, s.seed, _t(s.env)).cpu().numpy()
    ref = s.B_full()
    assert np.array_equal(B.view(np.uint64), ref.view(np.uint64))


# ---------------------------------------------------------------- OSVs
@pytest.mark.parametrize("n_vir,l_osv,lam", [(40, 0.0, 3.0), (70, 1e-4, 1.5), (200, 1e-4, 1.0), (260, 1e-3, 1.5)])
def test_osv_match_oracle(n_vir, l_osv, lam):
    s = synth.make_system(3, n_vir, 3 * n_vir // 2 + 7, seed=4, lam=lam)
    o = oracle.OSVSystem(s.B_block, 3, s.e_vir, s.f_occ, l_osv=l_osv)
    ctx = _ctx()
    n_osv = _build(ctx, s, l_osv)
    assert list(n_osv) == [q.shape[1] for q in o.Q]
    for i in range(3):
        Q, w = ctx.get_osv(i)
        Q, w = Q.cpu().numpy(), w.cpu().numpy()
        wr = o.omega[i]
        assert np.allclose(w, wr, rtol=1e-10, atol=1e-13 * wr.max())
        assert np.allclose(Q.T @ Q, np.eye(Q.shape[1]), atol=1e-11)
        # the kept space: projectors agree
        Pr = o.Q[i] @ o.Q[i].T
        assert np.abs(Q @ Q.T - Pr).max() < 1e-9
    ctx.close()


# ---------------------------------------------------------------- pair blocks
def test_pair_blocks_match_dense_definition():
    s = synth.make_system(4, 50, 80, seed=6, lam=2.0)
    ctx = _ctx()
    _build(ctx, s, 1e-4)
    pairs = [(0, 1), (1, 3), (2, 2)]
    ctx.pair_integrals(pairs)
    Qs = [ctx.get_osv(i)[0].cpu().numpy() for i in range(4)]
    for (i, j) in pairs:
        K, S, F = (x.cpu().numpy() for x in ctx.get_pair_blocks(i, j))
        P = oracle.pair_basis(Qs, i, j)
        Kr = oracle.exchange_block(P, s.B_block(i), s.B_block(j))
        assert np.allclose(K, Kr, rtol=1e-11, atol=1e-12 * np.abs(Kr).max())
        assert np.allclose(S, P.T @ P, atol=1e-13)
        assert np.allclose(F, P.T @ (s.e_vir[:, None] * P), atol=1e-12)
    ctx.close()


def test_preconditioner_invariants_and_spectrum():
    """Eq. prec_eig: X^T S X = 1, X^T F X = diag(e~); e~ equals the oracle's generalized eigenvalues."""
    s = synth.make_system(4, 60, 90, seed=8, lam=1.5)
    ctx = _ctx()
    _build(ctx, s, 1e-4)
    ctx.pair_integrals([(0, 1), (0, 3), (2, 2)])
    for (i, j) in [(0, 1), (0, 3), (2, 2), (1, 1)]:
        X, et = (x.cpu().numpy() for x in ctx.get_precond(i, j))
        _, S, F = (x.cpu().numpy() for x in ctx.get_pair_blocks(i, j))
        r = X.shape[1]
        assert np.allclose(X.T @ S @ X, np.eye(r), atol=1e-9)
        assert np.allclose(X.T @ F @ X, np.diag(et), atol=1e-8 * max(1.0, np.abs(et).max()))
        Xr, er = oracle.preconditioner(S, F, 1e-10)
        assert Xr.shape[1] == r
        assert np.allclose(np.sort(et), np.sort(er), rtol=1e-10, atol=1e-12)
    ctx.close()


def test_mixed_preconditioner_spans_and_spectrum():
    """Mixed form: block-structured canonical orthogonalisation (FP64) and F' diagonalised
    in FP32: same rank and spectrum as the oracle to FP32 accuracy; the leftovers
    X^T S X - 1 and X^T F X - diag(e~) are small (the solver adds them exactly)."""
    s = synth.make_system(4, 60, 90, seed=8, lam=1.5)
    ctx = _ctx()
    _build(ctx, s, 1e-4)
    pairs = [(0, 1), (0, 3), (2, 2)]
    ctx.pair_integrals(pairs, prec="mixed")
    for (i, j) in pairs:
        X, et = (x.cpu().numpy() for x in ctx.get_precond(i, j))
        _, S, F = (x.cpu().numpy() for x in ctx.get_pair_blocks(i, j))
        r = X.shape[1]
        Xr, er = oracle.preconditioner(S, F, 1e-10)
        assert Xr.shape[1] == r
        scale = max(1.0, np.abs(er).max())
        assert np.abs(X.T @ S @ X - np.eye(r)).max() < 1e-4
        assert np.abs(X.T @ F @ X - np.diag(et)).max() < 1e-4 * scale
        assert np.allclose(np.sort(et), np.sort(er), atol=1e-5 * scale)
    ctx.close()


# ---------------------------------------------------------------- full solve
@pytest.mark.parametrize("stored", [False, True])
def test_untruncated_solve_equals_closed_form(stored):
    s = synth.make_system(5, 14, 40, seed=11, lam=3.0, f_off=1e-2)
    ctx = _ctx()
    _build(ctx, s, 0.0, stored=stored)
    E, pe, it = ctx.solve(range(5))
    e_cf = oracle.canonical_mp2_energy(s.B_block, 5, s.f_occ, s.e_vir)
    assert abs(E - e_cf) < 1e-9 and abs(E - e_cf) < 1e-11 * abs(e_cf)
    r = oracle.OSVSystem(s.B_block, 5, s.e_vir, s.f_occ, l_osv=0.0).solve(range(5))
    ref = [r.pair_energy[(a, b)] for a in range(5) for b in range(a, 5)]
    assert np.allclose(pe, ref, rtol=1e-9, atol=1e-12)
    ctx.close()


def test_truncated_solve_matches_oracle():
    s = synth.make_system(6, 60, 100, seed=12, lam=1.5, f_off=2e-2)
    ctx = _ctx()
    _build(ctx, s, 1e-4)
    orbs = [0, 2, 3, 5]
    E, pe, it = ctx.solve(orbs)
    o = oracle.OSVSystem(s.B_block, 6, s.e_vir, s.f_occ, l_osv=1e-4)
    r = o.solve(orbs)
    assert abs(E - r.energy) < 1e-9
    ctx.close()


# ---------------------------------------------------------------- MBE(3)
def test_mbe3_energy_matches_oracle():
    s = synth.make_system(10, 64, 120, seed=21, lam=1.2)
    ctx = _ctx()
    _build(ctx, s, 1e-4)
    E, st = ctx.mbe3_energy(4.0, 3.5)
    o = oracle.OSVSystem(s.B_block, 10, s.e_vir, s.f_occ, l_osv=1e-4)
    E_ref, per = o.mbe3_energy(s.r_occ, 4.0, 3.5)
    orbs, w, ef = ctx.fragment_results()
    assert len(per) == len(orbs)
    for (ob, c, e_ref), ogpu, cg, eg in zip(per, orbs, w, ef):
        assert tuple(int(x) for x in ogpu if x >= 0) == ob and int(cg) == c
        assert abs(eg - e_ref) < 1e-10
    assert st["n_unconverged"] == 0
    assert abs(E - E_ref) < 1e-9
    ctx.close()


# ---------------------------------------------------------------- gradient
def test_gradient_matches_oracle():
    """Frozen-OSV adjoint (dE/dB, dE/de, dE/df) against the oracle gradient, which is pinned
    by central finite differences in the CPU tests."""
    s = synth.make_system(6, 40, 80, seed=29, lam=1.5, f_off=3e-2)
    r2, r3 = 4.5, 4.0
    ctx = _ctx()
    _build(ctx, s, 1e-3)
    E, dB, df, de, st = ctx.energy_grad(r2, r3)
    o = oracle.OSVSystem(s.B_block, 6, s.e_vir, s.f_occ, l_osv=1e-3)
    E_ref, dB_ref, de_ref, df_ref = oracle.mbe3_energy_gradient(o, s.r_occ, r2, r3, 40, 80)
    assert abs(E - E_ref) < 1e-9
    dB, df, de = dB.cpu().numpy(), df.cpu().numpy(), de.cpu().numpy()
    assert np.abs(dB - dB_ref).max() < 1e-9 * np.abs(dB_ref).max()
    assert np.abs(de - de_ref).max() < 1e-9 * np.abs(de_ref).max()
    assert np.abs(df - df_ref).max() < 1e-9 * np.abs(df_ref).max()
    ctx.close()


def test_autograd_function_backward():
    from paper_2603_16575_gb300 import osvmp2
    s = synth.make_system(5, 36, 70, seed=31, lam=1.5)
    ctx = _ctx()
    B = _t(s.B_full()).requires_grad_(True)
    f = _t(s.f_occ).requires_grad_(True)
    e = _t(s.e_vir).requires_grad_(True)
    Fn = osvmp2.mbe3_energy_function()
    E = Fn.apply(ctx, B, f, e, s.r_occ, 4.5, 4.0, "fp64", 1e-3)
    (3.0 * E).backward()
    E2, dB, df, de, _ = ctx.energy_grad(4.5, 4.0)
    assert torch.allclose(B.grad, 3.0 * dB) and torch.allclose(f.grad, 3.0 * df) and torch.allclose(e.grad, 3.0 * de)
    ctx.close()


# ---------------------------------------------------------------- mixed form
def test_mixed_mbe3_energy_within_one_microhartree():
    """Preconditioner-basis solve with FP32 coupling products: total and per-fragment
    energies against the FP64 oracle (target 1 uEh total)."""
    s = synth.make_system(12, 70, 130, seed=41, lam=1.2)
    ctx = _ctx()
    _build(ctx, s, 1e-4)
    E, st = ctx.mbe3_energy(4.5, 3.8, "mixed")
    o = oracle.OSVSystem(s.B_block, 12, s.e_vir, s.f_occ, l_osv=1e-4)
    E_ref, per = o.mbe3_energy(s.r_occ, 4.5, 3.8)
    _, _, ef = ctx.fragment_results()
    assert st["n_unconverged"] == 0
    # FP32 products: per-fragment error bounded by a few eps_32 of the fragment energy
    assert max(abs(a - b[2]) / max(1.0, abs(b[2])) for a, b in zip(ef, per)) < 1e-7
    assert abs(E - E_ref) < 1e-6
    E64, _ = ctx.mbe3_energy(4.5, 3.8, "fp64")
    assert abs(E64 - E_ref) < 1e-9
    ctx.close()


@pytest.mark.parametrize("n_vir,l_osv,lam", [(70, 1e-4, 1.5), (200, 1e-4, 1.0), (260, 1e-3, 1.5)])
def test_mixed_osv_build_matches_oracle(n_vir, l_osv, lam):
    """T_ii on the tensor cores (split-precision operands, ~35 bits): OSV counts exact,
    eigenvalues and kept spaces close to the FP64 oracle."""
    s = synth.make_system(3, n_vir, 3 * n_vir // 2 + 7, seed=4, lam=lam)
    o = oracle.OSVSystem(s.B_block, 3, s.e_vir, s.f_occ, l_osv=l_osv)
    ctx = _ctx(osv_prec="mixed")
    n_osv = _build(ctx, s, l_osv)
    assert list(n_osv) == [q.shape[1] for q in o.Q]
    for i in range(3):
        Q, w = ctx.get_osv(i)
        Q, w = Q.cpu().numpy(), w.cpu().numpy()
        wr = o.omega[i]
        assert np.abs(w - wr).max() < 1e-9 * wr.max()
        assert np.allclose(Q.T @ Q, np.eye(Q.shape[1]), atol=1e-11)
        # eigenvectors of the FP64 T_ii (Eq. osv_gen): the residual is set by the ~35-bit
        # T_ii, whatever the clustering of the kept eigenvalues
        T = oracle.semicanonical_tii(s.B_block(i), s.e_vir, s.f_occ[i, i])
        assert np.abs(T @ Q - Q * w).max() < 1e-8 * wr.max()
    ctx.close()


def test_mixed_osv_and_energy_within_one_microhartree():
    """Mixed OSV build and mixed pair solve together against the FP64 oracle."""
    s = synth.make_system(12, 70, 130, seed=41, lam=1.2)
    ctx = _ctx(osv_prec="mixed")
    _build(ctx, s, 1e-4)
    E, st = ctx.mbe3_energy(4.5, 3.8, "mixed")
    o = oracle.OSVSystem(s.B_block, 12, s.e_vir, s.f_occ, l_osv=1e-4)
    E_ref, _ = o.mbe3_energy(s.r_occ, 4.5, 3.8)
    assert st["n_unconverged"] == 0
    assert abs(E - E_ref) < 1e-6
    # switching back to the FP64 build restores the FP64-form parity
    ctx.set_opts(osv_prec="fp64")
    _build(ctx, s, 1e-4)
    E64, _ = ctx.mbe3_energy(4.5, 3.8, "fp64")
    assert abs(E64 - E_ref) < 1e-9
    ctx.close()


def test_mixed_gradient_close_to_oracle():
    s = synth.make_system(6, 40, 80, seed=29, lam=1.5, f_off=3e-2)
    ctx = _ctx()
    _build(ctx, s, 1e-3)
    E, dB, df, de, st = ctx.energy_grad(4.5, 4.0, "mixed")
    o = oracle.OSVSystem(s.B_block, 6, s.e_vir, s.f_occ, l_osv=1e-3)
    E_ref, dB_ref, de_ref, df_ref = oracle.mbe3_energy_gradient(o, s.r_occ, 4.5, 4.0, 40, 80)
    assert abs(E - E_ref) < 1e-6
    for g, r in ((dB, dB_ref), (df, df_ref), (de, de_ref)):
        g = g.cpu().numpy()
        assert np.abs(g - r).max() < 1e-6 * np.abs(r).max()
    ctx.close()


def test_mixed_autotuned_graph_replay_is_exact():
    """The autotuned launch shape and the CUDA-graph replay of the mixed fragment solve
    change time only: the same energy bit for bit as the fixed default shape, on the
    first (tuning) call, on graph replays, and after the fragment list changes."""
    s = synth.make_system(14, 60, 120, seed=43, lam=1.2)
    energies = []
    for no_tune in (1, 0):
        ctx = _ctx(no_autotune=no_tune)
        _build(ctx, s, 1e-4)
        runs = [ctx.mbe3_energy(4.5, 3.8, "mixed")[0] for _ in range(3)]
        plan = ctx.solve_plan()
        assert plan["tuned"] == (no_tune == 0) and plan["n_keys"] == 1
        assert runs[0] == runs[1] == runs[2]
        other = ctx.mbe3_energy(4.0, 3.5, "mixed")[0]   # a different fragment list: new key, new graph
        assert ctx.solve_plan()["n_keys"] == 2
        again = ctx.mbe3_energy(4.5, 3.8, "mixed")[0]
        assert again == runs[0]
        energies.append((runs[0], other))
        ctx.close()
    assert energies[0] == energies[1]


def test_mixed_launch_shapes_give_identical_energies():
    """The mixed solver built for 2 and for 3 resident CTAs per SM (128 and 80 registers per
    thread) and launched at 1, 2 or 3 CTAs per SM computes the same energies bit for bit."""
    s = synth.make_system(14, 60, 120, seed=43, lam=1.2)
    got = []
    for no_tune in (1, 2, 0):
        ctx = _ctx(no_autotune=no_tune)
        _build(ctx, s, 1e-4)
        E, _ = ctx.mbe3_energy(4.5, 3.8, "mixed")
        _, _, ef = ctx.fragment_results()
        plan = ctx.solve_plan()
        if no_tune:
            assert plan["ctas_per_sm"] == no_tune + 1 and not plan["tuned"]
        got.append((E, ef.copy()))
        ctx.close()
    for E, ef in got[1:]:
        assert E == got[0][0] and np.array_equal(ef, got[0][1])


def test_mixed_form_large_pair_orders():
    """Pairs of order above 192 (more OSVs per orbital than the 128-orbital workload): the
    mixed preconditioner (eigen-solver scratch sized at launch) and solver against the oracle."""
    s = synth.make_system(5, 220, 300, seed=47, lam=1.2)    # 89-167 OSVs per orbital
    ctx = _ctx()
    n_osv = list(_build(ctx, s, 1e-4))
    assert max(n_osv) * 2 > 192
    E, st = ctx.mbe3_energy(8.0, 6.0, "mixed")
    o = oracle.OSVSystem(s.B_block, 5, s.e_vir, s.f_occ, l_osv=1e-4)
    assert [q.shape[1] for q in o.Q] == n_osv
    E_ref, _ = o.mbe3_energy(s.r_occ, 8.0, 6.0)
    assert st["n_unconverged"] == 0
    assert abs(E - E_ref) < 1e-6
    ctx.close()
