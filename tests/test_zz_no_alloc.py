"""The allocation-free preconditioner entry point against the regular path.

Some callers of this library cannot allocate device memory while they run: a
process whose own pool allocator owns all GPU memory and forbids further driver
allocations, a plug-in working inside another application's CUDA context under
that application's memory budget, or a latency-critical loop in which a
cudaMalloc (which may synchronise the device) is unacceptable.
osvmp2_precond_noalloc serves them with a static device scratch array.  This
test calls it through the C ABI, twice in a row per pair, and checks its output
against the preconditioner that osvmp2_pair_integrals built for the same pair.
The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _t(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda:0")


def test_noalloc_precond_matches_regular_path_on_two_calls():
    from paper_2603_16575_gb300 import Context, osvmp2
    s = synth.make_system(4, 60, 90, seed=8, lam=1.5)
    ctx = Context(0)
    ctx.build_osv(_t(s.f_occ), _t(s.e_vir), 1e-4, env=_t(s.env), seed=s.seed, n_aux=s.n_aux, r_occ=s.r_occ)
    pairs = [(0, 1), (2, 2), (1, 3)]
    ctx.pair_integrals(pairs)
    L = osvmp2.lib()
    stream = torch.cuda.current_stream().cuda_stream
    for (i, j) in pairs:
        _, S, F = ctx.get_pair_blocks(i, j)
        X_ref, et_ref = ctx.get_precond(i, j)
        Xr, er = X_ref.cpu().numpy(), et_ref.cpu().numpy()
        m, r_ref = S.shape[0], Xr.shape[1]
        for _call in range(2):
            X = torch.full((m, m), float("nan"), dtype=torch.float64, device="cuda:0")
            et = torch.full((m,), float("nan"), dtype=torch.float64, device="cuda:0")
            r = torch.full((1,), -7, dtype=torch.int32, device="cuda:0")
            buf = ctypes.create_string_buffer(256)
            code = L.osvmp2_precond_noalloc(S.data_ptr(), F.data_ptr(), m, 1e-10, X.data_ptr(), et.data_ptr(),
                                            r.data_ptr(), stream, buf, 256)
            assert code == 0, buf.value
            torch.cuda.synchronize()
            assert int(r.item()) == r_ref
            Xg, eg = X[:, :r_ref].cpu().numpy(), et[:r_ref].cpu().numpy()
            assert np.allclose(np.sort(eg), np.sort(er), rtol=1e-10, atol=1e-12)
            # basis-independent comparison (eigenvector signs and order may differ)
            P_ref, P = Xr @ Xr.T, Xg @ Xg.T
            assert np.abs(P - P_ref).max() <= 1e-9 * np.abs(P_ref).max()
            G_ref, G = Xr @ np.diag(er) @ Xr.T, Xg @ np.diag(eg) @ Xg.T
            assert np.abs(G - G_ref).max() <= 1e-9 * np.abs(G_ref).max()
    # sizes beyond the static scratch are refused with a message
    big = torch.zeros((osvmp2.NOALLOC_MAX_M + 1,) * 2, dtype=torch.float64, device="cuda:0")
    out = torch.zeros_like(big)
    et = torch.zeros(big.shape[0], dtype=torch.float64, device="cuda:0")
    r = torch.zeros(1, dtype=torch.int32, device="cuda:0")
    buf = ctypes.create_string_buffer(256)
    code = L.osvmp2_precond_noalloc(big.data_ptr(), big.data_ptr(), big.shape[0], 1e-10, out.data_ptr(),
                                    et.data_ptr(), r.data_ptr(), stream, buf, 256)
    assert code == osvmp2.STATUS_CODES["E_ARG"] and b"outside" in buf.value
    ctx.close()


def _call(L, S, F, m, stream, tau_s=1e-10):
    X = torch.full((m, m), float("nan"), dtype=torch.float64, device="cuda:0")
    et = torch.full((m,), float("nan"), dtype=torch.float64, device="cuda:0")
    r = torch.full((1,), -7, dtype=torch.int32, device="cuda:0")
    buf = ctypes.create_string_buffer(256)
    code = L.osvmp2_precond_noalloc(S.data_ptr(), F.data_ptr(), m, tau_s, X.data_ptr(), et.data_ptr(), r.data_ptr(),
                                    stream, buf, 256)
    assert code == 0, buf.value
    torch.cuda.synchronize()
    return X, et, int(r.item())


@pytest.mark.parametrize("m", [200, 256])
def test_noalloc_precond_large_orders_in_global_scratch(m):
    """Orders above the shared-memory eigenvector limit (144) up to the static
    scratch's maximum (256): dense random S (SPD) and F (symmetric), two calls in a
    row; X^T S X = 1, X^T F X = diag(e~) and e~ equal to the generalized eigenvalues."""
    scipy_linalg = pytest.importorskip("scipy.linalg")
    from paper_2603_16575_gb300 import osvmp2
    rng = np.random.default_rng(m)
    A = rng.standard_normal((m, m))
    S_h = A @ A.T / m + 0.5 * np.eye(m)
    Fm = rng.standard_normal((m, m))
    F_h = 0.5 * (Fm + Fm.T)
    want = scipy_linalg.eigh(F_h, S_h, eigvals_only=True)
    S, F = _t(S_h), _t(F_h)
    L = osvmp2.lib()
    stream = torch.cuda.current_stream().cuda_stream
    for _call_no in range(2):
        X, et, r = _call(L, S, F, m, stream)
        assert r == m
        Xh, eh = X.cpu().numpy(), et.cpu().numpy()
        assert np.abs(Xh.T @ S_h @ Xh - np.eye(m)).max() < 1e-9
        assert np.abs(Xh.T @ F_h @ Xh - np.diag(eh)).max() < 1e-9 * max(1.0, np.abs(want).max())
        assert np.allclose(np.sort(eh), want, rtol=1e-10, atol=1e-10)


def test_noalloc_precond_degenerate_and_nonfinite_inputs():
    """S = 0 has no direction above tau_s * max: r = 0.  A NaN in S: r = -1."""
    from paper_2603_16575_gb300 import osvmp2
    L = osvmp2.lib()
    stream = torch.cuda.current_stream().cuda_stream
    m = 24
    F = _t(np.eye(m))
    for _call_no in range(2):
        _, _, r = _call(L, _t(np.zeros((m, m))), F, m, stream)
        assert r == 0
    S_nan = np.eye(m)
    S_nan[3, 5] = S_nan[5, 3] = np.nan
    _, _, r = _call(L, _t(S_nan), F, m, stream)
    assert r == -1
    # the Python wrapper refuses outputs that are too small for the kernel
    X = torch.zeros((m - 1, m), dtype=torch.float64, device="cuda:0")
    et = torch.zeros(m, dtype=torch.float64, device="cuda:0")
    rr = torch.zeros(1, dtype=torch.int32, device="cuda:0")
    with pytest.raises(ValueError):
        osvmp2.precond_noalloc(F, F, 1e-10, X, et, rr)
    with pytest.raises(TypeError):
        osvmp2.precond_noalloc(F, F, 1e-10, torch.zeros((m, m), dtype=torch.float64, device="cuda:0"), et,
                               rr.to(torch.int64))
