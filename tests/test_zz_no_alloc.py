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
