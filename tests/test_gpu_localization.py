"""Jacobi-sweep Pipek-Mezey localization (Algorithm 2) on the GPU through the C
ABI against the oracle on the same synthetic orbitals: the same number of
sweeps (the dL of every sweep kept away from l_loc), the functional L and the
rotation U (both follow the same sequence of rotations, so U agrees entry by
entry up to rounding), at a tight and at the paper's threshold; too few sweeps
give E_NOCONV."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,l_loc", [(24, 1e-9), (96, 1e-3)])
def test_localization_matches_oracle(n, l_loc):
    from paper_2603_16575_gb300 import Context
    ls = synth.make_loc_system(n, seed=7)
    ref = oracle.pm_localize(ls.C, ls.atom_ao, l_loc=l_loc, max_sweeps=200)
    assert ref.converged
    ctx = Context(0)
    C = torch.tensor(ls.C, dtype=torch.float64, device="cuda:0")
    U, L, sweeps = ctx.localize_pm(C, ls.atom_ao, l_loc=l_loc, max_sweeps=200)
    U = U.cpu().numpy()
    assert sweeps == ref.sweeps
    assert abs(L - ref.L) < 1e-10 * ref.L
    assert np.abs(U - ref.U).max() < 1e-7
    assert np.allclose(U.T @ U, np.eye(n), atol=1e-12)
    # the localized orbitals are the ones the input was mixed from
    assert np.all(np.abs(ls.L.T @ (ls.C @ U)).max(axis=0) > 0.9)
    ctx.close()


def test_localization_sweep_limit_is_reported():
    from paper_2603_16575_gb300 import Context, osvmp2
    ls = synth.make_loc_system(16, seed=2)
    ctx = Context(0)
    C = torch.tensor(ls.C, dtype=torch.float64, device="cuda:0")
    with pytest.raises(osvmp2.OSVMP2Error) as ei:
        ctx.localize_pm(C, ls.atom_ao, l_loc=1e-14, max_sweeps=1)
    assert ei.value.code == osvmp2.STATUS_CODES["E_NOCONV"]
    ctx.close()
