"""FP64 CPU oracle for the MBE(3)-OSV-MP2 pair-solve path.

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The product path (``paper_2603_16575_gb300``) never does, and the two share
no code.
"""
from .osv_mp2 import (  # noqa: F401
    semicanonical_tii, osv_from_tii, build_osv, pair_basis, swap_blocks,
    exchange_block, preconditioner, Fragment, FragmentResult, solve_fragment,
    solve_fragment_dense, canonical_mp2_energy, dist2, mbe3_fragments,
    OSVSystem, fragment_gradient, mbe3_energy_gradient,
    fragment_dE_dQ, osv_response, tii_adjoint, mbe3_energy_gradient_relaxed,
    s2b_metric, s2b_matrix, s3b_metric, Screen, screened_fragments, mbe3_diagonal_amplitudes,
    WeakResult, weak_pair, weak_residual, mbe3_screened_energy,
    RandomizedOSV, randomized_osv, build_osv_randomized,
)
from .pm_localization import charge_tensor, pm_functional, PMResult, pm_localize  # noqa: F401,E402
