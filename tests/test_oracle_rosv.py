"""Pins of the oracle's randomized OSV generation (Algorithm 3; Eqs. rsvd_z, tsub,
tii_rsvd, back_q, rsvd_za) against exact eigen-decompositions and the range
finder's error bound, with the Gaussian draws passed in as inputs.

* A T of exact rank k: the finder stops after k rows (the look-ahead rows
  vanish once Z spans the range), the singular values equal the eigenvalues and
  Q spans the same space as the exact eigenvectors.
* A semi-canonical T_ii of the synthetic workload: Z has orthonormal rows,
  ||(1 - Z^T Z) T||_2 <= l_osv (the bound the stopping rule l_osv/(10 sqrt(2/pi))
  is chosen for), the kept values lie within that bound of the exact eigenvalues
  and their count matches the exact count (margins checked).
* A stopping threshold without the 10 sqrt(2/pi) factor breaks the bound.
"""
import numpy as np
import pytest

import oracle
import synth


def _rows(seed, i, nv):
    return lambda k: synth.gauss_row(seed, i, k, nv)


def test_exact_rank_is_found_exactly():
    rng = np.random.default_rng(7)
    nv, k = 60, 9
    V, _ = np.linalg.qr(rng.standard_normal((nv, nv)))
    w = np.geomspace(1.0, 1e-3, k)
    T = (V[:, :k] * w) @ V[:, :k].T
    ro = oracle.randomized_osv(T, 1e-4, _rows(3, 0, nv))
    assert ro.n_rosv == k
    assert ro.window_max < 1e-12
    assert np.allclose(np.sort(ro.omega)[::-1], w, rtol=1e-12)
    assert np.abs(ro.Q @ ro.Q.T - V[:, :k] @ V[:, :k].T).max() < 1e-10
    assert np.allclose(ro.Z @ ro.Z.T, np.eye(k), atol=1e-13)


@pytest.mark.parametrize("i", [3, 9])
def test_range_finder_bound_and_counts_on_a_workload_tii(i):
    s = synth.make_system(16, 200, 400, seed=2, lam=1.0)
    T = oracle.semicanonical_tii(s.B_block(i), s.e_vir, s.f_occ[i, i])
    l_osv = 1e-4
    ro = oracle.randomized_osv(T, l_osv, _rows(s.seed, i, s.n_vir))
    Z = ro.Z
    assert np.allclose(Z @ Z.T, np.eye(Z.shape[0]), atol=1e-12)
    err = np.linalg.norm(T - Z.T @ (Z @ T), 2)
    assert err <= l_osv
    lam = np.linalg.eigvalsh(T)[::-1]
    k = int(np.sum(lam >= l_osv))
    margin = np.min(np.abs(lam - l_osv))
    assert margin > err                                    # the count is decided away from the cut
    assert ro.Q.shape[1] == k
    assert np.all(np.abs(ro.omega - lam[:k]) <= err)
    Qe, _ = oracle.osv_from_tii(T, l_osv)
    # kept spaces: the principal angles shrink with the gap below the cut
    c = np.linalg.svd(Qe.T @ ro.Q, compute_uv=False)
    assert c.min() > 1.0 - 1e-2


def test_loose_threshold_breaks_the_bound(monkeypatch):
    s = synth.make_system(16, 200, 400, seed=2, lam=1.0)
    T = oracle.semicanonical_tii(s.B_block(0), s.e_vir, s.f_occ[0, 0])
    l_osv = 1e-4
    # the stopping threshold without the 10 sqrt(2/pi) safety factor
    monkeypatch.setattr(oracle.osv_mp2.np, "sqrt", lambda x: np.float64(1.0 / 10.0) if x == 2.0 / np.pi else np.sqrt(x))
    ro = oracle.randomized_osv(T, l_osv, _rows(s.seed, 0, s.n_vir))
    monkeypatch.undo()
    good = oracle.randomized_osv(T, l_osv, _rows(s.seed, 0, s.n_vir))
    assert ro.n_rosv < good.n_rosv
    assert np.linalg.norm(T - ro.Z.T @ (ro.Z @ T), 2) > np.linalg.norm(T - good.Z.T @ (good.Z @ T), 2)
