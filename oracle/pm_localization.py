"""Plain FP64 CPU reference of the Jacobi-sweep Pipek-Mezey localization.

TEST INFRASTRUCTURE ONLY, like the rest of this package: only ``tests/``,
``__graft_entry__.smoke()`` and bench.py's oracle legs may use it; it shares no
code with the CUDA path.

Algorithm 2 of Liang & Yang (arXiv 2603.16575), Section 3.2, step by step:
  U = 1; P^A_ij = sum_{alpha in A} C~_alpha,i C~_alpha,j
  while dL > l_loc:
    dL = 0
    for every pair i < j in order:
      a_ij = sum_A (P^A_ij)^2 - (P^A_ii - P^A_jj)^2 / 4
      b_ij = sum_A P^A_ij (P^A_ii - P^A_jj)                      (Eq. loc_theta)
      theta = atan2(b_ij, -a_ij) / 4                              (reading R19)
      if |sin theta| >= 1e-10:
        dL += sqrt(a^2 + b^2) (1 - cos 4 theta)
        rotate columns i, j of U, then the first and the second MO index of P
The functional is L = sum_{i,A} (P^A_ii)^2.

Reading R19: the paper prints theta = arctan(b / -a) / 4, whose quadrant is
ambiguous; the two-argument form is the branch that maximises L, and the
paper's own dL = sqrt(a^2 + b^2)(1 - cos 4 theta) is the increase of L on that
branch (cos 4 theta = -a / sqrt(a^2 + b^2)).
"""
from __future__ import annotations

import dataclasses

import numpy as np


def charge_tensor(C: np.ndarray, atom_ao: np.ndarray) -> np.ndarray:
    """P[A, i, j] = sum_{alpha in A} C[alpha, i] C[alpha, j] (Algorithm 2, line 2)."""
    n_atom = len(atom_ao) - 1
    n = C.shape[1]
    P = np.empty((n_atom, n, n))
    for A in range(n_atom):
        blk = C[atom_ao[A]:atom_ao[A + 1]]
        P[A] = blk.T @ blk
    return P


def pm_functional(P: np.ndarray) -> float:
    """L = sum_{i, A} (P^A_ii)^2."""
    d = np.einsum("aii->ai", P)
    return float(np.sum(d * d))


@dataclasses.dataclass
class PMResult:
    U: np.ndarray
    L: float
    sweeps: int
    dL_last: float
    converged: bool


def pm_localize(C: np.ndarray, atom_ao: np.ndarray, l_loc: float = 1e-3, max_sweeps: int = 100) -> PMResult:
    """Jacobi-sweep Pipek-Mezey localization of the columns of C (Algorithm 2)."""
    n = C.shape[1]
    U = np.eye(n)
    P = charge_tensor(C, atom_ao)
    dL = np.inf
    sweeps = 0
    while dL > l_loc and sweeps < max_sweeps:
        sweeps += 1
        dL = 0.0
        for i in range(n):
            for j in range(i + 1, n):
                Pij, Pii, Pjj = P[:, i, j], P[:, i, i], P[:, j, j]
                a = float(np.sum(Pij * Pij - 0.25 * (Pii - Pjj) ** 2))
                b = float(np.sum(Pij * (Pii - Pjj)))
                theta = 0.25 * np.arctan2(b, -a)
                s, c = np.sin(theta), np.cos(theta)
                if abs(s) < 1e-10:
                    continue
                dL += np.sqrt(a * a + b * b) * (1.0 - np.cos(4.0 * theta))
                ui, uj = U[:, i].copy(), U[:, j].copy()
                U[:, i], U[:, j] = c * ui + s * uj, c * uj - s * ui
                ri, rj = P[:, i, :].copy(), P[:, j, :].copy()        # first MO index
                P[:, i, :], P[:, j, :] = c * ri + s * rj, c * rj - s * ri
                ci, cj = P[:, :, i].copy(), P[:, :, j].copy()        # second MO index
                P[:, :, i], P[:, :, j] = c * ci + s * cj, c * cj - s * ci
    return PMResult(U, pm_functional(P), sweeps, dL, dL <= l_loc)
