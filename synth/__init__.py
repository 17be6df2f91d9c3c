"""Seeded synthetic inputs for the MBE(3)-OSV-MP2 pair-solve path.

This module only *produces inputs*; it holds none of the method's arithmetic
(no amplitudes, no OSVs, no integrals beyond the raw three-index tensor B).
Both the FP64 CPU oracle and the CUDA path take their inputs from here; the
CUDA path additionally regenerates B on the device from the same counter-based
definition, written independently in CUDA.

Generator definition (the bit-level contract both implementations follow)
-------------------------------------------------------------------------
* ``mix64`` is the SplitMix64 output finaliser (Steele, Lea & Flood, OOPSLA
  2014; Vigna's reference ``splitmix64.c``)::

      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
      z = (z ^ (z >> 27)) * 0x94D049BB133111EB
      z =  z ^ (z >> 31)                         (all mod 2**64)

* a *stream key* is ``key(seed, s) = mix64(seed ^ (s * 0xD1B54A32D192ED03))``;
  draw number ``c`` of a stream is ``u64(key, c) = mix64(key + (c+1)*GAMMA)``
  with ``GAMMA = 0x9E3779B97F4A7C15`` -- i.e. the c-th SplitMix64 output of a
  generator whose state starts at ``key``.
* uniform on [0,1): ``(u64 >> 11) * 2**-53``.
* standard-normal stand-in: Irwin--Hall sum of twelve 16-bit uniforms taken
  from three consecutive draws ``3c, 3c+1, 3c+2``::

      S = sum of the four 16-bit fields of each of the three draws (integer)
      z = (S - 393210) * 2**-16

  mean 0, variance 1 - 2**-32, support [-6, 6]. Every step is exact in
  integer arithmetic and one exact FP64 scaling, so CPU and GPU agree bit for
  bit.
* ``B[i,a,P] = env[i,a] * z(key(seed, S_B), (i*n_vir + a)*n_aux + P)`` -- one
  correctly rounded FP64 product. ``env[i,a] = scale * exp(-|r_i - r_a| / lam)``
  is an input table computed here on the host and handed to the device as is.

System recipe (water-cluster-like box, or peptide-like chain)
-------------------------------------------------------------
* box: centres uniform in a cube of edge ``L = 10 A * (n_occ/20)**(1/3)``
  (constant density; 10 A at n_occ = 20), occupied and virtual centres alike.
* chain: ``r_i = (spacing*i, 0, 0)``; virtual ``a`` sits at site ``a mod n_occ``
  plus an isotropic jitter of ``0.7 A * z``.
* occupied energies U[-1.5, -0.3] Eh, virtual energies U[0.1, 5.0] Eh.
* occupied Fock: ``f_ii = e_i``; ``f_ij = 1e-2 * exp(-d_ij / 2 A)`` for i != j.
"""
from __future__ import annotations

import dataclasses
import numpy as np

GAMMA = 0x9E3779B97F4A7C15
STREAM_MUL = 0xD1B54A32D192ED03
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB

# stream ids
S_OCC_POS, S_VIR_POS, S_OCC_E, S_VIR_E, S_B, S_JITTER, S_ROSV = 1, 2, 3, 4, 5, 6, 7
# rows of the randomized OSV draws per orbital (counter layout of gauss_rows)
ROSV_ROWS_PER_ORBITAL = 1 << 16

_U64 = np.uint64
_MASK = (1 << 64) - 1


def mix64_int(z: int) -> int:
    """SplitMix64 finaliser on a Python int (reference scalar form)."""
    z &= _MASK
    z = ((z ^ (z >> 30)) * MIX1) & _MASK
    z = ((z ^ (z >> 27)) * MIX2) & _MASK
    return z ^ (z >> 31)


def stream_key(seed: int, stream: int) -> int:
    return mix64_int((seed & _MASK) ^ ((stream * STREAM_MUL) & _MASK))


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser, vectorised over a uint64 array (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = z.astype(_U64, copy=True)
        z ^= z >> _U64(30)
        z *= _U64(MIX1)
        z ^= z >> _U64(27)
        z *= _U64(MIX2)
        z ^= z >> _U64(31)
    return z


def draws(key: int, ctr: np.ndarray) -> np.ndarray:
    """u64(key, c) for every counter c in ``ctr`` (uint64 array)."""
    with np.errstate(over="ignore"):
        state = _U64(key) + (ctr.astype(_U64) + _U64(1)) * _U64(GAMMA)
    return mix64(state)


def uniform(key: int, ctr: np.ndarray) -> np.ndarray:
    return (draws(key, ctr) >> _U64(11)).astype(np.float64) * (2.0 ** -53)


def normal_ih12(key: int, ctr: np.ndarray) -> np.ndarray:
    """Irwin--Hall(12) standard-normal stand-in for each counter in ``ctr``."""
    ctr = np.asarray(ctr, dtype=_U64)
    s = np.zeros(ctr.shape, dtype=np.int64)
    m16 = _U64(0xFFFF)
    for t in range(3):
        with np.errstate(over="ignore"):
            h = draws(key, ctr * _U64(3) + _U64(t))
        for sh in (0, 16, 32, 48):
            s += ((h >> _U64(sh)) & m16).astype(np.int64)
    return (s - 393210).astype(np.float64) * (2.0 ** -16)


@dataclasses.dataclass
class System:
    """One synthetic closed-shell system (all arrays FP64, row-major).

    Shapes: r_occ (n_occ,3) A, r_vir (n_vir,3) A, e_occ (n_occ,),
    f_occ (n_occ,n_occ) symmetric, e_vir (n_vir,), env (n_occ,n_vir).
    """
    n_occ: int
    n_vir: int
    n_aux: int
    seed: int
    lam: float
    scale: float
    geometry: str
    r_occ: np.ndarray
    r_vir: np.ndarray
    e_occ: np.ndarray
    f_occ: np.ndarray
    e_vir: np.ndarray
    env: np.ndarray

    @property
    def b_key(self) -> int:
        return stream_key(self.seed, S_B)

    def B_block(self, i: int) -> np.ndarray:
        """B[i,:,:] of shape (n_vir, n_aux)."""
        nv, nx = self.n_vir, self.n_aux
        base = (i * nv) * nx
        ctr = np.arange(nv * nx, dtype=_U64) + _U64(base)
        z = normal_ih12(self.b_key, ctr).reshape(nv, nx)
        return self.env[i][:, None] * z

    def B_entry(self, i: int, a: int, p: int) -> float:
        c = np.array([(i * self.n_vir + a) * self.n_aux + p], dtype=_U64)
        return float(self.env[i, a] * normal_ih12(self.b_key, c)[0])

    def B_full(self) -> np.ndarray:
        out = np.empty((self.n_occ, self.n_vir, self.n_aux))
        for i in range(self.n_occ):
            out[i] = self.B_block(i)
        return out


def _pairwise_dist(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    d = a[:, None, :] - b[None, :, :]
    return np.sqrt(np.sum(d * d, axis=-1))


def make_system(n_occ: int, n_vir: int, n_aux: int, seed: int = 0, lam: float = 3.0,
                scale: float = 0.1, geometry: str = "box", box_edge: float | None = None,
                spacing: float = 1.5, f_off: float = 1e-2, f_len: float = 2.0,
                jitter: float = 0.7) -> System:
    """Build the seeded synthetic system described in the module docstring."""
    if geometry == "box":
        L = box_edge if box_edge is not None else 10.0 * (n_occ / 20.0) ** (1.0 / 3.0)
        r_occ = L * uniform(stream_key(seed, S_OCC_POS), np.arange(3 * n_occ)).reshape(n_occ, 3)
        r_vir = L * uniform(stream_key(seed, S_VIR_POS), np.arange(3 * n_vir)).reshape(n_vir, 3)
    elif geometry == "chain":
        r_occ = np.zeros((n_occ, 3))
        r_occ[:, 0] = spacing * np.arange(n_occ)
        site = np.arange(n_vir) % n_occ
        jit = normal_ih12(stream_key(seed, S_JITTER), np.arange(3 * n_vir, dtype=_U64)).reshape(n_vir, 3)
        r_vir = r_occ[site] + jitter * jit
    else:
        raise ValueError(f"unknown geometry {geometry!r}")
    e_occ = -1.5 + 1.2 * uniform(stream_key(seed, S_OCC_E), np.arange(n_occ))
    e_vir = 0.1 + 4.9 * uniform(stream_key(seed, S_VIR_E), np.arange(n_vir))
    d_oo = _pairwise_dist(r_occ, r_occ)
    f_occ = f_off * np.exp(-d_oo / f_len)
    np.fill_diagonal(f_occ, e_occ)
    env = scale * np.exp(-_pairwise_dist(r_occ, r_vir) / lam)
    return System(n_occ, n_vir, n_aux, seed, lam, scale, geometry,
                  np.ascontiguousarray(r_occ), np.ascontiguousarray(r_vir), e_occ,
                  np.ascontiguousarray(f_occ), e_vir, np.ascontiguousarray(env))


# Named workloads: shapes of the paper-scale synthetic cases. ``lam`` is the
# envelope length of B; 3.0 A is the literal recipe, 1.0 A the calibrated one
# that yields 20-70 OSVs per orbital at l_osv = 1e-4.
WORKLOADS = {
    "canonical_n20": dict(n_occ=20, n_vir=100, n_aux=400, lam=3.0, geometry="box"),
    "osv_n256": dict(n_occ=256, n_vir=1200, n_aux=4800, lam=1.0, geometry="box"),
    "mbe3_n128": dict(n_occ=128, n_vir=640, n_aux=2400, lam=1.0, geometry="box"),
    "mbe3_n32": dict(n_occ=32, n_vir=160, n_aux=600, lam=1.0, geometry="box"),
    # the per-orbital shapes of mbe3_n128 on fewer orbitals (kernel captures of a few GB)
    "mbe3_n48": dict(n_occ=48, n_vir=640, n_aux=2400, lam=1.0, geometry="box"),
    "grad_n64": dict(n_occ=64, n_vir=320, n_aux=1200, lam=1.0, geometry="box"),
    "chain_n800": dict(n_occ=800, n_vir=6000, n_aux=16000, lam=1.0, geometry="chain"),
}


def gauss_row(seed: int, i: int, k: int, n_vir: int) -> np.ndarray:
    """Row k of the Gaussian draws of orbital i for the randomized OSV range
    finder: z(key(seed, S_ROSV), (i * 2^16 + k) * n_vir + a), a = 0..n_vir-1,
    the Irwin-Hall(12) normal defined above.  The device draws the same numbers
    from the same definition."""
    base = (i * ROSV_ROWS_PER_ORBITAL + k) * n_vir
    return normal_ih12(stream_key(seed, S_ROSV), np.arange(n_vir, dtype=_U64) + _U64(base))


S_LOC, S_ROT = 8, 9


@dataclasses.dataclass
class LocSystem:
    """Delocalized orthonormal orbitals for the localization step: C = L R with L
    orthonormal orbitals each mostly on its own atom (the target of the
    localization) and R a Haar-random orthogonal mixing.  C is [n_ao, n_occ]
    with n_ao = ao_per_atom * n_atom; atom_ao are the AO offsets of the atoms."""
    C: np.ndarray
    L: np.ndarray
    atom_ao: np.ndarray
    r_atom: np.ndarray


def make_loc_system(n_occ: int, ao_per_atom: int = 4, seed: int = 0, tail: float = 0.3,
                    decay: float = 1.5) -> LocSystem:
    """n_occ atoms in the water-cluster box (constant density), one localized
    orbital per atom: its own AOs carry Irwin-Hall(12) normal weights, the AOs of
    other atoms tail * exp(-d / decay) times normal weights; orthonormalised by QR
    (input preparation), then mixed by a Haar rotation (QR of a normal matrix with
    the signs of R's diagonal fixed)."""
    n_atom = n_occ
    n_ao = ao_per_atom * n_atom
    L_box = 10.0 * (n_occ / 20.0) ** (1.0 / 3.0)
    r = L_box * uniform(stream_key(seed, S_OCC_POS), np.arange(3 * n_atom)).reshape(n_atom, 3)
    d = _pairwise_dist(r, r)
    z = normal_ih12(stream_key(seed, S_LOC), np.arange(n_ao * n_occ, dtype=_U64)).reshape(n_ao, n_occ)
    atom_of_ao = np.repeat(np.arange(n_atom), ao_per_atom)
    env = tail * np.exp(-d[atom_of_ao, :] / decay)
    env[atom_of_ao[:, None] == np.arange(n_occ)[None, :]] = 1.0
    Lmat, R0 = np.linalg.qr(z * env)
    Lmat = Lmat * np.sign(np.diag(R0))[None, :]
    g = normal_ih12(stream_key(seed, S_ROT), np.arange(n_occ * n_occ, dtype=_U64)).reshape(n_occ, n_occ)
    Qr, Rr = np.linalg.qr(g)
    Qr = Qr * np.sign(np.diag(Rr))[None, :]
    C = Lmat @ Qr
    return LocSystem(np.ascontiguousarray(C), np.ascontiguousarray(Lmat),
                     np.arange(0, n_ao + 1, ao_per_atom, dtype=np.int32), r)


def workload(name: str, seed: int = 0, **over) -> System:
    kw = dict(WORKLOADS[name])
    kw.update(over)
    return make_system(seed=seed, **kw)
