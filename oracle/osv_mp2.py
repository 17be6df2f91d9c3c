"""Plain FP64 CPU reference of the MBE(3)-OSV-MP2 pair-solve path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module; only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA path (the only shared module is ``synth``, which makes
the seeded inputs and holds none of the method's arithmetic).

Everything is NumPy FP64 with LAPACK ``eigh`` and BLAS GEMM as the only library
steps, written in the order and notation of Liang & Yang, "Multi-GPU
MBE(3)-OSV-MP2" (arXiv 2603.16575):

* OSV generation -- Eq. (osv_gen) with the semi-canonical diagonal amplitudes
  of Eq. (mp2_tkk); selection ``omega >= l_osv`` as in Algorithm 3.
* 4-block OSV pair matrices -- Eq. (4block_osv); exchange blocks from the
  OSV-projected three-index integrals, Eqs. (osv_imua) and (osv_close_k).
* preconditioner -- the generalized eigenproblem Eq. (prec_eig).
* residual -- Eq. (res_close); amplitude update and pair energy as in
  Algorithm 7 (close clusters) with the energy expression of Section 2.
* MBE(3) -- the amplitude expansion Eqs. (tmbediag)-(deltaoff) collected into
  inclusion-exclusion weights on the fragment energies.
* gradient -- Hellmann-Feynman derivative of the Hylleraas functional that
  Eq. (res_close) makes stationary (Section 2), with the OSVs held fixed; the
  OSV-relaxed form adds the first-order response of the kept eigenvectors of
  Eq. (osv_gen) to T_ii of Eq. (mp2_tkk).

Readings where the paper is silent or garbled (each one is listed, with its
reason, in the design notes):
  R1  energy ``<K(2T - T^+)>`` is the Frobenius product sum_ab K^ab(2T^ab - T^ba)
  R2  the right factor of Eq. (osv_close_k) takes its columns from LMO j
  R3  the update divides element-wise by D_mn = f_ii + f_jj - e~_m - e~_n
  R4  T_ii of Eq. (mp2_tkk) uses the positive denominator e_a + e_b - 2 f_ii
  R5  convergence on |dE| and max|update| (no l_mp2e value is printed)
  R6  all pairs of a fragment are updated from the previous sweep (Jacobi)
  R7  a singular S_(ij,ij) is handled by canonical orthogonalisation
      (eigenvalues below tau_s * max dropped) instead of Cholesky
  R8  the diagonal pair basis is P_ii = Q_i (one block)
  R9  OSVs are kept when omega >= l_osv, ordered by descending omega, each
      eigenvector signed so its largest-magnitude entry is positive
  R10 fragments: pairs with d^2 <= r2^2, triples whose three pairs all satisfy
      d^2 <= r3^2 (and are kept pairs); squared distances summed x, y, z in order
  R16 screened clusters: close pairs s2b >= 1e-2, weak 1e-7 <= s2b < 1e-2; a
      triple is a candidate only when its three pairs are close, kept when
      s3b >= 0.2 (keeps the cluster list closed under subsets)
  R17 the garbled weak-pair residual, Eq. (res_weak), is read as
      K + F_(i,i) T + T F_(j,j) - (f_ii + f_jj) T - f_ij [T_(i,i) S_(i,j) + S_(i,j) T_(j,j)]
      (the full residual projected onto Q_i x Q_j with k restricted to {i, j})
  R18 weak-pair energy: 2 <K_(i,j), T_(i,j)> per ordered pair, both orders
      counted, with T_(i,i) the MBE(3) diagonal amplitude of Eq. (tmbediag)
  R23 the OSV-relaxed gradient (named as future work in the conclusions) is the
      derivative with every orbital's OSV count held fixed: the truncated energy
      jumps where an eigenvalue of T_ii crosses l_osv, and the response term
      scales with 1 / (eigenvalue gap at the cut), which is reported
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Dict, List, Sequence, Tuple

import numpy as np

Pair = Tuple[int, int]


# --------------------------------------------------------------------------
# OSV generation: Eq. (mp2_tkk) and Eq. (osv_gen)
# --------------------------------------------------------------------------
def semicanonical_tii(B_i: np.ndarray, e_vir: np.ndarray, f_ii: float) -> np.ndarray:
    """T_ii^{ab} = sum_A B_ia^A B_ib^A / (e_a + e_b - 2 f_ii)   (Eq. mp2_tkk, reading R4)."""
    G = B_i @ B_i.T
    den = e_vir[:, None] + e_vir[None, :] - 2.0 * f_ii
    return G / den


def osv_from_tii(T_ii: np.ndarray, l_osv: float) -> Tuple[np.ndarray, np.ndarray]:
    """Eigenvectors of T_ii with omega >= l_osv (all if l_osv <= 0), Eq. (osv_gen).

    Returns (Q_i [n_vir, n_i], omega_i [n_i]) in descending omega order with the
    sign convention of reading R9.
    """
    w, V = np.linalg.eigh(T_ii)
    order = np.argsort(-w, kind="stable")
    w, V = w[order], V[:, order]
    if l_osv > 0:
        keep = w >= l_osv
        w, V = w[keep], V[:, keep]
    if V.shape[1]:
        big = np.argmax(np.abs(V), axis=0)
        sgn = np.sign(V[big, np.arange(V.shape[1])])
        sgn[sgn == 0] = 1.0
        V = V * sgn
    return np.ascontiguousarray(V), w


def build_osv(Bfun: Callable[[int], np.ndarray], n_occ: int, e_vir: np.ndarray,
              f_occ: np.ndarray, l_osv: float, orbitals=None) -> Tuple[List, List]:
    """OSVs of every occupied orbital (Algorithm 3's output, by exact eigh);
    with ``orbitals`` only those entries are built (the rest stay None)."""
    Q, W = [None] * n_occ, [None] * n_occ
    for i in (range(n_occ) if orbitals is None else orbitals):
        Q[i], W[i] = osv_from_tii(semicanonical_tii(Bfun(i), e_vir, f_occ[i, i]), l_osv)
    return Q, W


# --------------------------------------------------------------------------
# Pair quantities: Eq. (4block_osv), Eq. (osv_imua), Eq. (osv_close_k)
# --------------------------------------------------------------------------
def pair_basis(Q: Sequence[np.ndarray], i: int, j: int) -> np.ndarray:
    """P_ij = [Q_i Q_j] for i != j (either order); P_ii = Q_i (reading R8)."""
    return Q[i] if i == j else np.hstack([Q[i], Q[j]])


def swap_blocks(M: np.ndarray, n_first: int) -> np.ndarray:
    """Re-express a matrix over [Q_i Q_j] in the basis [Q_j Q_i] (rows and columns)."""
    perm = np.r_[np.arange(n_first, M.shape[0]), np.arange(n_first)]
    return M[np.ix_(perm, perm)]


def exchange_block(P: np.ndarray, B_i: np.ndarray, B_j: np.ndarray) -> np.ndarray:
    """K_(ij,ij) = [Q_i Q_j]^T (B_i B_j^T) [Q_i Q_j] via the projected integrals.

    The projections P^T B_x are the OSV half-transformed integrals of
    Eq. (osv_imua); rows of K come from LMO i and columns from LMO j (R2).
    """
    Li = P.T @ B_i
    Lj = P.T @ B_j
    return Li @ Lj.T


def preconditioner(S: np.ndarray, F: np.ndarray, tau_s: float) -> Tuple[np.ndarray, np.ndarray]:
    """Solve F X = S X E~ (Eq. prec_eig) with X^T S X = 1 (reading R7)."""
    s, U = np.linalg.eigh(S)
    keep = s > tau_s * s.max()
    Y = U[:, keep] / np.sqrt(s[keep])
    e_t, W = np.linalg.eigh(Y.T @ F @ Y)
    return Y @ W, e_t


# --------------------------------------------------------------------------
# One fragment (MBE cluster): Eq. (res_close) and Algorithm 7
# --------------------------------------------------------------------------
@dataclasses.dataclass
class FragmentResult:
    orbs: Tuple[int, ...]
    energy: float
    pair_energy: Dict[Pair, float]      # per stored pair i <= j, i != j counted twice
    T: Dict[Pair, np.ndarray]           # converged amplitudes in the basis P_ij, i <= j
    iterations: int
    max_update: float
    converged: bool


class Fragment:
    """All pair matrices of one fragment, built from the dense definitions."""

    def __init__(self, orbs: Sequence[int], Q: Sequence[np.ndarray],
                 Bfun: Callable[[int], np.ndarray], f_occ: np.ndarray,
                 e_vir: np.ndarray, tau_s: float = 1e-10):
        self.orbs = tuple(sorted(orbs))
        self.f = f_occ
        self.n = {i: Q[i].shape[1] for i in self.orbs}
        o = self.orbs
        self.ordered = [(i, j) for i in o for j in o]
        self.pairs = [(i, j) for a, i in enumerate(o) for j in o[a:]]
        self.P = {p: pair_basis(Q, *p) for p in self.ordered}
        B = {i: Bfun(i) for i in o}
        # blocks Q_x^T Q_y and Q_x^T diag(e) Q_y; S_(ij,kl), F_(ij,kl) are assembled
        # from them in the 4-block form of Eq. (4block_osv)
        self.Sb = {(x, y): Q[x].T @ Q[y] for x in o for y in o}
        self.Fb = {(x, y): Q[x].T @ (e_vir[:, None] * Q[y]) for x in o for y in o}
        self._cache = len(o) <= 4
        self._S: Dict = {}
        self._F: Dict = {}
        self.K = {p: exchange_block(self.P[p], B[p[0]], B[p[1]]) for p in self.pairs}
        self.X, self.Et = {}, {}
        for p in self.pairs:
            self.X[p], self.Et[p] = preconditioner(self.S(p, p), self.F(p, p), tau_s)

    @staticmethod
    def _blocks(p: Pair) -> Tuple[int, ...]:
        return (p[0],) if p[0] == p[1] else p

    def _assemble(self, blk, store, p: Pair, q: Pair) -> np.ndarray:
        if (p, q) in store:
            return store[p, q]
        M = np.block([[blk[(a, c)] for c in self._blocks(q)] for a in self._blocks(p)])
        if self._cache:
            store[p, q] = M
        return M

    def S(self, p: Pair, q: Pair) -> np.ndarray:
        """S_(p,q) = P_p^T P_q (Eq. 4block_osv with A = overlap)."""
        return self._assemble(self.Sb, self._S, p, q)

    def F(self, p: Pair, q: Pair) -> np.ndarray:
        """F_(p,q) = P_p^T diag(e_vir) P_q (Eq. 4block_osv with A = Fock)."""
        return self._assemble(self.Fb, self._F, p, q)

    def ordered_amp(self, T: Dict[Pair, np.ndarray], i: int, k: int) -> np.ndarray:
        """T_(ik,ik) in the basis [Q_i Q_k]; for i > k from the stored T_(ki) (T_ik = T_ki^T)."""
        if i <= k:
            return T[(i, k)]
        return swap_blocks(T[(k, i)].T, self.n[k])

    def residual(self, T: Dict[Pair, np.ndarray], p: Pair) -> np.ndarray:
        """R_(ij,ij) of Eq. (res_close) with k running over the fragment's LMOs."""
        i, j = p
        f = self.f
        R = self.K[p].copy()
        for k in self.orbs:
            ik, kj = (i, k), (k, j)
            left = self.S(p, ik) @ self.ordered_amp(T, i, k)
            bracket = -f[k, j] * self.S(ik, p)
            if k == j:
                bracket = bracket + self.F(ik, p)
            R += left @ bracket
            bracket = -f[i, k] * self.S(p, kj)
            if i == k:
                bracket = bracket + self.F(p, kj)
            R += bracket @ self.ordered_amp(T, k, j) @ self.S(kj, p)
        return R

    def pair_energy(self, T: Dict[Pair, np.ndarray], p: Pair) -> float:
        """<K_(ij,ij), 2T - T^T> (reading R1), doubled for i != j (both orders)."""
        Tp = T[p]
        e = float(np.sum(self.K[p] * (2.0 * Tp - Tp.T)))
        return e if p[0] == p[1] else 2.0 * e

    def energy(self, T: Dict[Pair, np.ndarray]) -> float:
        return float(sum(self.pair_energy(T, p) for p in self.pairs))


def solve_fragment(frag: Fragment, tol: float = 1e-7, e_tol: float = 1e-14,
                   max_iter: int = 500) -> FragmentResult:
    """Algorithm 7 (close clusters): R, R~ = X^T R X, T += X (R~ / D) X^T, E.

    All pairs are updated from the previous sweep's amplitudes (reading R6);
    the loop stops when max|R~/D| < tol and |dE| < e_tol (reading R5).
    """
    T = {p: np.zeros((frag.P[p].shape[1],) * 2) for p in frag.pairs}
    e_last = 0.0
    upd = np.inf
    for it in range(1, max_iter + 1):
        R = {p: frag.residual(T, p) for p in frag.pairs}
        upd = 0.0
        for p in frag.pairs:
            i, j = p
            X, et = frag.X[p], frag.Et[p]
            D = frag.f[i, i] + frag.f[j, j] - et[:, None] - et[None, :]
            Y = (X.T @ R[p] @ X) / D
            T[p] = T[p] + X @ Y @ X.T
            upd = max(upd, float(np.max(np.abs(Y))) if Y.size else 0.0)
        e_cur = frag.energy(T)
        if upd < tol and abs(e_cur - e_last) < e_tol:
            return _result(frag, T, it, upd, True)
        e_last = e_cur
    return _result(frag, T, max_iter, upd, False)


def _result(frag, T, it, upd, ok):
    pe = {p: frag.pair_energy(T, p) for p in frag.pairs}
    return FragmentResult(frag.orbs, float(sum(pe.values())), pe, T, it, upd, ok)


def solve_fragment_dense(frag: Fragment) -> FragmentResult:
    """Brute force: assemble the linear operator of X^T R(T) X = 0 in the
    preconditioner bases and solve it with dense LU (tiny fragments only)."""
    sizes = [frag.X[p].shape[1] for p in frag.pairs]
    offs = np.cumsum([0] + [r * r for r in sizes])
    N = int(offs[-1])

    def unpack(v):
        return {p: frag.X[p] @ v[offs[a]:offs[a + 1]].reshape(sizes[a], sizes[a]) @ frag.X[p].T
                for a, p in enumerate(frag.pairs)}

    def project(Rd):
        return np.concatenate([(frag.X[p].T @ Rd[p] @ frag.X[p]).ravel() for p in frag.pairs])

    zero = {p: np.zeros((frag.P[p].shape[1],) * 2) for p in frag.pairs}
    b = project({p: frag.residual(zero, p) for p in frag.pairs})     # = X^T K X
    A = np.empty((N, N))
    for c in range(N):
        e = np.zeros(N)
        e[c] = 1.0
        Tc = unpack(e)
        A[:, c] = project({p: frag.residual(Tc, p) for p in frag.pairs}) - b
    y = np.linalg.solve(A, -b)
    T = unpack(y)
    return _result(frag, T, 1, 0.0, True)


# --------------------------------------------------------------------------
# Closed form: canonical RI-MP2, Eq. (mp2_tmat) with the energy of Section 2
# --------------------------------------------------------------------------
def canonical_mp2_energy(Bfun: Callable[[int], np.ndarray], n_occ: int,
                         f_occ: np.ndarray, e_vir: np.ndarray) -> float:
    """sum_ijab (ia|jb)[2(ia|jb) - (ib|ja)] / (e_i + e_j - e_a - e_b) after
    diagonalising the occupied Fock block (f = U eps U^T, B'_k = sum_i U_ik B_i)."""
    eps, U = np.linalg.eigh(f_occ)
    Bs = np.stack([Bfun(i) for i in range(n_occ)])
    Bc = np.einsum("ik,iaP->kaP", U, Bs)
    E = 0.0
    for i in range(n_occ):
        for j in range(n_occ):
            K = Bc[i] @ Bc[j].T
            D = eps[i] + eps[j] - e_vir[:, None] - e_vir[None, :]
            E += float(np.sum(K * (2.0 * K - K.T) / D))
    return E


# --------------------------------------------------------------------------
# MBE(3): Eqs. (tmbediag), (tmbeoff), (deltaoff) as fragment weights
# --------------------------------------------------------------------------
def dist2(r: np.ndarray, i: int, j: int) -> float:
    dx = float(r[i, 0]) - float(r[j, 0])
    dy = float(r[i, 1]) - float(r[j, 1])
    dz = float(r[i, 2]) - float(r[j, 2])
    return dx * dx + dy * dy + dz * dz


def mbe3_fragments(r_occ: np.ndarray, r2: float, r3: float):
    """Kept 1-, 2- and 3-body clusters (reading R10) and their weights.

    Weights follow from expanding the amplitudes as in Eqs. (tmbediag) and
    (tmbeoff): c_ijk = 1, c_ij = 1 - #triples containing ij,
    c_i = 1 - #pairs containing i + #triples containing i.
    Returns a list of (orbs tuple, weight) in the order singles, pairs, triples
    (each lexicographic).
    """
    n = r_occ.shape[0]
    c2, c3 = r2 * r2, r3 * r3
    d2 = np.array([[dist2(r_occ, i, j) for j in range(n)] for i in range(n)])
    pairs = [(i, j) for i in range(n) for j in range(i + 1, n) if d2[i, j] <= c2]
    ok3 = (d2 <= c3) & (d2 <= c2)
    triples = [(i, j, k) for i in range(n) for j in range(i + 1, n) if ok3[i, j]
               for k in range(j + 1, n) if ok3[i, k] and ok3[j, k]]
    tri_per_pair: Dict[Pair, int] = {}
    tri_per_orb = np.zeros(n, dtype=np.int64)
    pair_per_orb = np.zeros(n, dtype=np.int64)
    for (i, j) in pairs:
        pair_per_orb[i] += 1
        pair_per_orb[j] += 1
    for (i, j, k) in triples:
        for p in ((i, j), (i, k), (j, k)):
            tri_per_pair[p] = tri_per_pair.get(p, 0) + 1
        for x in (i, j, k):
            tri_per_orb[x] += 1
    frags = [((i,), int(1 - pair_per_orb[i] + tri_per_orb[i])) for i in range(n)]
    frags += [((i, j), int(1 - tri_per_pair.get((i, j), 0))) for (i, j) in pairs]
    frags += [(t, 1) for t in triples]
    return frags


class OSVSystem:
    """Oracle-side state of one system: inputs plus OSVs."""

    def __init__(self, Bfun: Callable[[int], np.ndarray], n_occ: int, e_vir: np.ndarray,
                 f_occ: np.ndarray, l_osv: float, tau_s: float = 1e-10, cache_B: bool = True,
                 orbitals=None):
        self._B: Dict[int, np.ndarray] = {}
        self._Bsrc = Bfun
        self.cache = cache_B
        self.n_occ = n_occ
        self.e_vir = np.asarray(e_vir, dtype=np.float64)
        self.f_occ = np.asarray(f_occ, dtype=np.float64)
        self.tau_s = tau_s
        self.Q, self.omega = build_osv(self.B, n_occ, self.e_vir, self.f_occ, l_osv, orbitals)

    def B(self, i: int) -> np.ndarray:
        if i in self._B:
            return self._B[i]
        b = self._Bsrc(i)
        if self.cache:
            self._B[i] = b
        return b

    def fragment(self, orbs: Sequence[int]) -> Fragment:
        return Fragment(orbs, self.Q, self.B, self.f_occ, self.e_vir, self.tau_s)

    def solve(self, orbs: Sequence[int], **kw) -> FragmentResult:
        return solve_fragment(self.fragment(orbs), **kw)

    def mbe3_energy(self, r_occ: np.ndarray, r2: float, r3: float, **kw):
        frags = mbe3_fragments(r_occ, r2, r3)
        E = 0.0
        per = []
        for orbs, c in frags:
            res = self.solve(orbs, **kw)
            per.append((orbs, c, res.energy))
            E += c * res.energy
        return E, per


# --------------------------------------------------------------------------
# Gradient with frozen OSVs (Hellmann-Feynman on the Hylleraas functional)
# --------------------------------------------------------------------------
def fragment_gradient(frag: Fragment, res: FragmentResult, Bfun: Callable[[int], np.ndarray],
                      n_occ: int, n_vir: int, n_aux: int):
    """dE_C/dB (dict i -> [n_vir, n_aux]), dE_C/de_vir [n_vir], dE_C/df [n_occ, n_occ].

    With T stationary, E_C equals the Hylleraas functional
    sum_ij <T~_ij, 2 K_ij + (F T_ij + T_ij F - sum_k f_ik T_kj + f_kj T_ik)>,
    T~ = 2T - T^T, over ordered pairs in the full virtual space, whose explicit
    derivatives are
      dE/dB_i   = 4 sum_j T~_ij B_j
      dE/de_a   = 2 sum_ij sum_b T~_ij^ab T_ij^ab
      dE/df_kl  = -sum_j <T~_kj, T_lj> - sum_i <T~_il, T_ik>   (then symmetrised)
    """
    o = frag.orbs
    Tf = {}
    for (i, j) in frag.pairs:
        full = frag.P[(i, j)] @ res.T[(i, j)] @ frag.P[(i, j)].T
        Tf[(i, j)] = full
        Tf[(j, i)] = full.T
    Tt = {p: 2.0 * Tf[p] - Tf[p].T for p in Tf}
    dB = {i: 4.0 * sum(Tt[(i, j)] @ Bfun(j) for j in o) for i in o}
    de = np.zeros(n_vir)
    for p in Tf:
        de += 2.0 * np.sum(Tt[p] * Tf[p], axis=1)
    G = np.zeros((n_occ, n_occ))
    for k in o:
        for l in o:
            g = 0.0
            for j in o:
                g -= float(np.sum(Tt[(k, j)] * Tf[(l, j)]))
            for i in o:
                g -= float(np.sum(Tt[(i, l)] * Tf[(i, k)]))
            G[k, l] = g
    return dB, de, 0.5 * (G + G.T)


def mbe3_energy_gradient(osys: OSVSystem, r_occ: np.ndarray, r2: float, r3: float,
                         n_vir: int, n_aux: int, **kw):
    """E, dE/dB [n_occ,n_vir,n_aux], dE/de_vir, dE/df (symmetrised) for MBE(3)."""
    n = osys.n_occ
    dB = np.zeros((n, n_vir, n_aux))
    de = np.zeros(n_vir)
    df = np.zeros((n, n))
    E = 0.0
    for orbs, c in mbe3_fragments(r_occ, r2, r3):
        if c == 0:
            continue
        frag = osys.fragment(orbs)
        res = solve_fragment(frag, **kw)
        E += c * res.energy
        gB, ge, gf = fragment_gradient(frag, res, osys.B, n, n_vir, n_aux)
        for i, v in gB.items():
            dB[i] += c * v
        de += c * ge
        df += c * gf
    return E, dB, de, df


# --------------------------------------------------------------------------
# OSV-relaxed gradient: the frozen-OSV derivative plus the response of the
# OSVs of Eq. (osv_gen) to T_ii of Eq. (mp2_tkk) (reading R23)
# --------------------------------------------------------------------------
def fragment_dE_dQ(frag: Fragment, res: FragmentResult, Bfun: Callable[[int], np.ndarray],
                   e_vir: np.ndarray) -> Dict[int, np.ndarray]:
    """dE_C/dQ_x [n_vir, n_x] for every LMO x of the fragment, B, e and f fixed.

    With the amplitudes stationary, E_C is the Hylleraas functional of the
    frozen-OSV gradient with T_ij(full) = P_ij T_ij P_ij^T, and its variation
    in the full amplitudes is dE = 2 sum_(ordered ij) <dT_ij, R~_ij>, where
    R_ij = B_i B_j^T + diag(e) T_ij + T_ij diag(e) - sum_k (f_ik T_kj + f_kj T_ik)
    is the full-space residual of Eq. (res_close) and R~ = 2R - R^T.  Both
    orders of a pair i < j give the same term (R_ji = R_ij^T), so per stored
    pair dE = alpha <R~ P T^T + R~^T P T, dP> with alpha = 4 (i < j) or 2
    (i = j), and the columns of dP that belong to Q_x are dQ_x.
    """
    o = frag.orbs
    e = np.asarray(e_vir, dtype=np.float64)
    Tf = {}
    for (i, j) in frag.pairs:
        full = frag.P[(i, j)] @ res.T[(i, j)] @ frag.P[(i, j)].T
        Tf[(i, j)] = full
        Tf[(j, i)] = full.T
    B = {x: Bfun(x) for x in o}
    G = {x: np.zeros((e.size, frag.n[x])) for x in o}
    for (i, j) in frag.pairs:
        R = B[i] @ B[j].T + e[:, None] * Tf[(i, j)] + Tf[(i, j)] * e[None, :]
        for k in o:
            R -= frag.f[i, k] * Tf[(k, j)] + frag.f[k, j] * Tf[(i, k)]
        Rt = 2.0 * R - R.T
        P, T = frag.P[(i, j)], res.T[(i, j)]
        D = (2.0 if i == j else 4.0) * (Rt @ P @ T.T + Rt.T @ P @ T)
        ni = frag.n[i]
        G[i] += D[:, :ni]
        if i != j:
            G[j] += D[:, ni:]
    return G


def osv_response(T_ii: np.ndarray, Q_i: np.ndarray, G_i: np.ndarray) -> Tuple[np.ndarray, float]:
    """Adjoint of T_ii: the symmetric Z with dE = <Z, dT_ii> for the energy's
    dependence on the kept eigenvectors Q_i of Eq. (osv_gen), count held fixed.

    First-order perturbation of the eigenvectors of a symmetric matrix,
    dq_k = sum_(l != k) z_l (z_l^T dT q_k) / (omega_k - omega_l), summed over the
    discarded eigenvectors z_l only: the kept-kept terms cancel because E does
    not change under a rotation of Q_i within its span.  Returns (Z, gap) with
    gap = omega_(n_i - 1) - omega_(n_i), the eigenvalue gap at the cut.
    """
    w, V = np.linalg.eigh(T_ii)
    order = np.argsort(-w, kind="stable")
    w, V = w[order], V[:, order]
    ni = Q_i.shape[1]
    if ni == w.size:
        return np.zeros_like(T_ii), np.inf
    Zd, wd = V[:, ni:], w[ni:]
    Y = (Zd.T @ G_i) / (w[None, :ni] - wd[:, None])
    Xr = Zd @ Y
    Z = 0.5 * (Xr @ Q_i.T + Q_i @ Xr.T)
    return Z, float(w[ni - 1] - w[ni])


def tii_adjoint(Z: np.ndarray, B_i: np.ndarray, e_vir: np.ndarray, f_ii: float):
    """Chain rule through T_ii = B_i B_i^T / (e_a + e_b - 2 f_ii) (Eq. mp2_tkk, R4)
    for dE = <Z, dT_ii>, Z symmetric: (dE/dB_i, dE/de_vir, dE/df_ii)."""
    D = e_vir[:, None] + e_vir[None, :] - 2.0 * f_ii
    T = (B_i @ B_i.T) / D
    W = Z / D
    ZT = Z * T / D
    return 2.0 * W @ B_i, -2.0 * ZT.sum(axis=1), 2.0 * float(ZT.sum())


def mbe3_energy_gradient_relaxed(osys: OSVSystem, r_occ: np.ndarray, r2: float, r3: float,
                                 n_vir: int, n_aux: int, **kw):
    """E, dE/dB, dE/de_vir, dE/df (symmetrised) for MBE(3) with the OSVs rebuilt
    from B, e and f (reading R23), and the smallest eigenvalue gap at the cut."""
    n = osys.n_occ
    dB = np.zeros((n, n_vir, n_aux))
    de = np.zeros(n_vir)
    df = np.zeros((n, n))
    GQ: Dict[int, np.ndarray] = {}
    E = 0.0
    for orbs, c in mbe3_fragments(r_occ, r2, r3):
        if c == 0:
            continue
        frag = osys.fragment(orbs)
        res = solve_fragment(frag, **kw)
        E += c * res.energy
        gB, ge, gf = fragment_gradient(frag, res, osys.B, n, n_vir, n_aux)
        for i, v in gB.items():
            dB[i] += c * v
        de += c * ge
        df += c * gf
        for x, g in fragment_dE_dQ(frag, res, osys.B, osys.e_vir).items():
            GQ[x] = GQ.get(x, 0.0) + c * g
    gap = np.inf
    for x, g in sorted(GQ.items()):
        T_xx = semicanonical_tii(osys.B(x), osys.e_vir, osys.f_occ[x, x])
        Z, gx = osv_response(T_xx, osys.Q[x], g)
        gap = min(gap, gx)
        gB, ge, gf = tii_adjoint(Z, osys.B(x), osys.e_vir, osys.f_occ[x, x])
        dB[x] += gB
        de += ge
        df[x, x] += gf
    return E, dB, de, df, gap


# --------------------------------------------------------------------------
# Pair screening and weak pairs: Eqs. (s2b), (s3b), (osv_weak_k), (res_weak);
# the weak-pair branch of Algorithm 7
# --------------------------------------------------------------------------
def s2b_metric(Q: Sequence[np.ndarray], i: int, j: int) -> float:
    """s2b_ij = sum_{mu nu} <mu_i|nu_j>^2 / sqrt(n_i n_j)   (Eq. s2b)."""
    S = Q[i].T @ Q[j]
    return float(np.sum(S * S)) / np.sqrt(Q[i].shape[1] * Q[j].shape[1])


def s2b_matrix(Q: Sequence[np.ndarray]) -> np.ndarray:
    n = len(Q)
    M = np.ones((n, n))
    for i in range(n):
        for j in range(i + 1, n):
            M[i, j] = M[j, i] = s2b_metric(Q, i, j)
    return M


def s3b_metric(s2b: np.ndarray, i: int, j: int, k: int) -> float:
    """s3b_ijk = (s2b_ij + s2b_ik + s2b_jk) / 3   (Eq. s3b)."""
    return (s2b[i, j] + s2b[i, k] + s2b[j, k]) / 3.0


@dataclasses.dataclass
class Screen:
    """Pair-class cuts of Section 3.4: distant below s2b_distant, weak up to
    s2b_close, close above; triples of close pairs kept when s3b >= s3b_min."""
    s2b_distant: float = 1e-7
    s2b_close: float = 1e-2
    s3b_min: float = 0.2


def screened_fragments(s2b: np.ndarray, scr: Screen):
    """Clusters and weak pairs selected by s2b / s3b (reading R16).

    close pairs: s2b >= s2b_close; weak pairs: s2b_distant <= s2b < s2b_close;
    triples: all three pairs close and s3b >= s3b_min (so every kept cluster's
    sub-clusters are kept).  Weights are the inclusion-exclusion weights of
    Eqs. (tmbediag)-(deltaoff), as in mbe3_fragments.  Returns
    (list of (orbs, weight) -- singles, pairs, triples, each lexicographic --,
     list of weak pairs (i, j), i < j, lexicographic)."""
    n = s2b.shape[0]
    close = [(i, j) for i in range(n) for j in range(i + 1, n) if s2b[i, j] >= scr.s2b_close]
    weak = [(i, j) for i in range(n) for j in range(i + 1, n) if scr.s2b_distant <= s2b[i, j] < scr.s2b_close]
    is_close = np.zeros((n, n), dtype=bool)
    for (i, j) in close:
        is_close[i, j] = is_close[j, i] = True
    triples = [(i, j, k) for i in range(n) for j in range(i + 1, n) if is_close[i, j]
               for k in range(j + 1, n) if is_close[i, k] and is_close[j, k] and s3b_metric(s2b, i, j, k) >= scr.s3b_min]
    return _weighted(n, close, triples), weak


def _weighted(n, pairs, triples):
    tri_per_pair: Dict[Pair, int] = {}
    tri_per_orb = np.zeros(n, dtype=np.int64)
    pair_per_orb = np.zeros(n, dtype=np.int64)
    for (i, j) in pairs:
        pair_per_orb[i] += 1
        pair_per_orb[j] += 1
    for (i, j, k) in triples:
        for p in ((i, j), (i, k), (j, k)):
            tri_per_pair[p] = tri_per_pair.get(p, 0) + 1
        for x in (i, j, k):
            tri_per_orb[x] += 1
    frags = [((i,), int(1 - pair_per_orb[i] + tri_per_orb[i])) for i in range(n)]
    frags += [((i, j), int(1 - tri_per_pair.get((i, j), 0))) for (i, j) in pairs]
    frags += [(t, 1) for t in triples]
    return frags


def mbe3_diagonal_amplitudes(results, frags) -> Dict[int, np.ndarray]:
    """T_(ii,ii) in the basis Q_i from the cluster amplitudes, Eq. (tmbediag):
    T^i + sum_k dT^{i,k} + sum_{k>l} dT^{i,k,l} = sum over kept clusters C that
    contain i of c_C T^C_(ii,ii)."""
    out: Dict[int, np.ndarray] = {}
    for res, (orbs, c) in zip(results, frags):
        for i in orbs:
            t = c * res.T[(i, i)]
            out[i] = out[i] + t if i in out else t
    return out


@dataclasses.dataclass
class WeakResult:
    pair: Pair
    energy: float          # both orders of the pair
    T: np.ndarray          # T_(i,j) in the single-block basis Q_i (rows) x Q_j (columns)


def weak_pair(Q: Sequence[np.ndarray], Bfun: Callable[[int], np.ndarray], f_occ: np.ndarray,
              e_vir: np.ndarray, i: int, j: int, T_ii: np.ndarray, T_jj: np.ndarray) -> WeakResult:
    """Non-iterative weak-pair amplitude and energy (Algorithm 7, weak pairs).

    K_(i,j) = Gamma~_i^{mu_i} Gamma~_j^{nu_j}            (Eq. osv_weak_k)
    R_(i,j) = K_(i,j) + F_(i,i) T + T F_(j,j) - (f_ii + f_jj) T
              - f_ij [T_(i,i) S_(i,j) + S_(i,j) T_(j,j)]   (Eq. res_weak, reading R17)
    With S_(i,i) = 1 the preconditioner of the diagonal pair diagonalises
    F_(i,i) (Eq. prec_eig), so one update from T = 0 solves R = 0 exactly:
    T = X_i [X_i^T R(0) X_j / (f_ii + f_jj - e~_i - e~_j)] X_j^T.
    Energy: 2 <K_(i,j), T> per ordered pair with the exchange term dropped
    (reading R18), both orders counted."""
    Li = Q[i].T @ Bfun(i)          # OSV-projected integrals of Eq. (osv_imua), diagonal blocks only
    Lj = Q[j].T @ Bfun(j)
    K = Li @ Lj.T
    S = Q[i].T @ Q[j]
    Fii = Q[i].T @ (e_vir[:, None] * Q[i])
    Fjj = Q[j].T @ (e_vir[:, None] * Q[j])
    Xi, Ei = preconditioner(Q[i].T @ Q[i], Fii, 0.0)
    Xj, Ej = preconditioner(Q[j].T @ Q[j], Fjj, 0.0)
    R0 = K - f_occ[i, j] * (T_ii @ S + S @ T_jj)
    D = f_occ[i, i] + f_occ[j, j] - Ei[:, None] - Ej[None, :]
    T = Xi @ ((Xi.T @ R0 @ Xj) / D) @ Xj.T
    return WeakResult((i, j), 4.0 * float(np.sum(K * T)), T)


def weak_residual(Q, Bfun, f_occ, e_vir, i, j, T, T_ii, T_jj) -> np.ndarray:
    """R_(i,j) of Eq. (res_weak) (reading R17) for a given T_(i,j)."""
    K = (Q[i].T @ Bfun(i)) @ (Q[j].T @ Bfun(j)).T
    S = Q[i].T @ Q[j]
    Fii = Q[i].T @ (e_vir[:, None] * Q[i])
    Fjj = Q[j].T @ (e_vir[:, None] * Q[j])
    return (K + Fii @ T + T @ Fjj - (f_occ[i, i] + f_occ[j, j]) * T
            - f_occ[i, j] * (T_ii @ S + S @ T_jj))


def mbe3_screened_energy(osys: "OSVSystem", scr: Screen, **kw):
    """MBE(3) energy with the paper's cluster selection (Section 3.4) and the
    weak pairs of Algorithm 7: E = sum_C c_C E_C + sum_weak E_ij.
    Returns (E, E_weak, per-fragment [(orbs, c, E_C)], [WeakResult], s2b)."""
    s2b = s2b_matrix(osys.Q)
    frags, weak = screened_fragments(s2b, scr)
    results = [osys.solve(orbs, **kw) for orbs, _ in frags]
    E = sum(c * r.energy for (orbs, c), r in zip(frags, results))
    Tdiag = mbe3_diagonal_amplitudes(results, frags)
    wres = [weak_pair(osys.Q, osys.B, osys.f_occ, osys.e_vir, i, j, Tdiag[i], Tdiag[j]) for (i, j) in weak]
    E_weak = sum(w.energy for w in wres)
    per = [(orbs, c, r.energy) for (orbs, c), r in zip(frags, results)]
    return E + E_weak, E_weak, per, wres, s2b


# --------------------------------------------------------------------------
# Randomized OSV generation: Algorithm 3 with Eqs. (rsvd_z), (tsub),
# (tii_rsvd), (back_q) and (rsvd_za)
# --------------------------------------------------------------------------
@dataclasses.dataclass
class RandomizedOSV:
    Q: np.ndarray          # kept OSVs [n_vir, n_i], descending omega, sign convention R9
    omega: np.ndarray      # kept singular values of T~ (>= l_osv)
    Z: np.ndarray          # orthonormal rows of the range finder [n_rosv, n_vir]
    n_rosv: int            # rows taken (s at exit)
    window_max: float      # max norm of the r look-ahead rows at exit


def randomized_osv(T: np.ndarray, l_osv: float, gauss_row: Callable[[int], np.ndarray], r: int = 10,
                   n_max: int = 0) -> RandomizedOSV:
    """Adaptive randomized range finder on the rows of T_ii, then a low-rank SVD.

    gauss_row(k) gives Gaussian row k of the method's random draws (k = 0..r-1
    form G, k = r + s - 1 gives the fresh row g-bar^(s) of G-bar); the draws are
    inputs, not generated here.  Steps in the order of Algorithm 3:
      Y = G T (r rows); while the largest row norm of Y exceeds
      l_osv / (10 sqrt(2/pi)): s += 1; z^(s) from y^(s) by Eq. (rsvd_za)
      (projected against Z^(s-1), normalised) and appended to Z; the window
      shifts; the new last row is g-bar^(s) T (I - Z^(s-1)^T Z^(s-1)); every
      window row loses its z^(s) component (Y -= Y z^T z).
      T~ = Z T (Eq. tsub), T~ = Q~ omega V~^T (Eq. tii_rsvd), Q = Z^T Q~
      (Eq. back_q), kept where omega >= l_osv.
    n_max (0: n_vir) caps the rows; reaching it is reported through n_rosv."""
    nv = T.shape[0]
    n_max = n_max or nv
    thr = l_osv / (10.0 * np.sqrt(2.0 / np.pi))
    Y = np.stack([gauss_row(k) @ T for k in range(r)])
    Z = np.zeros((0, nv))
    s = 0
    while s < n_max and np.max(np.linalg.norm(Y, axis=1)) > thr:
        s += 1
        zt = Y[0] - (Y[0] @ Z.T) @ Z                    # Eq. (rsvd_za)
        z = zt / np.linalg.norm(zt)
        Z_prev = Z
        Z = np.vstack([Z, z])
        ybar = gauss_row(r + s - 1) @ T
        ynew = ybar - (ybar @ Z_prev.T) @ Z_prev
        Y = np.vstack([Y[1:], ynew])
        Y = Y - np.outer(Y @ z, z)
    Tt = Z @ T                                          # Eq. (tsub)
    Qt, w, _ = np.linalg.svd(Tt, full_matrices=False)   # Eq. (tii_rsvd)
    Q = Z.T @ Qt                                        # Eq. (back_q)
    keep = w >= l_osv
    Q, w = Q[:, keep], w[keep]
    if Q.shape[1]:
        big = np.argmax(np.abs(Q), axis=0)
        sgn = np.sign(Q[big, np.arange(Q.shape[1])])
        sgn[sgn == 0] = 1.0
        Q = Q * sgn
    return RandomizedOSV(np.ascontiguousarray(Q), w, Z, s, float(np.max(np.linalg.norm(Y, axis=1))))


def build_osv_randomized(Bfun: Callable[[int], np.ndarray], n_occ: int, e_vir: np.ndarray, f_occ: np.ndarray,
                         l_osv: float, gauss: Callable[[int, int], np.ndarray], r: int = 10, n_max: int = 0,
                         orbitals=None):
    """Randomized OSVs of every orbital (Algorithm 3); gauss(i, k) is Gaussian row k
    of orbital i.  Returns (Q list, omega list, RandomizedOSV list)."""
    Q, W, R = [None] * n_occ, [None] * n_occ, [None] * n_occ
    for i in (range(n_occ) if orbitals is None else orbitals):
        T = semicanonical_tii(Bfun(i), e_vir, f_occ[i, i])
        R[i] = randomized_osv(T, l_osv, lambda k, i=i: gauss(i, k), r=r, n_max=n_max)
        Q[i], W[i] = R[i].Q, R[i].omega
    return Q, W, R
