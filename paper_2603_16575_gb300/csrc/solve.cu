// A4-A5 in FP64: the pair residual of Eq. (res_close), the preconditioned
// update and pair energy of Algorithm 7, solved either per MBE fragment (one
// persistent launch; each CTA takes fragments from an atomic counter and
// iterates one to convergence) or for one large subsystem (pair-parallel
// kernels, one Jacobi sweep per launch), and the MBE(3) weighted energy sum.
#include "pairview.cuh"

namespace osv {

__device__ __forceinline__ int lpair(int a, int b, int nc) { return a * nc - a * (a - 1) / 2 + (b - a); }

// R_(ij,ij) of Eq. (res_close) for local pair (a,b), a <= b, of the subsystem
// orbs[0..nc).  With G1 = F_p - f_ii S_p and G2 = F_p - f_jj S_p the k = i
// and k = j terms of both sums fold into G1 T S + S T G2; every other k adds
// -f S_(p,q) op(T_q) S_(p,q)^T with q the stored pair of (i,k) or (k,j) and
// op the transpose when the ordered pair is reversed.
__device__ void pair_residual(const Tables& t, int nc, const int* orbs, double* const* T, int a, int b,
                              double* R, const double* G1, const double* G2, double* W, double* sm) {
  const int i = orbs[a], j = orbs[b];
  const int mp = pair_dim(t, i, j);
  const double* K = t.K[t.pair_id[i * t.n_occ + j]];
  const double* Tp = T[lpair(a, b, nc)];
  for (int idx = threadIdx.x; idx < mp * mp; idx += NT) R[idx] = K[idx];
  __syncthreads();
  const View Sp = pair_view(t, t.S, i, j, i, j);
  const View Tv = dense_view(Tp, mp, mp, mp);
  const View Wv = dense_view(W, mp, mp, mp);
  cta_gemm(mp, mp, mp, 1.0, Tv, Sp, 0.0, W, mp, sm);
  cta_gemm(mp, mp, mp, 1.0, dense_view(G1, mp, mp, mp), Wv, 1.0, R, mp, sm);
  cta_gemm(mp, mp, mp, 1.0, Tv, dense_view(G2, mp, mp, mp), 0.0, W, mp, sm);
  cta_gemm(mp, mp, mp, 1.0, Sp, Wv, 1.0, R, mp, sm);
  const double* f = t.f_occ;
  const int n = t.n_occ;
  for (int c = 0; c < nc; c++) {
    const int k = orbs[c];
    for (int s = 0; s < 2; s++) {
      int x, y;
      double coef;
      if (s == 0) {                 // -f_kj S_(ij,ik) T_(ik) S_(ik,ij)
        if (c == b) continue;
        x = a; y = c; coef = -f[k * n + j];
      } else {                      // -f_ik S_(ij,kj) T_(kj) S_(kj,ij)
        if (c == a) continue;
        x = c; y = b; coef = -f[i * n + k];
      }
      if (coef == 0.0) continue;
      const int qa = min(x, y), qb = max(x, y), tr = x > y;
      const int gi = orbs[qa], gj = orbs[qb];
      const int mq = pair_dim(t, gi, gj);
      const View Spq = pair_view(t, t.S, i, j, gi, gj);
      cta_gemm(mq, mp, mq, 1.0, dense_view(T[lpair(qa, qb, nc)], mq, mq, mq, tr), transpose(Spq), 0.0, W, mp, sm);
      cta_gemm(mp, mp, mq, coef, Spq, dense_view(W, mq, mp, mp), 1.0, R, mp, sm);
    }
  }
}

// T_p += X (X^T R X / D) X^T with D_mn = f_ii + f_jj - e~_m - e~_n; returns max |X^T R X / D|.
__device__ double pair_update(const Tables& t, int i, int j, const double* R, double* Tp, double* W, double* Rt,
                              double* sm, double* red) {
  const int mp = pair_dim(t, i, j);
  const int pid = t.pair_id[i * t.n_occ + j];
  const double* X = t.X[pid];
  const double* et = t.et[pid];
  const int r = t.r[pid];
  const double fij = t.f_occ[i * t.n_occ + i] + t.f_occ[j * t.n_occ + j];
  const View Xv = dense_view(X, mp, r, mp);
  cta_gemm(mp, r, mp, 1.0, dense_view(R, mp, mp, mp), Xv, 0.0, W, r, sm);
  cta_gemm(r, r, mp, 1.0, transpose(Xv), dense_view(W, mp, r, r), 0.0, Rt, r, sm);
  double um = 0.0;
  for (int idx = threadIdx.x; idx < r * r; idx += NT) {
    const int u = idx / r, v = idx % r;
    const double y = Rt[idx] / (fij - et[u] - et[v]);
    Rt[idx] = y;
    um = fmax(um, fabs(y));
  }
  um = cta_max(um, red);
  cta_gemm(r, mp, r, 1.0, dense_view(Rt, r, r, r), transpose(Xv), 0.0, W, mp, sm);
  cta_gemm(mp, mp, r, 1.0, Xv, dense_view(W, r, mp, mp), 1.0, Tp, mp, sm);
  return um;
}

// <K, 2T - T^T>_F, doubled for i != j (both orders of the pair).
__device__ double pair_energy(const double* K, const double* T, int m, int diag, double* red) {
  double s = 0.0;
  for (int idx = threadIdx.x; idx < m * m; idx += NT) {
    const int r = idx / m, c = idx % m;
    s += K[idx] * (2.0 * T[idx] - T[(size_t)c * m + r]);
  }
  s = cta_sum(s, red);
  return diag ? s : 2.0 * s;
}

// Zero T_p and build G1 = F_p - f_ii S_p, G2 = F_p - f_jj S_p.
__device__ void pair_prepare(const Tables& t, int i, int j, double* Tp, double* G1, double* G2) {
  const int mp = pair_dim(t, i, j);
  const View Sp = pair_view(t, t.S, i, j, i, j);
  const View Fp = pair_view(t, t.F, i, j, i, j);
  const double fi = t.f_occ[i * t.n_occ + i], fj = t.f_occ[j * t.n_occ + j];
  for (int idx = threadIdx.x; idx < mp * mp; idx += NT) {
    const int r = idx / mp, c = idx % mp;
    const double s = Sp.get(r, c), fv = Fp.get(r, c);
    Tp[idx] = 0.0;
    G1[idx] = fv - fi * s;
    G2[idx] = fv - fj * s;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(NT) k_frag_solve(Tables t, const int* __restrict__ frag_orbs,
                                                   const int* __restrict__ order, int n_frag, int max_m,
                                                   SolveOpts o, double* scratch, int* counter, FragOut* out,
                                                   double* Tstore, const long long* __restrict__ Toff) {
  __shared__ double sm[GEMM_SMEM_DOUBLES];
  __shared__ double red[40];
  __shared__ int s_f;
  const size_t M2 = (size_t)max_m * max_m;
  double* base = scratch + (size_t)blockIdx.x * frag_scratch_doubles(max_m);
  double* T[6];
  double* R[6];
  double* G1[6];
  double* G2[6];
  for (int u = 0; u < 6; u++) {
    T[u] = base + u * M2;
    R[u] = base + (6 + u) * M2;
    G1[u] = base + (12 + u) * M2;
    G2[u] = base + (18 + u) * M2;
  }
  double* W = base + 24 * M2;
  double* Rt = base + 25 * M2;
  while (true) {
    if (threadIdx.x == 0) s_f = atomicAdd(counter, 1);
    __syncthreads();
    const int f = s_f;
    __syncthreads();
    if (f >= n_frag) break;
    const int fid = order[f];
    int orbs[3];
    int nc = 0;
    for (int u = 0; u < 3; u++) {
      const int v = frag_orbs[3 * fid + u];
      if (v >= 0) orbs[nc++] = v;
    }
    for (int a = 0; a < nc; a++)
      for (int b = a; b < nc; b++) {
        const int lp = lpair(a, b, nc);
        pair_prepare(t, orbs[a], orbs[b], T[lp], G1[lp], G2[lp]);
      }
    double e_prev = 0.0, e = 0.0, um = 0.0;
    int status = ERR_NOCONV, iters = o.max_iter;
    for (int it = 1; it <= o.max_iter; it++) {
      for (int a = 0; a < nc; a++)
        for (int b = a; b < nc; b++) {
          const int lp = lpair(a, b, nc);
          pair_residual(t, nc, orbs, T, a, b, R[lp], G1[lp], G2[lp], W, sm);
        }
      um = 0.0;
      for (int a = 0; a < nc; a++)
        for (int b = a; b < nc; b++) {
          const int lp = lpair(a, b, nc);
          um = fmax(um, pair_update(t, orbs[a], orbs[b], R[lp], T[lp], W, Rt, sm, red));
        }
      e = 0.0;
      for (int a = 0; a < nc; a++)
        for (int b = a; b < nc; b++) {
          const int i = orbs[a], j = orbs[b];
          e += pair_energy(t.K[t.pair_id[i * t.n_occ + j]], T[lpair(a, b, nc)], pair_dim(t, i, j), a == b, red);
        }
      if (!isfinite(e) || !isfinite(um)) { status = ERR_NONFINITE; iters = it; break; }
      // energy test: tol_energy, or 16 ulps of |E_C| where that is larger (the
      // fragment energy cannot be resolved below its rounding floor)
      if (um < o.tol_update && fabs(e - e_prev) < fmax(o.tol_energy, 3.5527136788005009e-15 * fabs(e))) {
        status = 0;
        iters = it;
        break;
      }
      e_prev = e;
    }
    if (threadIdx.x == 0) out[fid] = FragOut{e, um, iters, status};
    if (Tstore) {
      double* dst = Tstore + Toff[fid];
      for (int a = 0; a < nc; a++)
        for (int b = a; b < nc; b++) {
          const int mp = pair_dim(t, orbs[a], orbs[b]);
          const double* src = T[lpair(a, b, nc)];
          for (int idx = threadIdx.x; idx < mp * mp; idx += NT) dst[idx] = src[idx];
          dst += (size_t)mp * mp;
        }
    }
    __syncthreads();
  }
}

void launch_frag_solve(const Tables& t, const int* frag_orbs, const int* order, int n_frag, int max_m,
                       SolveOpts o, double* scratch, int n_cta, int* counter, FragOut* out,
                       double* Tstore, const long long* Toff, cudaStream_t st) {
  if (n_frag == 0) return;
  cudaMemsetAsync(counter, 0, sizeof(int), st);
  k_frag_solve<<<n_cta, NT, 0, st>>>(t, frag_orbs, order, n_frag, max_m, o, scratch, counter, out, Tstore, Toff);
  note_launch(1);
}

// E = sum_f w_f E_f, one CTA, fixed order (strided partial sums, fixed tree).
__global__ void k_weighted_sum(const FragOut* out, const int* w, int n, double* e_out) {
  __shared__ double red[40];
  double s = 0.0;
  for (int f = threadIdx.x; f < n; f += NT) s += (double)w[f] * out[f].energy;
  s = cta_sum(s, red);
  if (threadIdx.x == 0) *e_out = s;
}

void launch_weighted_sum(const FragOut* out, const int* weights, int n, double* e_out, cudaStream_t st) {
  k_weighted_sum<<<1, NT, 0, st>>>(out, weights, n, e_out);
  note_launch(1);
}

// ---------------------------------------------------------------- subsystem
__device__ __forceinline__ void local_pair(int lp, int nc, int& a, int& b) {
  a = 0;
  while (lp >= nc - a) { lp -= nc - a; a++; }
  b = a + lp;
}

__global__ void __launch_bounds__(NT) k_sub_prepare(Tables t, SubDev s, int np) {
  for (int lp = blockIdx.x; lp < np; lp += gridDim.x) {
    int a, b;
    local_pair(lp, s.nc, a, b);
    pair_prepare(t, s.orbs[a], s.orbs[b], s.T[lp], s.G1[lp], s.G2[lp]);
  }
}
__global__ void __launch_bounds__(NT) k_sub_residual(Tables t, SubDev s, int np) {
  __shared__ double sm[GEMM_SMEM_DOUBLES];
  for (int lp = blockIdx.x; lp < np; lp += gridDim.x) {
    int a, b;
    local_pair(lp, s.nc, a, b);
    pair_residual(t, s.nc, s.orbs, s.T, a, b, s.R[lp], s.G1[lp], s.G2[lp], s.W[2 * blockIdx.x], sm);
  }
}
__global__ void __launch_bounds__(NT) k_sub_update(Tables t, SubDev s, int np) {
  __shared__ double sm[GEMM_SMEM_DOUBLES];
  __shared__ double red[40];
  for (int lp = blockIdx.x; lp < np; lp += gridDim.x) {
    int a, b;
    local_pair(lp, s.nc, a, b);
    const int i = s.orbs[a], j = s.orbs[b];
    const double um = pair_update(t, i, j, s.R[lp], s.T[lp], s.W[2 * blockIdx.x], s.W[2 * blockIdx.x + 1], sm, red);
    const double e = pair_energy(t.K[t.pair_id[i * t.n_occ + j]], s.T[lp], pair_dim(t, i, j), a == b, red);
    if (threadIdx.x == 0) { s.pe[lp] = e; s.pu[lp] = um; }
    __syncthreads();
  }
}
// pe/pu -> (sum pe, max pu) in s.pe[np], s.pu[np]
__global__ void k_sub_reduce(SubDev s, int np) {
  __shared__ double red[40];
  double e = 0.0, u = 0.0;
  for (int lp = threadIdx.x; lp < np; lp += NT) { e += s.pe[lp]; u = fmax(u, s.pu[lp]); }
  e = cta_sum(e, red);
  u = cta_max(u, red);
  if (threadIdx.x == 0) { s.pe[np] = e; s.pu[np] = u; }
}

void launch_sub_prepare(const Tables& t, const SubDev& s, int np, int n_cta, cudaStream_t st) {
  k_sub_prepare<<<n_cta, NT, 0, st>>>(t, s, np);
  note_launch(1);
}
void launch_sub_residual(const Tables& t, const SubDev& s, int np, int n_cta, cudaStream_t st) {
  k_sub_residual<<<n_cta, NT, 0, st>>>(t, s, np);
  note_launch(1);
}
void launch_sub_update(const Tables& t, const SubDev& s, int np, int n_cta, cudaStream_t st) {
  k_sub_update<<<n_cta, NT, 0, st>>>(t, s, np);
  note_launch(1);
  k_sub_reduce<<<1, NT, 0, st>>>(s, np);
  note_launch(1);
}

}  // namespace osv
