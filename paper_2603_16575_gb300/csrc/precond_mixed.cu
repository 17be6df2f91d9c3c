// A3 for the mixed form: a basis X of the pair space with X^T F X ~ diag(e~) and
// X^T S X ~ 1 (Eq. prec_eig), plus the exact leftovers
//   S^ = X^T S X - 1,   G^ = (X^T F X - diag(e~)) - (f_ii + f_jj)/2 S^
// (FP64 products, stored FP32: they are ~1e-7) that the mixed fragment solver
// adds to its update, so the iteration's fixed point is the exact one whatever
// the accuracy of X.
//
// Canonical orthogonalisation through the block structure of the overlap:
// S_(ij,ij) = [[1, M], [M^T, 1]] with M = Q_i^T Q_j (the OSVs of each orbital
// are orthonormal).  With C = 1 - M^T M = V diag(mu) V^T (FP64, order n_j),
//   Y = [[1, -M Z], [0, Z]],  Z = V_kept diag(mu_kept)^(-1/2),
// gives Y^T S Y = blockdiag(1, Z^T C Z) = 1.  The eigenvalues of S are 1 and
// 1 +- sigma_k (sigma_k^2 = 1 - mu_k), and a direction is dropped exactly when
// the canonical orthogonalisation drops the eigenvalue 1 - sigma_k =
// mu_k / (1 + sigma_k) below tau_s (1 + sigma_max).  Then F' = Y^T F Y (FP64,
// entries bounded by the virtual energies whatever the conditioning of Y) is
// diagonalised in FP32 (F' = W diag(e~) W^T) and X = Y W.  A diagonal pair has
// S_(ii,ii) = Q_i^T Q_i = 1: Y = 1, F' = F_(i,i).
//
// Four launches, each with one CTA per pair (grid-stride over the pairs in
// descending order, so the largest start first): (1) 1 - M^T M, its FP64
// eigen-decomposition, Y and Z^T C Z; (2) F' = Y^T F Y (tiled FP64 GEMMs);
// (3) FP32 eigen-decomposition of F'; (4) X = Y W and the leftovers (tiled FP64
// GEMMs).  The eigen-solvers (eig.cuh, Householder + implicit QR) keep the
// eigenvectors column-major so that the rotations of the QR sweeps, one thread
// per row, are coalesced.  Per-pair intermediates live in a scratch slot:
// Y [m][r], F' [r][r], W [r][r], Z^T C Z [nk][nk], e~ [r].
#include <algorithm>

#include "eig.cuh"
#include "pairview.cuh"

namespace osv {

constexpr int PM_MAXN = 192;   // largest pair order (static shared scratch of the eigen-solvers)

__host__ __device__ inline size_t pm_slot_doubles(int m) { return 4 * (size_t)m * m + (size_t)m + 8; }
// per-CTA scratch: (1) C, C0, V [3][max_m^2] + mu, e, tau; (2) F Y; (3) FP32 A, Z, e~, e, tau; (4) 3 blocks
__host__ __device__ inline size_t pm_cta_doubles(int max_m) {
  return 3 * (size_t)max_m * max_m + 3 * (size_t)max_m;
}

struct PmPair {              // per-pair view of the scratch slot
  double* Y;                 // [m][r]
  double* Fp;                // [r][r]
  double* W;                 // [r][r]
  double* ZCZ;               // [nk][nk]
  double* et;                // [r]
};
__device__ __forceinline__ PmPair pm_pair(double* slots, const long long* off, int jid, int m) {
  double* b = slots + off[jid];
  const size_t M2 = (size_t)m * m;
  return PmPair{b, b + M2, b + 2 * M2, b + 3 * M2, b + 4 * M2};
}

// (1) S part: C = 1 - M^T M, eig(C) (FP64), kept directions, Y, Z^T C Z, r
__global__ void __launch_bounds__(NT, 3) k_pm_overlap(Tables t, double tau_s, const PJob* __restrict__ jobs,
                                                      const int* __restrict__ order, int n_jobs, double* slots,
                                                      const long long* off, int max_m, double* scratch, int* err) {
  __shared__ double gsm[GEMM_SMEM_DOUBLES];
  __shared__ double esm[4 * PM_MAXN + 33];
  __shared__ int keep[PM_MAXN];
  __shared__ int s_nk;
  const size_t M2 = (size_t)max_m * max_m;
  double* Cw = scratch + (size_t)blockIdx.x * pm_cta_doubles(max_m);
  double* C0 = Cw + M2;
  double* V = C0 + M2;          // eigenvector k of C at V[k * nj ..]
  double* mu = V + M2;
  double* e = mu + max_m;
  double* tau = e + max_m;
  const int n = t.n_occ;
  for (int q = blockIdx.x; q < n_jobs; q += gridDim.x) {
    const int jid = order[q];
    const PJob jb = jobs[jid];
    const int i = jb.i, j = jb.j;
    const int ni = t.n_osv[i], nj = (i == j) ? 0 : t.n_osv[j];
    const int m = ni + nj;
    const PmPair pp = pm_pair(slots, off, jid, m);
    if (i == j) {
      if (threadIdx.x == 0) *jb.r = ni;
      continue;
    }
    const View Mv = dense_view(t.S[t.sf_id[i * n + j]], ni, nj, nj);
    cta_gemm(nj, nj, ni, -1.0, transpose(Mv), Mv, 0.0, Cw, nj, gsm);
    for (int c = threadIdx.x; c < nj; c += NT) Cw[(size_t)c * nj + c] += 1.0;
    __syncthreads();
    for (int idx = threadIdx.x; idx < nj * nj; idx += NT) C0[idx] = Cw[idx];
    __syncthreads();
    const int rc = cta_syev_cm(Cw, nj, nj, mu, V, nj, e, tau, esm);
    if (threadIdx.x == 0) {
      if (rc) atomicOr(err, ERR_EIG);
      double mumin = 1.0;
      for (int k = 0; k < nj; k++) mumin = fmin(mumin, mu[k]);
      const double smax = 1.0 + sqrt(fmax(0.0, 1.0 - mumin));
      int nk = 0;
      for (int k = 0; k < nj; k++) {
        const double lam = mu[k] / (1.0 + sqrt(fmax(0.0, 1.0 - mu[k])));
        if (mu[k] > 0.0 && lam > tau_s * smax) keep[nk++] = k;
      }
      s_nk = nk;
    }
    __syncthreads();
    const int nk = s_nk, r = ni + nk;
    double* Y = pp.Y;
    for (int idx = threadIdx.x; idx < m * r; idx += NT) {
      const int a = idx / r, b = idx % r;
      double y = 0.0;
      if (a < ni) y = (b == a) ? 1.0 : 0.0;
      else if (b >= ni) {
        const int k = keep[b - ni];
        y = V[(size_t)k * nj + (a - ni)] / sqrt(mu[k]);
      }
      Y[idx] = y;
    }
    __syncthreads();
    const View Zv = dense_view(Y + (size_t)ni * r + ni, nj, nk, r);
    cta_gemm(ni, nk, nj, -1.0, Mv, Zv, 0.0, Y + ni, r, gsm);                                     // -M Z
    cta_gemm(nj, nk, nj, 1.0, dense_view(C0, nj, nj, nj), Zv, 0.0, Cw, nk, gsm);                // C Z
    cta_gemm(nk, nk, nj, 1.0, transpose(Zv), dense_view(Cw, nj, nk, nk), 0.0, pp.ZCZ, nk, gsm);  // Z^T C Z
    if (threadIdx.x == 0) *jb.r = r;
  }
}

// (2) F' = Y^T F Y
__global__ void __launch_bounds__(NT) k_pm_fprime(Tables t, const PJob* __restrict__ jobs,
                                                  const int* __restrict__ order, int n_jobs, double* slots,
                                                  const long long* off, int max_m, double* scratch) {
  __shared__ double sm[GEMM_SMEM_DOUBLES];
  double* FY = scratch + (size_t)blockIdx.x * pm_cta_doubles(max_m);
  for (int q = blockIdx.x; q < n_jobs; q += gridDim.x) {
    const int jid = order[q];
    const PJob jb = jobs[jid];
    const int i = jb.i, j = jb.j;
    const int ni = t.n_osv[i], nj = (i == j) ? 0 : t.n_osv[j];
    const int m = ni + nj, r = *jb.r, nk = r - ni;
    const PmPair pp = pm_pair(slots, off, jid, m);
    const View Fv = pair_view(t, t.F, i, j, i, j);
    if (i == j) {
      for (int idx = threadIdx.x; idx < m * m; idx += NT) pp.Fp[idx] = Fv.get(idx / m, idx % m);
      __syncthreads();
      continue;
    }
    // F Y: the first ni columns of Y are unit vectors
    for (int idx = threadIdx.x; idx < m * ni; idx += NT)
      FY[(size_t)(idx / ni) * r + idx % ni] = Fv.get(idx / ni, idx % ni);
    cta_gemm(m, nk, m, 1.0, Fv, dense_view(pp.Y + ni, m, nk, r), 0.0, FY + ni, r, sm);
    cta_gemm(r, r, m, 1.0, transpose(dense_view(pp.Y, m, r, r)), dense_view(FY, m, r, r), 0.0, pp.Fp, r, sm);
  }
}

// (3) FP32 eigen-decomposition of F' (symmetrised): W, e~
__global__ void __launch_bounds__(NT, 3) k_pm_eig32(const PJob* __restrict__ jobs, const int* __restrict__ order,
                                                    int n_jobs, double* slots, const long long* off,
                                                    const int* mdim, int max_m, double* scratch, int* err) {
  __shared__ float esm[4 * PM_MAXN + 33];
  const size_t M2 = (size_t)max_m * max_m;
  float* A32 = reinterpret_cast<float*>(scratch + (size_t)blockIdx.x * pm_cta_doubles(max_m));
  float* Z32 = A32 + M2;        // eigenvector t at Z32[t * r ..]
  float* e32 = Z32 + M2;
  float* eb = e32 + max_m;
  float* tau32 = eb + max_m;
  for (int q = blockIdx.x; q < n_jobs; q += gridDim.x) {
    const int jid = order[q];
    const PJob jb = jobs[jid];
    const int m = mdim[jid], r = *jb.r;
    const PmPair pp = pm_pair(slots, off, jid, m);
    for (int idx = threadIdx.x; idx < r * r; idx += NT) {
      const int a = idx / r, b = idx % r;
      A32[idx] = (float)(0.5 * (pp.Fp[idx] + pp.Fp[(size_t)b * r + a]));
    }
    __syncthreads();
    const int rc = cta_syev_cm(A32, r, r, e32, Z32, r, eb, tau32, esm);
    if (threadIdx.x == 0 && rc) atomicOr(err, ERR_EIG);
    for (int idx = threadIdx.x; idx < r * r; idx += NT) {   // W[a][t] = component a of eigenvector t
      const int tv = idx / r, a = idx % r;
      pp.W[(size_t)a * r + tv] = (double)Z32[idx];
    }
    for (int c = threadIdx.x; c < r; c += NT) pp.et[c] = (double)e32[c];
    __syncthreads();
  }
}

// (4) X = Y W; S~ = W^T (Y^T S Y) W; F~ = W^T F' W; leftovers
__global__ void __launch_bounds__(NT) k_pm_final(Tables t, const PJob* __restrict__ jobs,
                                                 const int* __restrict__ order, int n_jobs, double* slots,
                                                 const long long* off, int max_m, double* scratch, int* err) {
  __shared__ double sm[GEMM_SMEM_DOUBLES];
  const size_t M2 = (size_t)max_m * max_m;
  double* T1 = scratch + (size_t)blockIdx.x * pm_cta_doubles(max_m);
  double* St = T1 + M2;
  double* Ft = St + M2;
  const int n = t.n_occ;
  for (int q = blockIdx.x; q < n_jobs; q += gridDim.x) {
    const int jid = order[q];
    const PJob jb = jobs[jid];
    const int i = jb.i, j = jb.j;
    const int ni = t.n_osv[i], nj = (i == j) ? 0 : t.n_osv[j];
    const int m = ni + nj, r = *jb.r, nk = r - ni;
    const PmPair pp = pm_pair(slots, off, jid, m);
    const View Wv = dense_view(pp.W, r, r, r);
    if (i != j) {
      cta_gemm(m, r, r, 1.0, dense_view(pp.Y, m, r, r), Wv, 0.0, jb.X, m, sm);       // X = Y W
      for (int idx = threadIdx.x; idx < ni * r; idx += NT) T1[idx] = pp.W[idx];        // (Y^T S Y) W, top rows
      cta_gemm(nk, r, nk, 1.0, dense_view(pp.ZCZ, nk, nk, nk), dense_view(pp.W + (size_t)ni * r, nk, r, r), 0.0,
               T1 + (size_t)ni * r, r, sm);
    } else {
      for (int idx = threadIdx.x; idx < m * r; idx += NT) jb.X[(size_t)(idx / r) * m + idx % r] = pp.W[idx];
      cta_gemm(r, r, r, 1.0, dense_view(t.S[t.sf_id[i * n + i]], ni, ni, ni), Wv, 0.0, T1, r, sm);
    }
    cta_gemm(r, r, r, 1.0, transpose(Wv), dense_view(T1, r, r, r), 0.0, St, r, sm);      // S~
    cta_gemm(r, r, r, 1.0, dense_view(pp.Fp, r, r, r), Wv, 0.0, T1, r, sm);
    cta_gemm(r, r, r, 1.0, transpose(Wv), dense_view(T1, r, r, r), 0.0, Ft, r, sm);      // F~
    const double fh = 0.5 * (t.f_occ[i * n + i] + t.f_occ[j * n + j]);
    for (int idx = threadIdx.x; idx < r * r; idx += NT) {
      const int a = idx / r, b = idx % r;
      const double sh = St[idx] - (a == b ? 1.0 : 0.0);
      const double gh = Ft[idx] - (a == b ? pp.et[a] : 0.0) - fh * sh;
      jb.Sh[idx] = (float)sh;
      jb.Gh[idx] = (float)gh;
      if (!isfinite(sh) || !isfinite(gh)) atomicOr(err, ERR_NONFINITE);
    }
    for (int c = threadIdx.x; c < r; c += NT) jb.et[c] = pp.et[c];
    __syncthreads();
  }
}

size_t precond_mixed_slot_doubles(int m) { return pm_slot_doubles(m); }

size_t precond_mixed_scratch_doubles(int max_m, int n_cta) { return (size_t)n_cta * pm_cta_doubles(max_m); }

int launch_precond_mixed(const Tables& t, double tau_s, const PJob* jobs, const int* order, int n_jobs, int max_m,
                         double* slots, const long long* off, const int* mdim, double* scratch, int n_cta, int* err,
                         cudaStream_t st) {
  if (!n_jobs) return 0;
  if (max_m > PM_MAXN) return -1;
  k_pm_overlap<<<n_cta, NT, 0, st>>>(t, tau_s, jobs, order, n_jobs, slots, off, max_m, scratch, err);
  k_pm_fprime<<<n_cta, NT, 0, st>>>(t, jobs, order, n_jobs, slots, off, max_m, scratch);
  k_pm_eig32<<<n_cta, NT, 0, st>>>(jobs, order, n_jobs, slots, off, mdim, max_m, scratch, err);
  k_pm_final<<<n_cta, NT, 0, st>>>(t, jobs, order, n_jobs, slots, off, max_m, scratch, err);
  note_launch(4);
  return 0;
}

}  // namespace osv
