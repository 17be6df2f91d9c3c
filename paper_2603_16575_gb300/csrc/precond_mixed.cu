// A3 for the mixed form: a basis X of the pair space with X^T F X ~ diag(e~) and
// X^T S X ~ 1 (Eq. prec_eig), plus the exact leftovers
//   S^ = X^T S X - 1,   G^ = (X^T F X - diag(e~)) - (f_ii + f_jj)/2 S^
// (double-float products, stored FP32: they are ~1e-7) that the mixed fragment solver
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
// mu_k / (1 + sigma_k) below tau_s (1 + sigma_max).  Then F' = Y^T F Y (double-float,
// entries bounded by the virtual energies whatever the conditioning of Y) is
// diagonalised in FP32 (F' = W diag(e~) W^T) and X = Y W.  A diagonal pair has
// S_(ii,ii) = Q_i^T Q_i = 1: Y = 1, F' = F_(i,i).
//
// Launches (CTA kernels take one pair per CTA, grid-stride over the pairs in
// descending order, so the largest start first):
//   (1a) C = 1 - M^T M, Householder tridiagonalisation and Z (FP64, CTA);
//   (1b) the QR bulge chase of every C, one pair per thread (FP64);
//   (1c) recorded rotations applied to Z, kept directions, Y, Z^T C Z (CTA; the
//        products with Z in double-float);
//   (2)  F' = Y^T F Y (tiled double-float GEMMs, CTA);
//   (3a-c) the same three steps for the FP32 eigen-decomposition of F';
//   (4)  X = Y W and the leftovers (tiled double-float GEMMs, CTA).
// C and its eigen-decomposition stay FP64: C = 1 - M^T M cancels, and its small
// eigenvalues set both the kept directions and Z.  The products with Z, Y and W
// carry ~2^-48 relative error; it enters X, U = P X and the leftovers alike, so
// the fixed point does not move.
// The eigen-solver is Householder + implicit QR (eig.cuh) with the chase run
// per thread over many pairs at once and its rotations recorded, then applied
// to the eigenvectors (kept column-major, so the rotations are coalesced) by a
// CTA; a pair whose record overflows is redone by the in-CTA solver.
// Per-pair intermediates live in a scratch slot: Y [m][r], F' [r][r], W [r][r],
// Z^T C Z [nk][nk], e~ [r], and the eigen-solver's work area.
#include <algorithm>

#include "eig.cuh"
#include "pairview.cuh"

namespace osv {


// eigen-solver work area of a pair of order m: status and sweep count, Z (m x m),
// d and e (m each), the sweep record (cap_s (l, h) pairs) and the rotation
// record (cap_r (c, s) pairs); typed FP64 or FP32 by the step that uses it
__host__ __device__ inline int pm_cap_s(int m) { return 4 * m + 64; }
__host__ __device__ inline int pm_cap_r(int m) { return 2 * m * m + 64; }
__host__ __device__ inline size_t pm_work_doubles(int m) {
  return 2 + (size_t)m * m + 2 * (size_t)m + (size_t)pm_cap_s(m) + 2 * (size_t)pm_cap_r(m);
}
__host__ __device__ inline size_t pm_slot_doubles(int m) {
  return 4 * (size_t)m * m + (size_t)m + 8 + pm_work_doubles(m);
}
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
  double* wk;                // eigen-solver work area
};
__device__ __forceinline__ PmPair pm_pair(double* slots, const long long* off, int jid, int m) {
  double* b = slots + off[jid];
  const size_t M2 = (size_t)m * m;
  return PmPair{b, b + M2, b + 2 * M2, b + 3 * M2, b + 4 * M2, b + 4 * M2 + m + 8};
}

template <class T>
struct PmEig {               // typed view of a pair's eigen-solver work area
  int* hdr;                  // [0] status of the chase (0, 1 no convergence, 2 record overflow), [1] sweeps
  T* Z;                      // eigenvector t at Z[t * n ..] (column-major eigenvector matrix)
  T* d;                      // eigenvalues after the chase
  T* e;
  int* swp;
  T* rot;
};
template <class T>
__device__ __forceinline__ PmEig<T> pm_eig(double* wk, int m) {
  const size_t M2 = (size_t)m * m;
  PmEig<T> w;
  w.hdr = reinterpret_cast<int*>(wk);
  w.Z = reinterpret_cast<T*>(wk + 2);
  w.d = reinterpret_cast<T*>(wk + 2 + M2);
  w.e = reinterpret_cast<T*>(wk + 2 + M2 + m);
  w.swp = reinterpret_cast<int*>(wk + 2 + M2 + 2 * m);
  w.rot = reinterpret_cast<T*>(wk + 2 + M2 + 2 * m + pm_cap_s(m));
  return w;
}

// Householder tridiagonalisation of A (order n, destroyed) and the column-major
// Z of its reflectors into the work area (CTA); tau: n elements, sm: 4n + 33.
template <class T>
__device__ void pm_tridiag(T* A, int n, const PmEig<T>& w, T* tau, T* sm) {
  if (n == 1) {
    if (threadIdx.x == 0) { w.d[0] = A[0]; w.e[0] = T(0.0); w.Z[0] = T(1.0); }
    __syncthreads();
    return;
  }
  cta_tridiag(A, n, n, w.d, w.e, tau, sm, sm + n, sm + 4 * n);
  cta_form_z_cm(A, n, n, tau, w.Z, n, sm, sm + n);
  if (threadIdx.x == 0) w.e[n - 1] = T(0.0);
  __syncthreads();
}

// (1b) / (3b): the QR chase of one pair per thread; which = 0: C (order n_j),
// 1: F' (order r).  Pairs in the order array, so a warp holds pairs of similar size.
template <class T>
__global__ void __launch_bounds__(32) k_pm_chase(Tables t, const PJob* __restrict__ jobs,
                                                 const int* __restrict__ order, int n_jobs, double* slots,
                                                 const long long* off, const int* mdim, int which, int* err) {
  const int q = blockIdx.x * 32 + threadIdx.x;
  if (q >= n_jobs) return;
  const int jid = order[q];
  const PJob jb = jobs[jid];
  const int m = mdim[jid];
  const int ne = which == 0 ? (jb.i == jb.j ? 0 : t.n_osv[jb.j]) : *jb.r;
  if (ne == 0) return;
  const PmEig<T> w = pm_eig<T>(pm_pair(slots, off, jid, m).wk, m);
  int ns = 0;
  const int rc = tridiag_qr_record(w.d, w.e, ne, w.swp, pm_cap_s(m), w.rot, pm_cap_r(m), &ns);
  w.hdr[0] = rc;
  w.hdr[1] = ns;
  if (rc == 1) atomicOr(err, ERR_EIG);
}

// (1a) C = 1 - M^T M, tridiagonalised, Z of the reflectors
__global__ void __launch_bounds__(NT, 3) k_pm_overlap_a(Tables t, const PJob* __restrict__ jobs,
                                                        const int* __restrict__ order, int n_jobs, double* slots,
                                                        const long long* off, int max_m, double* scratch) {
  __shared__ double gsm[GEMM_SMEM_DOUBLES];
  extern __shared__ double esm[];   // eigen-solver scratch: 4 max_m + 33 doubles
  const size_t M2 = (size_t)max_m * max_m;
  double* Cw = scratch + (size_t)blockIdx.x * pm_cta_doubles(max_m);
  double* tau = Cw + M2;
  const int n = t.n_occ;
  for (int q = blockIdx.x; q < n_jobs; q += gridDim.x) {
    const int jid = order[q];
    const PJob jb = jobs[jid];
    const int i = jb.i, j = jb.j;
    if (i == j) continue;
    const int ni = t.n_osv[i], nj = t.n_osv[j], m = ni + nj;
    const View Mv = dense_view(t.S[t.sf_id[i * n + j]], ni, nj, nj);
    cta_gemm(nj, nj, ni, -1.0, transpose(Mv), Mv, 0.0, Cw, nj, gsm);
    for (int c = threadIdx.x; c < nj; c += NT) Cw[(size_t)c * nj + c] += 1.0;
    __syncthreads();
    pm_tridiag(Cw, nj, pm_eig<double>(pm_pair(slots, off, jid, m).wk, m), tau, esm);
  }
}

// (1c) eig(C) completed (mu, V), kept directions, Y, Z^T C Z, r
__global__ void __launch_bounds__(NT, 3) k_pm_overlap_c(Tables t, double tau_s, const PJob* __restrict__ jobs,
                                                        const int* __restrict__ order, int n_jobs, double* slots,
                                                        const long long* off, int max_m, double* scratch,
                                                        int* err) {
  __shared__ double gsm[GEMM_SMEM_DOUBLES];
  extern __shared__ double esm[];   // eigen-solver scratch: 4 max_m + 33 doubles, then keep [max_m]
  int* keep = reinterpret_cast<int*>(esm + 4 * max_m + 33);
  __shared__ int s_nk;
  const size_t M2 = (size_t)max_m * max_m;
  double* C0 = scratch + (size_t)blockIdx.x * pm_cta_doubles(max_m);
  double* CZ = C0 + M2;
  double* Af = CZ + M2;         // in-CTA solve of a pair whose chase record overflowed
  double* muf = Af + M2;
  double* ef = muf + max_m;
  double* tauf = ef + max_m;
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
    cta_gemm(nj, nj, ni, -1.0, transpose(Mv), Mv, 0.0, C0, nj, gsm);
    for (int c = threadIdx.x; c < nj; c += NT) C0[(size_t)c * nj + c] += 1.0;
    __syncthreads();
    const PmEig<double> w = pm_eig<double>(pp.wk, m);
    const double* mu = w.d;
    const double* V = w.Z;      // eigenvector k of C at V[k * nj ..]
    if (w.hdr[0] == 2) {
      for (int idx = threadIdx.x; idx < nj * nj; idx += NT) Af[idx] = C0[idx];
      __syncthreads();
      if (cta_syev_cm(Af, nj, nj, muf, w.Z, nj, ef, tauf, esm) && threadIdx.x == 0) atomicOr(err, ERR_EIG);
      mu = muf;
    } else {
      apply_qr_record_cm(w.Z, nj, nj, w.swp, w.hdr[1], w.rot);
    }
    if (threadIdx.x == 0) {
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
    // (double-float products; C itself, with its cancellation, is formed in FP64 above)
    cta_gemm_df_r<4>(ni, nk, nj, -1.0, Mv, Zv, 0.0, Y + ni, r, gsm);                                     // -M Z
    cta_gemm_df_r<4>(nj, nk, nj, 1.0, dense_view(C0, nj, nj, nj), Zv, 0.0, CZ, nk, gsm);                // C Z
    cta_gemm_df_r<4>(nk, nk, nj, 1.0, transpose(Zv), dense_view(CZ, nj, nk, nk), 0.0, pp.ZCZ, nk, gsm);  // Z^T C Z
    if (threadIdx.x == 0) *jb.r = r;
  }
}

// (2) F' = Y^T F Y
__global__ void __launch_bounds__(NT, 2) k_pm_fprime(Tables t, const PJob* __restrict__ jobs,
                                                  const int* __restrict__ order, int n_jobs, double* slots,
                                                  const long long* off, int max_m, double* scratch) {
  __shared__ double sm[GEMM_SMEM_WIDE];
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
    cta_gemm_df(m, nk, m, 1.0, Fv, dense_view(pp.Y + ni, m, nk, r), 0.0, FY + ni, r, sm);
    cta_gemm_df(r, r, m, 1.0, transpose(dense_view(pp.Y, m, r, r)), dense_view(FY, m, r, r), 0.0, pp.Fp, r, sm);
  }
}

// (3a) F' symmetrised in FP32, tridiagonalised, Z of the reflectors
__global__ void __launch_bounds__(NT, 3) k_pm_eig32_a(const PJob* __restrict__ jobs, const int* __restrict__ order,
                                                      int n_jobs, double* slots, const long long* off,
                                                      const int* mdim, int max_m, double* scratch) {
  extern __shared__ float esmf[];   // eigen-solver scratch: 4 max_m + 33 floats
  float* esm = esmf;
  const size_t M2 = (size_t)max_m * max_m;
  float* A32 = reinterpret_cast<float*>(scratch + (size_t)blockIdx.x * pm_cta_doubles(max_m));
  float* tau32 = A32 + M2;
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
    pm_tridiag(A32, r, pm_eig<float>(pp.wk, m), tau32, esm);
  }
}

// (3c) eig(F') completed: W, e~
__global__ void __launch_bounds__(NT, 3) k_pm_eig32_c(const PJob* __restrict__ jobs, const int* __restrict__ order,
                                                      int n_jobs, double* slots, const long long* off,
                                                      const int* mdim, int max_m, double* scratch, int* err) {
  extern __shared__ float esmf[];   // eigen-solver scratch: 4 max_m + 33 floats
  float* esm = esmf;
  const size_t M2 = (size_t)max_m * max_m;
  float* A32 = reinterpret_cast<float*>(scratch + (size_t)blockIdx.x * pm_cta_doubles(max_m));
  float* e32 = A32 + M2;        // in-CTA solve of a pair whose chase record overflowed
  float* eb = e32 + max_m;
  float* tau32 = eb + max_m;
  for (int q = blockIdx.x; q < n_jobs; q += gridDim.x) {
    const int jid = order[q];
    const PJob jb = jobs[jid];
    const int m = mdim[jid], r = *jb.r;
    const PmPair pp = pm_pair(slots, off, jid, m);
    const PmEig<float> w = pm_eig<float>(pp.wk, m);
    const float* ev = w.d;
    if (w.hdr[0] == 2) {
      for (int idx = threadIdx.x; idx < r * r; idx += NT) {
        const int a = idx / r, b = idx % r;
        A32[idx] = (float)(0.5 * (pp.Fp[idx] + pp.Fp[(size_t)b * r + a]));
      }
      __syncthreads();
      if (cta_syev_cm(A32, r, r, e32, w.Z, r, eb, tau32, esm) && threadIdx.x == 0) atomicOr(err, ERR_EIG);
      ev = e32;
    } else {
      apply_qr_record_cm(w.Z, r, r, w.swp, w.hdr[1], w.rot);
    }
    for (int idx = threadIdx.x; idx < r * r; idx += NT) {   // W[a][t] = component a of eigenvector t
      const int tv = idx / r, a = idx % r;
      pp.W[(size_t)a * r + tv] = (double)w.Z[idx];
    }
    for (int c = threadIdx.x; c < r; c += NT) pp.et[c] = (double)ev[c];
    __syncthreads();
  }
}

// (4) X = Y W; S~ = W^T (Y^T S Y) W; F~ = W^T F' W; leftovers.  The products run in
// double-float (~48 bits): W holds FP32 values and Y^T S Y, F' are FP64 with entries
// ~1, so the leftovers (~1e-6) keep ~9 significant digits.  X = Y W (entries up to
// lambda_min(S)^(-1/2)) is double-float as well: U = P X and the leftovers are
// formed from the same X, so its ~2^-48 relative rounding does not move the
// fixed point.
__global__ void __launch_bounds__(NT, 2) k_pm_final(Tables t, const PJob* __restrict__ jobs,
                                                 const int* __restrict__ order, int n_jobs, double* slots,
                                                 const long long* off, int max_m, double* scratch, int* err) {
  __shared__ double sm[GEMM_SMEM_WIDE];
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
      cta_gemm_df(m, r, r, 1.0, dense_view(pp.Y, m, r, r), Wv, 0.0, jb.X, m, sm);       // X = Y W
      for (int idx = threadIdx.x; idx < ni * r; idx += NT) T1[idx] = pp.W[idx];        // (Y^T S Y) W, top rows
      cta_gemm_df(nk, r, nk, 1.0, dense_view(pp.ZCZ, nk, nk, nk), dense_view(pp.W + (size_t)ni * r, nk, r, r), 0.0,
               T1 + (size_t)ni * r, r, sm);
    } else {
      for (int idx = threadIdx.x; idx < m * r; idx += NT) jb.X[(size_t)(idx / r) * m + idx % r] = pp.W[idx];
      cta_gemm_df(r, r, r, 1.0, dense_view(t.S[t.sf_id[i * n + i]], ni, ni, ni), Wv, 0.0, T1, r, sm);
    }
    cta_gemm_df(r, r, r, 1.0, transpose(Wv), dense_view(T1, r, r, r), 0.0, St, r, sm);      // S~
    cta_gemm_df(r, r, r, 1.0, dense_view(pp.Fp, r, r, r), Wv, 0.0, T1, r, sm);
    cta_gemm_df(r, r, r, 1.0, transpose(Wv), dense_view(T1, r, r, r), 0.0, Ft, r, sm);      // F~
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
  const size_t sm_d = ((size_t)4 * max_m + 33) * sizeof(double) + (size_t)max_m * sizeof(int);
  const size_t sm_f = ((size_t)4 * max_m + 33) * sizeof(float);
  if (sm_d > 160 * 1024) return -1;
  if (cudaFuncSetAttribute(k_pm_overlap_a, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_d) != cudaSuccess ||
      cudaFuncSetAttribute(k_pm_overlap_c, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_d) != cudaSuccess ||
      cudaFuncSetAttribute(k_pm_eig32_a, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_f) != cudaSuccess ||
      cudaFuncSetAttribute(k_pm_eig32_c, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_f) != cudaSuccess)
    return -1;
  const int n_chase = (n_jobs + 31) / 32;
  k_pm_overlap_a<<<n_cta, NT, sm_d, st>>>(t, jobs, order, n_jobs, slots, off, max_m, scratch);
  k_pm_chase<double><<<n_chase, 32, 0, st>>>(t, jobs, order, n_jobs, slots, off, mdim, 0, err);
  k_pm_overlap_c<<<n_cta, NT, sm_d, st>>>(t, tau_s, jobs, order, n_jobs, slots, off, max_m, scratch, err);
  k_pm_fprime<<<n_cta, NT, 0, st>>>(t, jobs, order, n_jobs, slots, off, max_m, scratch);
  k_pm_eig32_a<<<n_cta, NT, sm_f, st>>>(jobs, order, n_jobs, slots, off, mdim, max_m, scratch);
  k_pm_chase<float><<<n_chase, 32, 0, st>>>(t, jobs, order, n_jobs, slots, off, mdim, 1, err);
  k_pm_eig32_c<<<n_cta, NT, sm_f, st>>>(jobs, order, n_jobs, slots, off, mdim, max_m, scratch, err);
  k_pm_final<<<n_cta, NT, 0, st>>>(t, jobs, order, n_jobs, slots, off, max_m, scratch, err);
  note_launch(8);
  return 0;
}

}  // namespace osv
