// A3: preconditioner of every pair, F_(ij,ij) X = S_(ij,ij) X E~ (Eq. prec_eig),
// solved as canonical orthogonalisation of S (eigenvalues below tau_s * max
// dropped) followed by the eigen-decomposition of Y^T F Y; X = Y W.
#include "eig.cuh"
#include "pairview.cuh"

namespace osv {

constexpr int ZMAX_P = 144;   // eigenvector matrix kept in shared memory up to this order

__global__ void __launch_bounds__(NT) k_precond(Tables t, double tau_s, const PJob* __restrict__ jobs, int n_jobs,
                                                int max_m, double* scratch, int* err) {
  extern __shared__ double dyn[];
  __shared__ int s_r;
  double* gsm = dyn;                                   // GEMM tiles
  double* esm = dyn + GEMM_SMEM_DOUBLES;               // eigen-solver scratch (4 max_m + 64)
  double* zsm = esm + 4 * max_m + 64;                  // Z in shared memory (ZMAX_P x (ZMAX_P+1))
  int* keep = reinterpret_cast<int*>(esm);             // reused after the S eigen-solve
  const size_t M2 = (size_t)max_m * max_m;
  double* base = scratch + (size_t)blockIdx.x * precond_scratch_doubles(max_m);
  double* Sw = base;
  double* Fw = Sw + M2;
  double* Zg = Fw + M2;
  double* Yw = Zg + M2;
  double* W1 = Yw + M2;
  double* Fp = W1 + M2;
  double* e = Fp + M2;
  double* tau = e + max_m;
  double* ws = tau + max_m;
  double* w2 = ws + max_m;
  for (int jid = blockIdx.x; jid < n_jobs; jid += gridDim.x) {
    const PJob jb = jobs[jid];
    const int m = pair_dim(t, jb.i, jb.j);
    const View Sv = pair_view(t, t.S, jb.i, jb.j, jb.i, jb.j);
    const View Fv = pair_view(t, t.F, jb.i, jb.j, jb.i, jb.j);
    for (int idx = threadIdx.x; idx < m * m; idx += NT) {
      const int r = idx / m, c = idx % m;
      Sw[idx] = Sv.get(r, c);
      Fw[idx] = Fv.get(r, c);
    }
    __syncthreads();
    double* Z = (m <= ZMAX_P) ? zsm : Zg;
    const int ldz = (m <= ZMAX_P) ? m + 1 : m;
    int rc = cta_syev(Sw, m, m, ws, Z, ldz, e, tau, esm);
    if (threadIdx.x == 0) {
      double smax = 0.0;
      for (int c = 0; c < m; c++) smax = fmax(smax, ws[c]);
      int r = 0;
      for (int c = 0; c < m; c++)
        if (ws[c] > tau_s * smax) keep[r++] = c;
      s_r = r;
      if (rc) atomicOr(err, ERR_EIG);
    }
    __syncthreads();
    const int r = s_r;
    for (int idx = threadIdx.x; idx < m * r; idx += NT) {
      const int row = idx / r, c = idx % r;
      const int kc = keep[c];
      Yw[(size_t)row * m + c] = Z[(size_t)row * ldz + kc] / sqrt(ws[kc]);
    }
    __syncthreads();
    const View Yv = dense_view(Yw, m, r, m);
    cta_gemm(m, r, m, 1.0, dense_view(Fw, m, m, m), Yv, 0.0, W1, m, gsm);
    cta_gemm(r, r, m, 1.0, transpose(Yv), dense_view(W1, m, r, m), 0.0, Fp, r, gsm);
    double* Z2 = (r <= ZMAX_P) ? zsm : Zg;
    const int ldz2 = (r <= ZMAX_P) ? r + 1 : r;
    rc = cta_syev(Fp, r, r, w2, Z2, ldz2, e, tau, esm);
    if (threadIdx.x == 0 && rc) atomicOr(err, ERR_EIG);
    cta_gemm(m, r, r, 1.0, Yv, dense_view(Z2, r, r, ldz2), 0.0, jb.X, m, gsm);
    for (int c = threadIdx.x; c < r; c += NT) {
      jb.et[c] = w2[c];
      if (!isfinite(w2[c])) atomicOr(err, ERR_NONFINITE);
    }
    if (threadIdx.x == 0) *jb.r = r;
    __syncthreads();
  }
}

void launch_precond(const Tables& t, double tau_s, const PJob* jobs, int n_jobs, int max_m, double* scratch,
                    int n_cta, int* err, cudaStream_t st) {
  if (n_jobs == 0) return;
  const size_t smem = (size_t)(GEMM_SMEM_DOUBLES + 4 * max_m + 64 + ZMAX_P * (ZMAX_P + 1)) * sizeof(double);
  cudaFuncSetAttribute(k_precond, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_precond<<<n_cta, NT, smem, st>>>(t, tau_s, jobs, n_jobs, max_m, scratch, err);
  note_launch(1);
}

}  // namespace osv
