// A6 in the mixed form.  The solver keeps Y_p (T_p = X_p Y_p X_p^T) per
// fragment; with U_p = P_p X_p (orthonormal columns) every full-space
// quantity of the frozen-OSV gradient is written in the pair basis:
//   P T~ P^T = U Y~ U^T,  P (T~ S T^T) P^T = U (Y~ Y^T) U^T,
//   <T~_kj, T_lj> = <op(Y~_q1), Sigma_q1q2 op(Y_q2) Sigma_q1q2^T>,  Sigma = U_q1^T U_q2,
// so the products never pass through the ill-conditioned X.  Reductions run in
// FP64 over FP32 products, in a fixed order.
#include "pairview.cuh"

namespace osv {

// W~_p = sum c Y~, H~_p = sum c (Y~ Y^T + [i!=j] Y~^T Y)   (r x r, FP64)
__global__ void __launch_bounds__(NT) k_gradm_pair(Tables t, const GradPairJob* __restrict__ jobs, int n_jobs,
                                                   const GradContrib* __restrict__ contrib, double* scratch,
                                                   int max_m) {
  __shared__ double sm[GEMM_SMEM_DOUBLES];
  double* Yt = scratch + (size_t)blockIdx.x * max_m * max_m;
  for (int jid = blockIdx.x; jid < n_jobs; jid += gridDim.x) {
    const GradPairJob jb = jobs[jid];
    const int r = t.r[t.pair_id[jb.i * t.n_occ + jb.j]];
    for (int idx = threadIdx.x; idx < r * r; idx += NT) { jb.W[idx] = 0.0; jb.H[idx] = 0.0; }
    __syncthreads();
    for (int q = jb.c0; q < jb.c1; q++) {
      const GradContrib cb = contrib[q];
      const double* Y = cb.T;
      const double w = (double)cb.weight;
      for (int idx = threadIdx.x; idx < r * r; idx += NT) {
        const int a = idx / r, b = idx % r;
        const double yt = 2.0 * Y[idx] - Y[(size_t)b * r + a];
        Yt[idx] = yt;
        jb.W[idx] += w * yt;
      }
      __syncthreads();
      cta_gemm(r, r, r, w, dense_view(Yt, r, r, r), dense_view(Y, r, r, r, 1), 1.0, jb.H, r, sm);
      if (jb.i != jb.j) cta_gemm(r, r, r, w, dense_view(Yt, r, r, r, 1), dense_view(Y, r, r, r), 1.0, jb.H, r, sm);
    }
  }
}

// d_p[a] = (U H~ U^T)_aa
__global__ void __launch_bounds__(NT) k_gradm_de_pair(Tables t, const GradPairJob* __restrict__ jobs, int n_jobs,
                                                      double* scratch, int max_m, double* dpair) {
  __shared__ float sm[GEMM_SMEM_DOUBLES];
  const int nv = t.n_vir;
  float* M = reinterpret_cast<float*>(scratch + (size_t)blockIdx.x * nv * max_m);
  for (int jid = blockIdx.x; jid < n_jobs; jid += gridDim.x) {
    const GradPairJob jb = jobs[jid];
    const int pid = t.pair_id[jb.i * t.n_occ + jb.j];
    const int r = t.r[pid];
    const float* U = t.U[pid];
    cta_gemm_t<float, float>(nv, r, r, 1.f, ViewF{U, r, 0}, dense_view(jb.H, r, r, r), 0.f, M, r, sm);
    for (int a = threadIdx.x; a < nv; a += NT) {
      double s = 0.0;
      for (int c = 0; c < r; c++) s += (double)M[(size_t)a * r + c] * (double)U[(size_t)a * r + c];
      dpair[(size_t)jid * nv + a] = s;
    }
    __syncthreads();
  }
}

// per fragment: c_C (-sum_j <T~_kj, T_lj> - sum_i <T~_il, T_ik>) from Y and Sigma = U^T U
__device__ double ydot(const Tables& t, const int* orbs, double* const* Y, const int* pid, int nc, int x1, int y1,
                       int x2, int y2, float* W, float* V, double* red, float* sm) {
  const int a1 = min(x1, y1), b1 = max(x1, y1), t1 = x1 > y1;
  const int a2 = min(x2, y2), b2 = max(x2, y2), t2 = x2 > y2;
  const int lp1 = a1 * nc - a1 * (a1 - 1) / 2 + (b1 - a1);
  const int lp2 = a2 * nc - a2 * (a2 - 1) / 2 + (b2 - a2);
  const int r1 = t.r[pid[lp1]], r2 = t.r[pid[lp2]];
  const float* U1 = t.U[pid[lp1]];
  const float* U2 = t.U[pid[lp2]];
  // Sigma = U1^T U2 (r1 x r2) -> W ; V = Sigma op2(Y2) Sigma^T
  cta_gemm_t<float, float>(r1, r2, t.n_vir, 1.f, ViewF{U1, r1, 1}, ViewF{U2, r2, 0}, 0.f, W, r2, sm);
  float* Z = V + (size_t)r1 * r1;
  cta_gemm_t<float, float>(r1, r2, r2, 1.f, ViewF{W, r2, 0}, dense_view(Y[lp2], r2, r2, r2, t2), 0.f, Z, r2, sm);
  cta_gemm_t<float, float>(r1, r1, r2, 1.f, ViewF{Z, r2, 0}, ViewF{W, r2, 1}, 0.f, V, r1, sm);
  const double* A = Y[lp1];
  double s = 0.0;
  for (int idx = threadIdx.x; idx < r1 * r1; idx += NT) {
    const int rr = idx / r1, cc = idx % r1;
    const double tr_ = t1 ? A[(size_t)cc * r1 + rr] : A[idx];
    const double tc_ = t1 ? A[idx] : A[(size_t)cc * r1 + rr];
    s += (2.0 * tr_ - tc_) * (double)V[idx];
  }
  return cta_sum(s, red);
}

__global__ void __launch_bounds__(NT) k_gradm_df_frag(Tables t, const int* __restrict__ frag_orbs,
                                                      const int* __restrict__ weights, const double* Tstore,
                                                      const long long* __restrict__ Toff, int n_frag, int max_m,
                                                      double* scratch, double* out) {
  __shared__ float sm[GEMM_SMEM_DOUBLES];
  __shared__ double red[40];
  const size_t M2 = (size_t)max_m * max_m;
  float* W = reinterpret_cast<float*>(scratch + (size_t)blockIdx.x * 2 * M2);
  float* V = W + M2;
  for (int f = blockIdx.x; f < n_frag; f += gridDim.x) {
    int orbs[3], nc = 0;
    for (int u = 0; u < 3; u++)
      if (frag_orbs[3 * f + u] >= 0) orbs[nc++] = frag_orbs[3 * f + u];
    double* Y[6];
    int pid[6];
    double* base = const_cast<double*>(Tstore) + Toff[f];
    {
      size_t off = 0;
      for (int a = 0; a < nc; a++)
        for (int b = a; b < nc; b++) {
          const int lp = a * nc - a * (a - 1) / 2 + (b - a);
          Y[lp] = base + off;
          pid[lp] = t.pair_id[orbs[a] * t.n_occ + orbs[b]];
          const size_t m = pair_dim(t, orbs[a], orbs[b]);
          off += m * m;
        }
    }
    const double c = (double)weights[f];
    for (int k = 0; k < nc; k++)
      for (int l = 0; l < nc; l++) {
        double g = 0.0;
        for (int j = 0; j < nc; j++) g -= ydot(t, orbs, Y, pid, nc, k, j, l, j, W, V, red, sm);
        for (int i = 0; i < nc; i++) g -= ydot(t, orbs, Y, pid, nc, i, l, i, k, W, V, red, sm);
        if (threadIdx.x == 0) out[(size_t)f * 9 + k * 3 + l] = c * g;
      }
    __syncthreads();
  }
}

// Z = op(W~) G_partner   [r][n_aux].  grid: (job, P tile, mu tile)
__global__ void __launch_bounds__(NT) k_gradm_Z(int n_aux, const GradZJob* __restrict__ jobs) {
  __shared__ float sm[GEMM_SMEM_DOUBLES];
  const GradZJob jb = jobs[blockIdx.x];
  const int m0 = blockIdx.z * TM, n0 = blockIdx.y * TN;
  if (m0 >= jb.r) return;
  float acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; u++)
#pragma unroll
    for (int v = 0; v < 4; v++) acc[u][v] = 0.f;
  tile_mma_t<float>(jb.r, n_aux, jb.r, m0, n0, dense_view(jb.W, jb.r, jb.r, jb.r, jb.trans), ViewF{jb.G, n_aux, 0},
                    acc, sm);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int u = 0; u < 4; u++)
#pragma unroll
    for (int v = 0; v < 4; v++) {
      const int rr = m0 + ty + 16 * u, c = n0 + tx + 16 * v;
      if (rr < jb.r && c < n_aux) jb.Z[(size_t)rr * n_aux + c] = acc[u][v];
    }
}

// dB_o[a][P] = 4 sum over (pair, side) terms of U_p[a][:] Z[:][P].  grid: (orbital job, P tile, a tile)
__global__ void __launch_bounds__(NT) k_gradm_dB(int n_vir, int n_aux, const GradBJob* __restrict__ jobs,
                                                 const GradMBTerm* __restrict__ terms, double* dB) {
  __shared__ float sm[GEMM_SMEM_DOUBLES];
  const GradBJob jb = jobs[blockIdx.x];
  const int m0 = blockIdx.z * TM, n0 = blockIdx.y * TN;
  float acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; u++)
#pragma unroll
    for (int v = 0; v < 4; v++) acc[u][v] = 0.f;
  for (int q = jb.t0; q < jb.t1; q++) {
    const GradMBTerm tm = terms[q];
    tile_mma_t<float>(n_vir, n_aux, tm.r, m0, n0, ViewF{tm.U, tm.r, 0}, ViewF{tm.Z, n_aux, 0}, acc, sm);
  }
  double* out = dB + (size_t)jb.i * n_vir * n_aux;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int u = 0; u < 4; u++)
#pragma unroll
    for (int v = 0; v < 4; v++) {
      const int rr = m0 + ty + 16 * u, c = n0 + tx + 16 * v;
      if (rr < n_vir && c < n_aux) out[(size_t)rr * n_aux + c] = 4.0 * (double)acc[u][v];
    }
}

void launch_gradm_pair(const Tables& t, const GradPairJob* jobs, int n_jobs, const GradContrib* contrib,
                       double* scratch, int n_cta, int max_m, cudaStream_t st) {
  if (!n_jobs) return;
  k_gradm_pair<<<n_cta, NT, 0, st>>>(t, jobs, n_jobs, contrib, scratch, max_m);
  note_launch(1);
}
void launch_gradm_de(const Tables& t, const GradPairJob* jobs, int n_jobs, double* scratch, int n_cta, int max_m,
                     double* dpair, double* de, cudaStream_t st) {
  if (!n_jobs) return;
  k_gradm_de_pair<<<n_cta, NT, 0, st>>>(t, jobs, n_jobs, scratch, max_m, dpair);
  note_launch(1);
  launch_grad_de_reduce(dpair, n_jobs, t.n_vir, de, st);
}
void launch_gradm_df(const Tables& t, const int* frag_orbs, const int* weights, const double* Tstore,
                     const long long* Toff, int n_frag, int max_m, double* scratch, int n_cta, double* gfrag,
                     const int* fptr, const int* flist, double* df, cudaStream_t st) {
  if (!n_frag) return;
  k_gradm_df_frag<<<n_cta, NT, 0, st>>>(t, frag_orbs, weights, Tstore, Toff, n_frag, max_m, scratch, gfrag);
  note_launch(1);
  launch_grad_df_reduce(t, frag_orbs, gfrag, n_frag, fptr, flist, df, st);
}
void launch_gradm_Z(int n_aux, const GradZJob* jobs, int n_jobs, int max_r, cudaStream_t st) {
  if (!n_jobs) return;
  dim3 grid(n_jobs, (n_aux + TN - 1) / TN, (max_r + TM - 1) / TM);
  k_gradm_Z<<<grid, NT, 0, st>>>(n_aux, jobs);
  note_launch(1);
}
void launch_gradm_dB(int n_vir, int n_aux, const GradBJob* jobs, int n_jobs, const GradMBTerm* terms, double* dB,
                     cudaStream_t st) {
  if (!n_jobs) return;
  dim3 grid(n_jobs, (n_aux + TN - 1) / TN, (n_vir + TM - 1) / TM);
  k_gradm_dB<<<grid, NT, 0, st>>>(n_vir, n_aux, jobs, terms, dB);
  note_launch(1);
}

}  // namespace osv
