// A6: frozen-OSV gradient of the MBE(3) energy.  With the amplitudes of every
// fragment stationary (Eq. res_close is the stationarity condition of the
// Hylleraas functional, Section 2), dE/dtheta is the explicit derivative of
// that functional at the converged amplitudes:
//   dE/dB_i  = 4 sum_C c_C sum_j T~_ij B_j
//   dE/de_a  = 2 sum_C c_C sum_ij sum_b T~_ij^ab T_ij^ab
//   dE/df_kl = -sum_C c_C [sum_j <T~_kj, T_lj> + sum_i <T~_il, T_ik>]   (symmetrised)
// with T~ = 2T - T^T in the full virtual space, evaluated here in the OSV pair
// bases.  Every sum over fragments runs in a fixed order (deterministic).
#include "pairview.cuh"

namespace osv {

// ---- per pair: W_p = sum_C c_C T~_p and H_p = sum_C c_C (T~ S T^T + [i!=j] T~^T S T)
__global__ void __launch_bounds__(NT) k_grad_pair(Tables t, const GradPairJob* __restrict__ jobs, int n_jobs,
                                                  const GradContrib* __restrict__ contrib, double* scratch,
                                                  int max_m) {
  __shared__ double sm[GEMM_SMEM_DOUBLES];
  const size_t M2 = (size_t)max_m * max_m;
  double* Tt = scratch + (size_t)blockIdx.x * 2 * M2;   // T~ of one fragment
  double* G = Tt + M2;                                   // T~ S (or T~^T S)
  for (int jid = blockIdx.x; jid < n_jobs; jid += gridDim.x) {
    const GradPairJob jb = jobs[jid];
    const int m = pair_dim(t, jb.i, jb.j);
    const View Sp = pair_view(t, t.S, jb.i, jb.j, jb.i, jb.j);
    for (int idx = threadIdx.x; idx < m * m; idx += NT) { jb.W[idx] = 0.0; jb.H[idx] = 0.0; }
    __syncthreads();
    for (int q = jb.c0; q < jb.c1; q++) {
      const GradContrib cb = contrib[q];
      const double* T = cb.T;
      const double w = (double)cb.weight;
      for (int idx = threadIdx.x; idx < m * m; idx += NT) {
        const int r = idx / m, c = idx % m;
        const double tt = 2.0 * T[idx] - T[(size_t)c * m + r];
        Tt[idx] = tt;
        jb.W[idx] += w * tt;
      }
      __syncthreads();
      const View Tv = dense_view(T, m, m, m);
      cta_gemm(m, m, m, 1.0, dense_view(Tt, m, m, m), Sp, 0.0, G, m, sm);
      cta_gemm(m, m, m, w, dense_view(G, m, m, m), transpose(Tv), 1.0, jb.H, m, sm);
      if (jb.i != jb.j) {
        cta_gemm(m, m, m, 1.0, dense_view(Tt, m, m, m, 1), Sp, 0.0, G, m, sm);
        cta_gemm(m, m, m, w, dense_view(G, m, m, m), Tv, 1.0, jb.H, m, sm);
      }
    }
  }
}

// ---- per pair: d_p[a] = (P H_p P^T)_aa
__global__ void __launch_bounds__(NT) k_grad_de_pair(Tables t, const GradPairJob* __restrict__ jobs, int n_jobs,
                                                     double* scratch, int max_m, double* dpair) {
  __shared__ double sm[GEMM_SMEM_DOUBLES];
  const int nv = t.n_vir;
  double* M = scratch + (size_t)blockIdx.x * (size_t)nv * max_m;   // P H  [nv][m]
  for (int jid = blockIdx.x; jid < n_jobs; jid += gridDim.x) {
    const GradPairJob jb = jobs[jid];
    const int ni = t.n_osv[jb.i], nj = (jb.i == jb.j) ? 0 : t.n_osv[jb.j];
    const int m = ni + nj;
    View P;
    P.rows = nv; P.cols = m; P.rs = nv; P.cs = ni;
    P.b[0][0] = P.b[1][0] = Blk{t.Q[jb.i], ni, 0};
    P.b[0][1] = P.b[1][1] = Blk{nj ? t.Q[jb.j] : t.Q[jb.i], nj ? nj : ni, 0};
    cta_gemm(nv, m, m, 1.0, P, dense_view(jb.H, m, m, m), 0.0, M, m, sm);
    for (int a = threadIdx.x; a < nv; a += NT) {
      double s = 0.0;
      for (int c = 0; c < m; c++) s += M[(size_t)a * m + c] * P.get(a, c);
      dpair[(size_t)jid * nv + a] = s;
    }
    __syncthreads();
  }
}

// dE/de[a] = 2 sum_p d_p[a] (fixed pair order)
__global__ void k_grad_de_reduce(const double* __restrict__ dpair, int n_pairs, int nv, double* de) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < nv; a += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int p = 0; p < n_pairs; p++) s += dpair[(size_t)p * nv + a];
    de[a] = 2.0 * s;
  }
}

// ---- per fragment: c_C * (-sum_j <T~_kj, T_lj> - sum_i <T~_il, T_ik>) for k, l in C
// Full-space inner product of two ordered-pair amplitudes expressed in their
// stored bases q1, q2 (transposed when the ordered pair is reversed):
// <P1 op1(A) P1^T, P2 op2(B) P2^T> = <op1(A), S_(q1,q2) op2(B) S_(q1,q2)^T>.
__device__ double full_dot(const Tables& t, const int* orbs, double* const* T, int nc, int x1, int y1, int x2, int y2,
                           double* W, double* V, double* red, double* sm) {
  const int a1 = min(x1, y1), b1 = max(x1, y1), t1 = x1 > y1;
  const int a2 = min(x2, y2), b2 = max(x2, y2), t2 = x2 > y2;
  const int gi1 = orbs[a1], gj1 = orbs[b1], gi2 = orbs[a2], gj2 = orbs[b2];
  const int m1 = pair_dim(t, gi1, gj1), m2 = pair_dim(t, gi2, gj2);
  const int lp1 = a1 * nc - a1 * (a1 - 1) / 2 + (b1 - a1);
  const int lp2 = a2 * nc - a2 * (a2 - 1) / 2 + (b2 - a2);
  const View S12 = pair_view(t, t.S, gi1, gj1, gi2, gj2);
  cta_gemm(m1, m2, m2, 1.0, S12, dense_view(T[lp2], m2, m2, m2, t2), 0.0, W, m2, sm);
  cta_gemm(m1, m1, m2, 1.0, dense_view(W, m1, m2, m2), transpose(S12), 0.0, V, m1, sm);
  const double* A = T[lp1];
  double s = 0.0;
  for (int idx = threadIdx.x; idx < m1 * m1; idx += NT) {
    const int r = idx / m1, c = idx % m1;
    // op1(T~)[r][c] with T~ = 2T - T^T
    const double tr_ = t1 ? A[(size_t)c * m1 + r] : A[idx];
    const double tc_ = t1 ? A[idx] : A[(size_t)c * m1 + r];
    s += (2.0 * tr_ - tc_) * V[idx];
  }
  return cta_sum(s, red);
}

__global__ void __launch_bounds__(NT) k_grad_df_frag(Tables t, const int* __restrict__ frag_orbs,
                                                     const int* __restrict__ weights, const double* Tstore,
                                                     const long long* __restrict__ Toff, int n_frag, int max_m,
                                                     double* scratch, double* out /*[n_frag][9]*/) {
  __shared__ double sm[GEMM_SMEM_DOUBLES];
  __shared__ double red[40];
  const size_t M2 = (size_t)max_m * max_m;
  double* W = scratch + (size_t)blockIdx.x * 2 * M2;
  double* V = W + M2;
  for (int f = blockIdx.x; f < n_frag; f += gridDim.x) {
    int orbs[3], nc = 0;
    for (int u = 0; u < 3; u++)
      if (frag_orbs[3 * f + u] >= 0) orbs[nc++] = frag_orbs[3 * f + u];
    double* T[6];
    double* base = const_cast<double*>(Tstore) + Toff[f];
    {
      size_t off = 0;
      for (int a = 0; a < nc; a++)
        for (int b = a; b < nc; b++) {
          T[a * nc - a * (a - 1) / 2 + (b - a)] = base + off;
          const size_t m = pair_dim(t, orbs[a], orbs[b]);
          off += m * m;
        }
    }
    const double c = (double)weights[f];
    for (int k = 0; k < nc; k++)
      for (int l = 0; l < nc; l++) {
        double g = 0.0;
        for (int j = 0; j < nc; j++) g -= full_dot(t, orbs, T, nc, k, j, l, j, W, V, red, sm);
        for (int i = 0; i < nc; i++) g -= full_dot(t, orbs, T, nc, i, l, i, k, W, V, red, sm);
        if (threadIdx.x == 0) out[(size_t)f * 9 + k * 3 + l] = c * g;
      }
    __syncthreads();
  }
}

// dE/df = sym(sum_f G_f) in fragment order; one thread per (k, l).
__global__ void k_grad_df_reduce(const int* __restrict__ frag_orbs, const double* __restrict__ gfrag, int n_frag,
                                 int n_occ, const int* __restrict__ fptr, const int* __restrict__ flist,
                                 double* df) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_occ * n_occ; e += gridDim.x * blockDim.x) {
    const int k = e / n_occ, l = e % n_occ;
    double s = 0.0;
    // fragments containing orbital k, ascending
    for (int q = fptr[k]; q < fptr[k + 1]; q++) {
      const int f = flist[q];
      int a = -1, b = -1;
      for (int u = 0; u < 3; u++) {
        if (frag_orbs[3 * f + u] == k) a = u;
        if (frag_orbs[3 * f + u] == l) b = u;
      }
      if (b < 0) continue;
      // local indices among the non-negative entries (fragments are stored packed, -1 padded)
      s += 0.5 * (gfrag[(size_t)f * 9 + a * 3 + b] + gfrag[(size_t)f * 9 + b * 3 + a]);
    }
    df[e] = s;
  }
}

// ---- Y_o^(x)[mu][P] = sum over contributions of rows of W'_p times (P_p^T B_partner)
__global__ void __launch_bounds__(NT) k_grad_Y(Tables t, int n_aux, const GradYJob* __restrict__ jobs,
                                               const GradYTerm* __restrict__ terms) {
  __shared__ double sm[GEMM_SMEM_DOUBLES];
  const GradYJob jb = jobs[blockIdx.x];
  const int nx = t.n_osv[jb.x];
  const int m0 = blockIdx.z * TM, n0 = blockIdx.y * TN;
  if (m0 >= nx) return;
  double acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; u++)
#pragma unroll
    for (int v = 0; v < 4; v++) acc[u][v] = 0.0;
  for (int q = jb.t0; q < jb.t1; q++) {
    const GradYTerm tm = terms[q];
    const int ni = t.n_osv[tm.pi], nj = (tm.pi == tm.pj) ? 0 : t.n_osv[tm.pj];
    const int m = ni + nj;
    // A(mu, nu) = W'[row0 + mu][nu], W' = W or W^T
    View A = dense_view(tm.W + (tm.trans ? tm.row0 : (size_t)tm.row0 * m), nx, m, m, tm.trans);
    // B(nu, P) = (P_p^T B_partner)[nu][P] from the stored projections
    View Bv;
    Bv.rows = m; Bv.cols = n_aux; Bv.rs = ni; Bv.cs = n_aux;
    Bv.b[0][0] = Bv.b[0][1] = Blk{tm.Bt_i, ni, 1};
    Bv.b[1][0] = Bv.b[1][1] = Blk{nj ? tm.Bt_j : tm.Bt_i, nj ? nj : ni, 1};
    tile_mma(nx, n_aux, m, m0, n0, A, Bv, acc, sm);
  }
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int u = 0; u < 4; u++)
#pragma unroll
    for (int v = 0; v < 4; v++) {
      const int r = m0 + ty + 16 * u, c = n0 + tx + 16 * v;
      if (r < nx && c < n_aux) jb.Y[(size_t)r * n_aux + c] = acc[u][v];
    }
}

// ---- dB_i[a][P] = 4 sum_x sum_mu Q_x[a][mu] Y_i^(x)[mu][P]
__global__ void __launch_bounds__(NT) k_grad_dB(Tables t, int n_aux, const GradBJob* __restrict__ jobs,
                                                const GradBTerm* __restrict__ terms, double* dB) {
  __shared__ double sm[GEMM_SMEM_DOUBLES];
  const GradBJob jb = jobs[blockIdx.x];
  const int nv = t.n_vir;
  const int m0 = blockIdx.z * TM, n0 = blockIdx.y * TN;
  double acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; u++)
#pragma unroll
    for (int v = 0; v < 4; v++) acc[u][v] = 0.0;
  for (int q = jb.t0; q < jb.t1; q++) {
    const GradBTerm tm = terms[q];
    const int nx = t.n_osv[tm.x];
    tile_mma(nv, n_aux, nx, m0, n0, dense_view(t.Q[tm.x], nv, nx, nx), dense_view(tm.Y, nx, n_aux, n_aux), acc, sm);
  }
  double* out = dB + (size_t)jb.i * nv * n_aux;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int u = 0; u < 4; u++)
#pragma unroll
    for (int v = 0; v < 4; v++) {
      const int r = m0 + ty + 16 * u, c = n0 + tx + 16 * v;
      if (r < nv && c < n_aux) out[(size_t)r * n_aux + c] = 4.0 * acc[u][v];
    }
}

// ---------------------------------------------------------------- launchers
void launch_grad_pair(const Tables& t, const GradPairJob* jobs, int n_jobs, const GradContrib* contrib,
                      double* scratch, int n_cta, int max_m, cudaStream_t st) {
  if (!n_jobs) return;
  k_grad_pair<<<n_cta, NT, 0, st>>>(t, jobs, n_jobs, contrib, scratch, max_m);
  note_launch(1);
}
void launch_grad_de(const Tables& t, const GradPairJob* jobs, int n_jobs, double* scratch, int n_cta, int max_m,
                    double* dpair, double* de, cudaStream_t st) {
  if (!n_jobs) return;
  k_grad_de_pair<<<n_cta, NT, 0, st>>>(t, jobs, n_jobs, scratch, max_m, dpair);
  note_launch(1);
  k_grad_de_reduce<<<(t.n_vir + 255) / 256, 256, 0, st>>>(dpair, n_jobs, t.n_vir, de);
  note_launch(1);
}
void launch_grad_df(const Tables& t, const int* frag_orbs, const int* weights, const double* Tstore,
                    const long long* Toff, int n_frag, int max_m, double* scratch, int n_cta, double* gfrag,
                    const int* fptr, const int* flist, double* df, cudaStream_t st) {
  if (!n_frag) return;
  k_grad_df_frag<<<n_cta, NT, 0, st>>>(t, frag_orbs, weights, Tstore, Toff, n_frag, max_m, scratch, gfrag);
  note_launch(1);
  k_grad_df_reduce<<<(t.n_occ * t.n_occ + 255) / 256, 256, 0, st>>>(frag_orbs, gfrag, n_frag, t.n_occ, fptr, flist,
                                                                     df);
  note_launch(1);
}
void launch_grad_de_reduce(const double* dpair, int n_pairs, int nv, double* de, cudaStream_t st) {
  k_grad_de_reduce<<<(nv + 255) / 256, 256, 0, st>>>(dpair, n_pairs, nv, de);
  note_launch(1);
}
void launch_grad_df_reduce(const Tables& t, const int* frag_orbs, const double* gfrag, int n_frag, const int* fptr,
                           const int* flist, double* df, cudaStream_t st) {
  k_grad_df_reduce<<<(t.n_occ * t.n_occ + 255) / 256, 256, 0, st>>>(frag_orbs, gfrag, n_frag, t.n_occ, fptr, flist,
                                                                     df);
  note_launch(1);
}
void launch_grad_Y(const Tables& t, int n_aux, const GradYJob* jobs, int n_jobs, const GradYTerm* terms, int max_n,
                   cudaStream_t st) {
  if (!n_jobs) return;
  dim3 grid(n_jobs, (n_aux + TN - 1) / TN, (max_n + TM - 1) / TM);
  k_grad_Y<<<grid, NT, 0, st>>>(t, n_aux, jobs, terms);
  note_launch(1);
}
void launch_grad_dB(const Tables& t, int n_aux, const GradBJob* jobs, int n_jobs, const GradBTerm* terms, double* dB,
                    cudaStream_t st) {
  if (!n_jobs) return;
  dim3 grid(n_jobs, (n_aux + TN - 1) / TN, (t.n_vir + TM - 1) / TM);
  k_grad_dB<<<grid, NT, 0, st>>>(t, n_aux, jobs, terms, dB);
  note_launch(1);
}

}  // namespace osv
