// A6, OSV-relaxed part: the response of the kept OSVs of Eq. osv_gen to T_ii of
// Eq. mp2_tkk, added to the frozen-OSV gradient (FP64 form).
//
// With the amplitudes stationary, E is the Hylleraas functional of the frozen
// gradient with T_p(full) = P_p T_p P_p^T, and per stored pair p = (i, j)
//   dE/dP_p = alpha_p [R~_p P_p T_p^T + R~_p^T P_p T_p]     (alpha = 4 for i < j, 2 for i = j)
// summed over the fragments with their weights, where
//   R_p = B_i B_j^T + diag(e) T_p + T_p diag(e) - sum_k (f_ik T_kj + f_kj T_ik)
// is the full-space residual of Eq. res_close and R~ = 2R - R^T; the columns of
// dP_p that belong to Q_x are dQ_x.  The exchange part is linear in the
// amplitudes and runs once per pair on W~_p = sum_C c_C T~_p:
//   alpha [B_i (A_j W~^T) + B_j (A_i W~)],  A_x = B_x^T P_p  (the stored projections);
// the rest runs per fragment in the full virtual space.  Then, per orbital x,
// with the eigenpairs (omega, z) of T_xx (descending) and the OSV count n_x
// held fixed (the energy jumps where an eigenvalue crosses l_osv):
//   Y_lk = z_l^T g_k / (omega_k - omega_l) over the discarded l,
//   Z = (Z_d Y Q_x^T + Q_x Y^T Z_d^T) / 2,  D_ab = e_a + e_b - 2 f_xx,
//   dE/dB_x += 2 (Z / D) B_x,  dE/de_a -= 2 sum_b (Z T / D)_ab,  dE/df_xx += 2 sum (Z T / D).
// Every sum runs in a fixed order (deterministic).
#include "pairview.cuh"

namespace osv {

namespace {

struct BRows {   // B_i as an n_vir x n_aux matrix
  BSrc s;
  int i;
  __device__ __forceinline__ double get(int a, int P) const { return s.get(i, a, P); }
};

// P_p = [Q_i Q_j] (n_vir x m); P_ii = Q_i
__device__ inline View pbasis(const Tables& t, int i, int j) {
  const int nv = t.n_vir, ni = t.n_osv[i];
  if (i == j) return dense_view(t.Q[i], nv, ni, ni);
  const int nj = t.n_osv[j];
  View v;
  v.rows = nv; v.cols = ni + nj; v.rs = nv; v.cs = ni;
  v.b[0][0] = v.b[1][0] = Blk{t.Q[i], ni, 0};
  v.b[0][1] = v.b[1][1] = Blk{t.Q[j], nj, 0};
  return v;
}

// A = B_a^T P_p (n_aux x m) from the stored projections B_a^T Q_x ([n_aux][n_x])
__device__ inline View proj_view(const RelaxKJob& jb, int side, int ni, int nj, int n_aux) {
  if (jb.i == jb.j) return dense_view(jb.bt_ii, n_aux, ni, ni);
  const double* left = side ? jb.bt_ji : jb.bt_ii;    // B_a^T Q_i
  const double* right = side ? jb.bt_jj : jb.bt_ij;   // B_a^T Q_j
  View v;
  v.rows = n_aux; v.cols = ni + nj; v.rs = n_aux; v.cs = ni;
  v.b[0][0] = v.b[1][0] = Blk{left, ni, 0};
  v.b[0][1] = v.b[1][1] = Blk{right, nj, 0};
  return v;
}

}  // namespace

// ---- exchange part, one CTA per stored pair: out = alpha [B_i (A_j W~^T) + B_j (A_i W~)]
__global__ void __launch_bounds__(NT) k_relax_kpart(Tables t, BSrc bs, const RelaxKJob* __restrict__ jobs,
                                                    int n_jobs, double* scratch, int max_m) {
  __shared__ double sm[GEMM_SMEM_DOUBLES];
  const int nx = bs.n_aux, nv = t.n_vir;
  double* M1 = scratch + (size_t)blockIdx.x * 2 * nx * max_m;
  double* M2 = M1 + (size_t)nx * max_m;
  for (int jid = blockIdx.x; jid < n_jobs; jid += gridDim.x) {
    const RelaxKJob jb = jobs[jid];
    const int i = jb.i, j = jb.j, ni = t.n_osv[i], nj = (i == j) ? 0 : t.n_osv[j], m = ni + nj;
    const double alpha = (i == j) ? 2.0 : 4.0;
    const View W = dense_view(jb.W, m, m, m);
    cta_gemm(nx, m, m, 1.0, proj_view(jb, 1, ni, nj, nx), transpose(W), 0.0, M1, m, sm);   // A_j W~^T
    cta_gemm(nx, m, m, 1.0, proj_view(jb, 0, ni, nj, nx), W, 0.0, M2, m, sm);              // A_i W~
    cta_gemm(nv, m, nx, alpha, BRows{bs, i}, dense_view(M1, nx, m, m), 0.0, jb.out, m, sm);
    cta_gemm(nv, m, nx, alpha, BRows{bs, j}, dense_view(M2, nx, m, m), 1.0, jb.out, m, sm);
  }
}

// ---- the rest, one CTA per fragment in the full virtual space; the Q_x columns of
// every pair's dP are summed (in pair order) into the fragment's slot of orbital x.
__global__ void __launch_bounds__(NT) k_relax_frag(Tables t, const double* __restrict__ e_vir,
                                                   const RelaxFragJob* __restrict__ jobs, int n_jobs,
                                                   double* scratch, size_t scr_per, int max_m) {
  __shared__ double sm[GEMM_SMEM_DOUBLES];
  const int nv = t.n_vir, n = t.n_occ;
  const size_t V2 = (size_t)nv * nv;
  double* TF = scratch + (size_t)blockIdx.x * scr_per;   // up to 6 pairs, nv x nv each
  double* XL = TF + 6 * V2;
  double* Y = XL + V2;                                    // P T    [nv][m]
  double* Yt = Y + (size_t)nv * max_m;                    // P T^T  [nv][m]
  double* Dt = Yt + (size_t)nv * max_m;                   // dP     [nv][m]
  for (int jid = blockIdx.x; jid < n_jobs; jid += gridDim.x) {
    const RelaxFragJob jb = jobs[jid];
    const int no = jb.no;
    int pi[6], pj[6], pm[6], uid[9];
    const double* Tp[6];
    int np = 0;
    size_t off = 0;
    for (int a = 0; a < no; a++)
      for (int b = a; b < no; b++) {
        pi[np] = jb.orbs[a];
        pj[np] = jb.orbs[b];
        pm[np] = pair_dim(t, pi[np], pj[np]);
        Tp[np] = jb.T + off;
        off += (size_t)pm[np] * pm[np];
        uid[a * 3 + b] = uid[b * 3 + a] = np;
        np++;
      }
    for (int a = 0; a < no; a++) {
      const size_t len = (size_t)nv * t.n_osv[jb.orbs[a]];
      for (size_t idx = threadIdx.x; idx < len; idx += NT) jb.slot[a][idx] = 0.0;
    }
    // full-space amplitudes T_u = P_u T_u P_u^T
    for (int u = 0; u < np; u++) {
      const int m = pm[u];
      const View P = pbasis(t, pi[u], pj[u]);
      cta_gemm(nv, m, m, 1.0, P, dense_view(Tp[u], m, m, m), 0.0, Y, m, sm);
      cta_gemm(nv, nv, m, 1.0, dense_view(Y, nv, m, m), transpose(P), 0.0, TF + (size_t)u * V2, nv, sm);
    }
    for (int u = 0; u < np; u++) {
      const int i = pi[u], j = pj[u], m = pm[u];
      int ai = 0, aj = 0;
      for (int a = 0; a < no; a++) {
        if (jb.orbs[a] == i) ai = a;
        if (jb.orbs[a] == j) aj = a;
      }
      const double scale = ((i == j) ? 2.0 : 4.0) * jb.c;
      // residual (without exchange) at (a, b): element (a, b) of the ordered pair (x, y)
      // is TF_(x<=y)[a][b], or TF_(y,x)[b][a] for x > y
      auto rl = [&](int a, int b) {
        double r = (e_vir[a] + e_vir[b]) * TF[(size_t)u * V2 + (size_t)a * nv + b];
        for (int k = 0; k < no; k++) {
          const int ok = jb.orbs[k];
          const double fik = t.f_occ[(size_t)i * n + ok], fkj = t.f_occ[(size_t)ok * n + j];
          const double* Tkj = TF + (size_t)uid[k * 3 + aj] * V2;
          const double* Tik = TF + (size_t)uid[ai * 3 + k] * V2;
          const double vkj = (k <= aj) ? Tkj[(size_t)a * nv + b] : Tkj[(size_t)b * nv + a];
          const double vik = (ai <= k) ? Tik[(size_t)a * nv + b] : Tik[(size_t)b * nv + a];
          r -= fik * vkj + fkj * vik;
        }
        return r;
      };
      for (size_t idx = threadIdx.x; idx < V2; idx += NT) {
        const int a = (int)(idx / nv), b = (int)(idx % nv);
        XL[idx] = scale * (2.0 * rl(a, b) - rl(b, a));
      }
      __syncthreads();
      const View P = pbasis(t, i, j);
      const View Tv = dense_view(Tp[u], m, m, m);
      cta_gemm(nv, m, m, 1.0, P, transpose(Tv), 0.0, Yt, m, sm);
      cta_gemm(nv, m, m, 1.0, P, Tv, 0.0, Y, m, sm);
      const View X = dense_view(XL, nv, nv, nv);
      cta_gemm(nv, m, nv, 1.0, X, dense_view(Yt, nv, m, m), 0.0, Dt, m, sm);
      cta_gemm(nv, m, nv, 1.0, transpose(X), dense_view(Y, nv, m, m), 1.0, Dt, m, sm);
      const int ni = t.n_osv[i], nj = (i == j) ? 0 : t.n_osv[j];
      for (size_t idx = threadIdx.x; idx < (size_t)nv * m; idx += NT) {
        const int r = (int)(idx / m), col = (int)(idx % m);
        if (col < ni) jb.slot[ai][(size_t)r * ni + col] += Dt[idx];
        else jb.slot[aj][(size_t)r * nj + col - ni] += Dt[idx];
      }
      __syncthreads();
    }
  }
}

// ---- G_x = sum of its terms (fragment slots, then exchange parts), in list order
__global__ void k_relax_gather(int n_vir, const int* __restrict__ n_osv, const RelaxGJob* __restrict__ jobs,
                               const RelaxGTerm* __restrict__ terms) {
  const RelaxGJob jb = jobs[blockIdx.y];
  const int nk = n_osv[jb.x];
  const size_t len = (size_t)n_vir * nk;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < len; idx += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / nk), k = (int)(idx % nk);
    double s = 0.0;
    for (int q = jb.t0; q < jb.t1; q++) s += terms[q].p[(size_t)r * terms[q].ld + terms[q].col0 + k];
    jb.G[idx] = s;
  }
}

// ---- eigenvector response, one CTA per orbital: W = Z / D (in place of Z), de_x, df_x
__global__ void __launch_bounds__(NT) k_relax_resp(Tables t, const double* __restrict__ e_vir,
                                                   const RelaxRJob* __restrict__ jobs) {
  __shared__ double sm[GEMM_SMEM_DOUBLES];
  const RelaxRJob jb = jobs[blockIdx.x];
  const int x = jb.x, nv = t.n_vir, nk = t.n_osv[x], nd = nv - nk;
  const size_t V2 = (size_t)nv * nv;
  if (nd > 0) {
    const View ZdT = dense_view(jb.V + (size_t)nk * nv, nd, nv, nv);   // rows: discarded eigenvectors
    cta_gemm(nd, nk, nv, 1.0, ZdT, dense_view(jb.G, nv, nk, nk), 0.0, jb.Y, nk, sm);
    for (int idx = threadIdx.x; idx < nd * nk; idx += NT) {
      const int l = idx / nk, k = idx % nk;
      jb.Y[idx] /= jb.w[k] - jb.w[nk + l];
    }
    __syncthreads();
    cta_gemm(nv, nk, nd, 1.0, transpose(ZdT), dense_view(jb.Y, nd, nk, nk), 0.0, jb.Xr, nk, sm);
    const View Qv = dense_view(t.Q[x], nv, nk, nk);
    const View Xv = dense_view(jb.Xr, nv, nk, nk);
    cta_gemm(nv, nv, nk, 0.5, Xv, transpose(Qv), 0.0, jb.Z, nv, sm);
    cta_gemm(nv, nv, nk, 0.5, Qv, transpose(Xv), 1.0, jb.Z, nv, sm);
  } else {
    for (size_t idx = threadIdx.x; idx < V2; idx += NT) jb.Z[idx] = 0.0;
    __syncthreads();
  }
  const double f2 = 2.0 * t.f_occ[(size_t)x * t.n_occ + x];
  for (int a = threadIdx.x; a < nv; a += NT) {
    double s = 0.0;
    for (int b = 0; b < nv; b++) {
      const double D = e_vir[a] + e_vir[b] - f2;
      const double z = jb.Z[(size_t)a * nv + b];
      s += z * jb.T[(size_t)a * nv + b] / D;
      jb.Z[(size_t)a * nv + b] = z / D;
    }
    jb.de[a] = -2.0 * s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int a = 0; a < nv; a++) s -= jb.de[a];
    *jb.df = s;
  }
}

// ---- dB_x += 2 W_x B_x, 64 x 64 output tiles
__global__ void __launch_bounds__(NT) k_relax_dB(Tables t, BSrc bs, const RelaxRJob* __restrict__ jobs, double* dB) {
  __shared__ double sm[GEMM_SMEM_DOUBLES];
  const RelaxRJob jb = jobs[blockIdx.x];
  const int nv = t.n_vir, nx = bs.n_aux;
  const int m0 = blockIdx.z * TM, n0 = blockIdx.y * TN;
  double acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; u++)
#pragma unroll
    for (int v = 0; v < 4; v++) acc[u][v] = 0.0;
  tile_mma(nv, nx, nv, m0, n0, dense_view(jb.Z, nv, nv, nv), BRows{bs, jb.x}, acc, sm);
  double* out = dB + (size_t)jb.x * nv * nx;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int u = 0; u < 4; u++)
#pragma unroll
    for (int v = 0; v < 4; v++) {
      const int r = m0 + ty + 16 * u, c = n0 + tx + 16 * v;
      if (r < nv && c < nx) out[(size_t)r * nx + c] += 2.0 * acc[u][v];
    }
}

// ---- dE/de += sum_x de_x (batch order), dE/df_xx += df_x
__global__ void k_relax_de_df(int n_vir, int n_occ, const RelaxRJob* __restrict__ jobs, int nb, double* de,
                              double* df) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < n_vir; a += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int u = 0; u < nb; u++) s += jobs[u].de[a];
    if (de) de[a] += s;
  }
  if (df && blockIdx.x == 0 && threadIdx.x == 0)
    for (int u = 0; u < nb; u++) df[(size_t)jobs[u].x * n_occ + jobs[u].x] += *jobs[u].df;
}

// ---------------------------------------------------------------- launchers
void launch_relax_kpart(const Tables& t, const BSrc& bs, const RelaxKJob* jobs, int n_jobs, double* scratch,
                        int n_cta, int max_m, cudaStream_t st) {
  if (!n_jobs) return;
  k_relax_kpart<<<n_cta, NT, 0, st>>>(t, bs, jobs, n_jobs, scratch, max_m);
  note_launch(1);
}
void launch_relax_frag(const Tables& t, const double* e_vir, const RelaxFragJob* jobs, int n_jobs, double* scratch,
                       size_t scr_per, int n_cta, int max_m, cudaStream_t st) {
  if (!n_jobs) return;
  k_relax_frag<<<n_cta, NT, 0, st>>>(t, e_vir, jobs, n_jobs, scratch, scr_per, max_m);
  note_launch(1);
}
void launch_relax_gather(int n_vir, const int* n_osv, const RelaxGJob* jobs, int n_jobs, const RelaxGTerm* terms,
                         cudaStream_t st) {
  if (!n_jobs) return;
  dim3 grid(16, n_jobs);
  k_relax_gather<<<grid, 256, 0, st>>>(n_vir, n_osv, jobs, terms);
  note_launch(1);
}
void launch_relax_resp(const Tables& t, const BSrc& bs, const double* e_vir, const RelaxRJob* jobs, int nb,
                       double* dB, double* de, double* df, cudaStream_t st) {
  if (!nb) return;
  k_relax_resp<<<nb, NT, 0, st>>>(t, e_vir, jobs);
  note_launch(1);
  if (dB) {
    dim3 grid(nb, (bs.n_aux + TN - 1) / TN, (t.n_vir + TM - 1) / TM);
    k_relax_dB<<<grid, NT, 0, st>>>(t, bs, jobs, dB);
    note_launch(1);
  }
  if (de || df) {
    k_relax_de_df<<<(t.n_vir + 255) / 256, 256, 0, st>>>(t.n_vir, t.n_occ, jobs, nb, de, df);
    note_launch(1);
  }
}

}  // namespace osv
