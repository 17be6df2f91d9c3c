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
// the rest runs per fragment in the OSV bases, from the stored S and F blocks.  Then, per orbital x,
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

// ---- the rest, one CTA per fragment, in the OSV bases: with T~ = 2T - T^T,
//   dP_u = c alpha [R_L P T~^T + R_L^T P T~]   (R_L: the residual without exchange)
//        = diag(e) P_u (T S_uu T~^T + T^T S_uu T~) + P_u (T F_uu T~^T + T^T F_uu T~)
//          + sum over (x, y) in {(k, j), (i, k)} of coef P_q (op(T_q) S_qu T~^T + op(T_q)^T S_qu T~)
// (coef = -f_ik, -f_kj; q the stored pair of (x, y), op the transpose when x > y,
// because T_(x,y)(full) = P_q op(T_q) P_q^T).  The small factors are summed per
// orbital block of the fragment (N: plain, Ne: scaled by e), then multiplied by Q_x.
// The Q_x columns of every pair's dP are summed (in pair order) into the fragment's
// slot of orbital x.
__global__ void __launch_bounds__(NT) k_relax_frag(Tables t, const double* __restrict__ e_vir,
                                                   const RelaxFragJob* __restrict__ jobs, int n_jobs,
                                                   double* scratch, size_t scr_per, int max_m) {
  __shared__ double sm[GEMM_SMEM_DOUBLES];
  const int nv = t.n_vir, n = t.n_occ;
  const size_t M2 = (size_t)max_m * max_m;
  double* Tt = scratch + (size_t)blockIdx.x * scr_per;   // T~ of the pair   [m][m]
  double* W1 = Tt + M2;                                   // op(T_q) S_qu     [m_q][m]
  double* N = W1 + M2;                                    // per-block factors [sum n_x][m]
  double* Ne = N + 3 * M2;
  double* Dt = Ne + 3 * M2;                               // dP               [nv][m]
  for (int jid = blockIdx.x; jid < n_jobs; jid += gridDim.x) {
    const RelaxFragJob jb = jobs[jid];
    const int no = jb.no;
    int pi[6], pj[6], pm[6], uid[9], off[3], nb[3];
    const double* Tp[6];
    int np = 0, rows = 0;
    size_t o = 0;
    for (int a = 0; a < no; a++) {
      nb[a] = t.n_osv[jb.orbs[a]];
      off[a] = rows;
      rows += nb[a];
    }
    for (int a = 0; a < no; a++)
      for (int b = a; b < no; b++) {
        pi[np] = jb.orbs[a];
        pj[np] = jb.orbs[b];
        pm[np] = pair_dim(t, pi[np], pj[np]);
        Tp[np] = jb.T + o;
        o += (size_t)pm[np] * pm[np];
        uid[a * 3 + b] = uid[b * 3 + a] = np;
        np++;
      }
    for (int a = 0; a < no; a++)
      for (size_t idx = threadIdx.x; idx < (size_t)nv * nb[a]; idx += NT) jb.slot[a][idx] = 0.0;
    int u = 0;
    for (int ua = 0; ua < no; ua++)
      for (int ub = ua; ub < no; ub++, u++) {
        const int i = pi[u], j = pj[u], m = pm[u];
        const double ac = ((i == j) ? 2.0 : 4.0) * jb.c;
        const double* T = Tp[u];
        for (int idx = threadIdx.x; idx < m * m; idx += NT) {
          const int r = idx / m, c = idx % m;
          Tt[idx] = 2.0 * T[idx] - T[(size_t)c * m + r];
        }
        for (size_t idx = threadIdx.x; idx < (size_t)rows * m; idx += NT) { N[idx] = 0.0; Ne[idx] = 0.0; }
        __syncthreads();
        const View Ttv = dense_view(Tt, m, m, m);
        // W1 (m_q x m) times T~^T and times T~ into the rows of the blocks (qa, qb) of Acc
        auto add_rows = [&](int mq, int qa, int qb, double coef, const View& Wop, const View& Tside, double* Acc) {
          const int n1 = nb[qa];
          cta_gemm(n1, m, m, coef, Wop, Tside, 1.0, Acc + (size_t)off[qa] * m, m, sm);
          if (qa != qb) {
            View w2 = Wop;   // rows [n1, mq) of a dense row-major view
            w2.b[0][0].p += (size_t)n1 * w2.b[0][0].ld;
            w2.b[0][1] = w2.b[1][0] = w2.b[1][1] = w2.b[0][0];
            w2.rows = w2.rs = mq - n1;
            cta_gemm(mq - n1, m, m, coef, w2, Tside, 1.0, Acc + (size_t)off[qb] * m, m, sm);
          }
        };
        // self terms: diag(e) P (T S T~^T + T^T S T~) and P (T F T~^T + T^T F T~)
        for (int s2 = 0; s2 < 2; s2++) {
          const View Mu = pair_view(t, s2 ? t.F : t.S, i, j, i, j);
          double* Acc = s2 ? N : Ne;
          for (int tr = 0; tr < 2; tr++) {
            cta_gemm(m, m, m, 1.0, dense_view(T, m, m, m, tr), Mu, 0.0, W1, m, sm);
            add_rows(m, ua, ub, ac, dense_view(W1, m, m, m), tr ? Ttv : transpose(Ttv), Acc);
          }
        }
        // couplings: -f_ik T_(k,j) and -f_kj T_(i,k) for every k of the fragment
        for (int kc = 0; kc < no; kc++) {
          const int k = jb.orbs[kc];
          for (int s2 = 0; s2 < 2; s2++) {
            const int x = s2 ? ua : kc, y = s2 ? kc : ub;
            const double coef = s2 ? -t.f_occ[(size_t)k * n + j] : -t.f_occ[(size_t)i * n + k];
            if (coef == 0.0) continue;
            const int qa = min(x, y), qb = max(x, y), trq = x > y;
            const int q = uid[qa * 3 + qb], mq = pm[q];
            const View Squ = pair_view(t, t.S, jb.orbs[qa], jb.orbs[qb], i, j);
            for (int tr = 0; tr < 2; tr++) {
              cta_gemm(mq, m, mq, 1.0, dense_view(Tp[q], mq, mq, mq, trq ^ tr), Squ, 0.0, W1, m, sm);
              add_rows(mq, qa, qb, ac * coef, dense_view(W1, mq, m, m), tr ? Ttv : transpose(Ttv), N);
            }
          }
        }
        // dP = diag(e) (Q_i Ne_i + Q_j Ne_j) + sum_x Q_x N_x
        cta_gemm(nv, m, nb[ua], 1.0, dense_view(t.Q[i], nv, nb[ua], nb[ua]),
                 dense_view(Ne + (size_t)off[ua] * m, nb[ua], m, m), 0.0, Dt, m, sm);
        if (ub != ua)
          cta_gemm(nv, m, nb[ub], 1.0, dense_view(t.Q[j], nv, nb[ub], nb[ub]),
                   dense_view(Ne + (size_t)off[ub] * m, nb[ub], m, m), 1.0, Dt, m, sm);
        for (size_t idx = threadIdx.x; idx < (size_t)nv * m; idx += NT) Dt[idx] *= e_vir[idx / m];
        __syncthreads();
        for (int a = 0; a < no; a++)
          cta_gemm(nv, m, nb[a], 1.0, dense_view(t.Q[jb.orbs[a]], nv, nb[a], nb[a]),
                   dense_view(N + (size_t)off[a] * m, nb[a], m, m), 1.0, Dt, m, sm);
        const int ni = t.n_osv[i], nj = (i == j) ? 0 : t.n_osv[j];
        for (size_t idx = threadIdx.x; idx < (size_t)nv * m; idx += NT) {
          const int r = (int)(idx / m), col = (int)(idx % m);
          if (col < ni) jb.slot[ua][(size_t)r * ni + col] += Dt[idx];
          else jb.slot[ub][(size_t)r * nj + col - ni] += Dt[idx];
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
