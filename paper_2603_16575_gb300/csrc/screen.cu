// Pair screening and weak pairs (FP64; in the mixed form the weak-pair K_(i,j) and
// the diagonal projections are double-float products):
//   s2b_ij = sum_{mu nu} (Q_i^T Q_j)_{mu nu}^2 / sqrt(n_i n_j)           (Eq. s2b)
//   T_(ii,ii) = sum over kept clusters C containing i of c_C T^C_(ii,ii)   (Eq. tmbediag)
//   weak pairs: K_(i,j) = B~_i^(i)T B~_j^(j) (Eq. osv_weak_k) and the single-block
//   residual K + F_(i,i) T + T F_(j,j) - (f_ii + f_jj) T - f_ij [T_(i,i) S_(i,j) + S_(i,j) T_(j,j)]
//   (Eq. res_weak as the projected pair equation), solved in one update in the
//   eigenbases X_i of F_(i,i) (Algorithm 7, weak pairs), energy 2 <K, T> per
//   ordered pair, both orders counted.
#include "internal.h"

namespace osv {

// S = Q_i^T Q_j tile by tile (16R x 16R outputs), summing the squares of the
// finished tile entries; one CTA per pair.
template <int R>
__device__ double s2b_tiles(int ni, int nj, int nv, const double* __restrict__ qi, const double* __restrict__ qj,
                            double* sm) {
  constexpr int T = 16 * R;
  double* As = sm;
  double* Bs = sm + TK * T;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double sq = 0.0;
  for (int m0 = 0; m0 < ni; m0 += T)
    for (int n0 = 0; n0 < nj; n0 += T) {
      double acc[R][R];
#pragma unroll
      for (int u = 0; u < R; u++)
#pragma unroll
        for (int v = 0; v < R; v++) acc[u][v] = 0.0;
      for (int k0 = 0; k0 < nv; k0 += TK) {
        for (int e = tid; e < TK * T; e += NT) {
          const int k = e / T, m = e % T, gk = k0 + k;
          As[e] = (gk < nv && m0 + m < ni) ? qi[(size_t)gk * ni + m0 + m] : 0.0;
          Bs[e] = (gk < nv && n0 + m < nj) ? qj[(size_t)gk * nj + n0 + m] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < TK; k++) {
          double a[R], b[R];
#pragma unroll
          for (int u = 0; u < R; u++) a[u] = As[k * T + ty + 16 * u];
#pragma unroll
          for (int v = 0; v < R; v++) b[v] = Bs[k * T + tx + 16 * v];
#pragma unroll
          for (int u = 0; u < R; u++)
#pragma unroll
            for (int v = 0; v < R; v++) acc[u][v] = fma(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
      }
#pragma unroll
      for (int u = 0; u < R; u++)
#pragma unroll
        for (int v = 0; v < R; v++) sq = fma(acc[u][v], acc[u][v], sq);   // padding entries are exact zeros
    }
  return sq;
}

__global__ void __launch_bounds__(NT) k_s2b(Tables t, const int2* __restrict__ pairs, int n_pairs, double* s2b) {
  __shared__ double sm[2 * TK * 80];
  __shared__ double red[33];
  for (int p = blockIdx.x; p < n_pairs; p += gridDim.x) {
    const int i = pairs[p].x, j = pairs[p].y;
    const int ni = t.n_osv[i], nj = t.n_osv[j], nv = t.n_vir;
    const int w = max(ni, nj);
    double sq;
    if (w <= 48) sq = s2b_tiles<3>(ni, nj, nv, t.Q[i], t.Q[j], sm);
    else if (w <= 64) sq = s2b_tiles<4>(ni, nj, nv, t.Q[i], t.Q[j], sm);
    else sq = s2b_tiles<5>(ni, nj, nv, t.Q[i], t.Q[j], sm);
    sq = cta_sum(sq, red);
    if (threadIdx.x == 0) s2b[p] = sq / sqrt((double)ni * (double)nj);
  }
}

void launch_s2b(const Tables& t, const int2* pairs, int n_pairs, double* s2b, int n_cta, cudaStream_t st) {
  if (n_pairs == 0) return;
  k_s2b<<<n_cta, NT, 0, st>>>(t, pairs, n_pairs, s2b);
  note_launch(1);
}

// T_ii (n x n, raw OSV basis) = sum_c w_c A_c with A_c the (ii) amplitude of a
// cluster solve; the mixed form stores Y (r x r, T = X Y X^T in the pair's
// preconditioner basis), transformed here after the weighted sum.
__global__ void __launch_bounds__(NT) k_diag_amp(Tables t, const DiagJob* __restrict__ jobs, int n_jobs,
                                                 const GradContrib* __restrict__ contrib, int mixed,
                                                 double* scratch, int max_n) {
  __shared__ double sm[GEMM_SMEM_DOUBLES];
  double* Ys = scratch + (size_t)blockIdx.x * 2 * max_n * max_n;
  double* W = Ys + (size_t)max_n * max_n;
  for (int q = blockIdx.x; q < n_jobs; q += gridDim.x) {
    const DiagJob jb = jobs[q];
    const int n = t.n_osv[jb.i];
    const int r = mixed ? t.r[jb.pid] : n;
    double* acc = mixed ? Ys : jb.T;
    for (int idx = threadIdx.x; idx < r * r; idx += NT) {
      double s = 0.0;
      for (int c = jb.c0; c < jb.c1; c++) s = fma((double)contrib[c].weight, contrib[c].T[idx], s);
      acc[idx] = s;
    }
    __syncthreads();
    if (mixed) {   // T = X_r Y X_r^T, X [n][n] row-major with r valid columns
      const View X = dense_view(t.X[jb.pid], n, r, n);
      cta_gemm(n, r, r, 1.0, X, dense_view(Ys, r, r, r), 0.0, W, r, sm);
      cta_gemm(n, n, r, 1.0, dense_view(W, n, r, r), transpose(X), 0.0, jb.T, n, sm);
    }
    __syncthreads();
  }
}

void launch_diag_amp(const Tables& t, const DiagJob* jobs, int n_jobs, const GradContrib* contrib, int mixed,
                     double* scratch, int max_n, int n_cta, cudaStream_t st) {
  if (n_jobs == 0) return;
  k_diag_amp<<<n_cta, NT, 0, st>>>(t, jobs, n_jobs, contrib, mixed, scratch, max_n);
  note_launch(1);
}

// One weak pair per CTA iteration (grid-stride); scratch: 6 max_n^2 doubles per CTA.
// FP64 form: X_i, X_j are exact eigenbases of F_(i,i), F_(j,j) and one update from
// T = 0 solves the single-block equation.  Mixed form: K_(i,j) in double-float, and
// X_i, X_j are the mixed preconditioner bases of the diagonal pairs (X^T X = 1 + O(1e-7));
// the update is repeated on the raw-basis residual
// R = K + F_(i,i) T + T F_(j,j) - (f_ii + f_jj) T - f_ij [T_(i,i) S + S T_(j,j)]
// (three times), which converges to the same fixed point.
constexpr int WEAK_MIXED_SWEEPS = 3;

struct AuxRows {          // A(P, a) = B[i, a, P0 + P]
  BSrc s;
  int i, P0;
  __device__ __forceinline__ double get(int P, int a) const { return s.get(i, a, P0 + P); }
};

__global__ void __launch_bounds__(NT) k_weak(Tables t, int n_aux, const WeakJob* __restrict__ jobs, int n_jobs,
                                             double* scratch, int max_n, double* e_out, int mixed) {
  __shared__ double sm[GEMM_SMEM_WIDE];
  __shared__ double red[33];
  const size_t M2 = (size_t)max_n * max_n;
  double* K = scratch + (size_t)blockIdx.x * 6 * M2;
  double* C = K + M2;
  double* W = C + M2;
  double* Rt = W + M2;
  double* T = Rt + M2;
  double* R = T + M2;
  for (int q = blockIdx.x; q < n_jobs; q += gridDim.x) {
    const WeakJob jb = jobs[q];
    const int ni = t.n_osv[jb.i], nj = t.n_osv[jb.j];
    const double fii = t.f_occ[(size_t)jb.i * t.n_occ + jb.i], fjj = t.f_occ[(size_t)jb.j * t.n_occ + jb.j];
    const double fij = t.f_occ[(size_t)jb.i * t.n_occ + jb.j];
    const View S = dense_view(jb.S, ni, nj, nj);
    const View Xi = dense_view(jb.Xi, ni, ni, jb.ldxi), Xj = dense_view(jb.Xj, nj, nj, jb.ldxj);
    const View Bi = transpose(dense_view(jb.Bii, n_aux, ni, ni)), Bj = dense_view(jb.Bjj, n_aux, nj, nj);
    // K_(i,j) = B~_i^(i)T B~_j^(j): the projections are [n_aux][n] row-major
    if (mixed) cta_gemm_df(ni, nj, n_aux, 1.0, Bi, Bj, 0.0, K, nj, sm);
    else cta_gemm(ni, nj, n_aux, 1.0, Bi, Bj, 0.0, K, nj, sm);
    // A = K - f_ij (T_ii S + S T_jj)
    cta_gemm(ni, nj, ni, 1.0, dense_view(jb.Ti, ni, ni, ni), S, 0.0, C, nj, sm);
    cta_gemm(ni, nj, nj, 1.0, S, dense_view(jb.Tj, nj, nj, nj), 1.0, C, nj, sm);
    for (int idx = threadIdx.x; idx < ni * nj; idx += NT) C[idx] = K[idx] - fij * C[idx];
    __syncthreads();
    double e = 0.0;
    if (!mixed) {
      // R~ = X_i^T A X_j and K~ = X_i^T K X_j; Y~ = R~ / (f_ii + f_jj - e_i - e_j); E = 4 <K~, Y~>
      cta_gemm(ni, nj, ni, 1.0, transpose(Xi), dense_view(C, ni, nj, nj), 0.0, W, nj, sm);
      cta_gemm(ni, nj, nj, 1.0, dense_view(W, ni, nj, nj), Xj, 0.0, Rt, nj, sm);
      cta_gemm(ni, nj, ni, 1.0, transpose(Xi), dense_view(K, ni, nj, nj), 0.0, W, nj, sm);
      cta_gemm(ni, nj, nj, 1.0, dense_view(W, ni, nj, nj), Xj, 0.0, T, nj, sm);
      for (int idx = threadIdx.x; idx < ni * nj; idx += NT) {
        const int mu = idx / nj, nu = idx % nj;
        e = fma(T[idx], Rt[idx] / (fii + fjj - jb.ei[mu] - jb.ej[nu]), e);
      }
    } else {
      for (int idx = threadIdx.x; idx < ni * nj; idx += NT) {
        T[idx] = 0.0;
        R[idx] = C[idx];
      }
      __syncthreads();
      for (int sw = 0; sw < WEAK_MIXED_SWEEPS; sw++) {
        cta_gemm(ni, nj, ni, 1.0, transpose(Xi), dense_view(R, ni, nj, nj), 0.0, W, nj, sm);
        cta_gemm(ni, nj, nj, 1.0, dense_view(W, ni, nj, nj), Xj, 0.0, Rt, nj, sm);
        for (int idx = threadIdx.x; idx < ni * nj; idx += NT) {
          const int mu = idx / nj, nu = idx % nj;
          Rt[idx] /= (fii + fjj - jb.ei[mu] - jb.ej[nu]);
        }
        __syncthreads();
        cta_gemm(ni, nj, ni, 1.0, Xi, dense_view(Rt, ni, nj, nj), 0.0, W, nj, sm);
        cta_gemm(ni, nj, nj, 1.0, dense_view(W, ni, nj, nj), transpose(Xj), 1.0, T, nj, sm);
        if (sw + 1 < WEAK_MIXED_SWEEPS) {   // R = A + F_ii T + T F_jj - (f_ii + f_jj) T
          for (int idx = threadIdx.x; idx < ni * nj; idx += NT) R[idx] = C[idx] - (fii + fjj) * T[idx];
          __syncthreads();
          cta_gemm(ni, nj, ni, 1.0, dense_view(jb.Fi, ni, ni, ni), dense_view(T, ni, nj, nj), 1.0, R, nj, sm);
          cta_gemm(ni, nj, nj, 1.0, dense_view(T, ni, nj, nj), dense_view(jb.Fj, nj, nj, nj), 1.0, R, nj, sm);
        }
      }
      for (int idx = threadIdx.x; idx < ni * nj; idx += NT) e = fma(K[idx], T[idx], e);
    }
    e = cta_sum(e, red);
    if (threadIdx.x == 0) e_out[q] = 4.0 * e;
    __syncthreads();
  }
}

void launch_weak(const Tables& t, int n_aux, const WeakJob* jobs, int n_jobs, double* scratch, int max_n, int n_cta,
                 double* e_out, int mixed, cudaStream_t st) {
  if (n_jobs == 0) return;
  k_weak<<<n_cta, NT, 0, st>>>(t, n_aux, jobs, n_jobs, scratch, max_n, e_out, mixed);
  note_launch(1);
}

// Mixed form: B~_i^(i) = B_i^T Q_i ([n_aux][n_i]) in double-float, one CTA per
// (orbital, tile of WPROJ_ROWS aux rows).
constexpr int WPROJ_ROWS = 96;
__global__ void __launch_bounds__(NT) k_project_df(BSrc src, Tables t, const ProjJob* __restrict__ jobs) {
  __shared__ double sm[GEMM_SMEM_WIDE];
  const ProjJob jb = jobs[blockIdx.x];
  const int nx = t.n_osv[jb.x];
  const int P0 = blockIdx.y * WPROJ_ROWS;
  const int M = min(WPROJ_ROWS, src.n_aux - P0);
  if (M <= 0) return;
  cta_gemm_df(M, nx, src.n_vir, 1.0, AuxRows{src, jb.i, P0}, dense_view(t.Q[jb.x], src.n_vir, nx, nx), 0.0,
              jb.out + (size_t)P0 * nx, nx, sm);
}

void launch_project_df(const BSrc& src, const Tables& t, const ProjJob* jobs, int n_jobs, cudaStream_t st) {
  if (n_jobs == 0) return;
  dim3 grid(n_jobs, (src.n_aux + WPROJ_ROWS - 1) / WPROJ_ROWS);
  k_project_df<<<grid, NT, 0, st>>>(src, t, jobs);
  note_launch(1);
}

}  // namespace osv
