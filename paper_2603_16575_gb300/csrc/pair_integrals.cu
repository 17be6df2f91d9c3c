// A1-A2 in FP64: OSV projection of the RI integrals (Eq. osv_imua),
// exchange blocks K_(ij,ij) (Eq. osv_close_k, columns from LMO j) and the OSV
// overlap / Fock blocks of Algorithm 5 (Eq. 4block_osv with A = S, F).
#include "internal.h"

namespace osv {

struct ProjA {            // A(P, a) = B[i,a,P]
  BSrc s;
  int i;
  __device__ __forceinline__ double get(int P, int a) const { return s.get(i, a, P); }
};
struct RowMajor {         // B(r, c) = p[r*ld + c]
  const double* p;
  int ld;
  __device__ __forceinline__ double get(int r, int c) const { return p[(size_t)r * ld + c]; }
};

// grid: (job, P tile, mu tile).  V = double (FP64 form) or float (mixed form:
// FP32 products and accumulation, result stored as FP64).
template <class V>
__global__ void __launch_bounds__(NT) k_project(BSrc src, Tables t, const ProjJob* __restrict__ jobs) {
  __shared__ V sm[GEMM_SMEM_DOUBLES];
  const ProjJob jb = jobs[blockIdx.x];
  const int nx = t.n_osv[jb.x];
  const int m0 = blockIdx.y * TM, n0 = blockIdx.z * TN;
  if (n0 >= nx) return;
  const int M = src.n_aux, N = nx, K = src.n_vir;
  V acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; u++)
#pragma unroll
    for (int v = 0; v < 4; v++) acc[u][v] = V(0);
  tile_mma_t<V>(M, N, K, m0, n0, ProjA{src, jb.i}, RowMajor{t.Q[jb.x], nx}, acc, sm);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int u = 0; u < 4; u++)
#pragma unroll
    for (int v = 0; v < 4; v++) {
      const int r = m0 + ty + 16 * u, c = n0 + tx + 16 * v;
      if (r < M && c < N) jb.out[(size_t)r * N + c] = (double)acc[u][v];
    }
}

void launch_project(const BSrc& src, const Tables& t, const ProjJob* jobs, int n_jobs, int max_nx, int fp32,
                    cudaStream_t st) {
  if (n_jobs == 0) return;
  dim3 grid(n_jobs, (src.n_aux + TM - 1) / TM, (max_nx + TN - 1) / TN);
  if (fp32) k_project<float><<<grid, NT, 0, st>>>(src, t, jobs);
  else k_project<double><<<grid, NT, 0, st>>>(src, t, jobs);
  note_launch(1);
}

// K_(ij,ij)[mu][nu] = sum_P L[P][mu] R[P][nu] with L = [B~_i^(i) B~_i^(j)],
// R = [B~_j^(i) B~_j^(j)] (aux x OSV, row-major).  grid: (job, tile r, tile c)
template <class V>
__global__ void __launch_bounds__(NT) k_exchange(Tables t, int n_aux, const KJob* __restrict__ jobs) {
  __shared__ V sm[GEMM_SMEM_DOUBLES];
  const KJob jb = jobs[blockIdx.x];
  const int ni = t.n_osv[jb.i];
  const int nj = (jb.i == jb.j) ? 0 : t.n_osv[jb.j];
  const int m = ni + nj;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.z * TN;
  if (m0 >= m || n0 >= m) return;
  View A, B;
  A.rows = m; A.cols = n_aux; A.rs = ni; A.cs = n_aux;
  A.b[0][0] = A.b[0][1] = Blk{jb.Bii, ni, 1};
  A.b[1][0] = A.b[1][1] = Blk{jb.Bij ? jb.Bij : jb.Bii, nj > 0 ? nj : ni, 1};
  B.rows = n_aux; B.cols = m; B.rs = n_aux; B.cs = ni;
  if (nj == 0) {
    B.b[0][0] = B.b[0][1] = B.b[1][0] = B.b[1][1] = Blk{jb.Bii, ni, 0};
  } else {
    B.b[0][0] = B.b[1][0] = Blk{jb.Bji, ni, 0};
    B.b[0][1] = B.b[1][1] = Blk{jb.Bjj, nj, 0};
  }
  V acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; u++)
#pragma unroll
    for (int v = 0; v < 4; v++) acc[u][v] = V(0);
  tile_mma_t<V>(m, m, n_aux, m0, n0, A, B, acc, sm);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int u = 0; u < 4; u++)
#pragma unroll
    for (int v = 0; v < 4; v++) {
      const int r = m0 + ty + 16 * u, c = n0 + tx + 16 * v;
      if (r < m && c < m) jb.out[(size_t)r * m + c] = (double)acc[u][v];
    }
}

void launch_exchange(const Tables& t, int n_aux, const KJob* jobs, int n_jobs, int max_m, int fp32, cudaStream_t st) {
  if (n_jobs == 0) return;
  const int nt = (max_m + TM - 1) / TM;
  dim3 grid(n_jobs, nt, nt);
  if (fp32) k_exchange<float><<<grid, NT, 0, st>>>(t, n_aux, jobs);
  else k_exchange<double><<<grid, NT, 0, st>>>(t, n_aux, jobs);
  note_launch(1);
}


// S_(x,y) = Q_x^T Q_y and F_(x,y) = Q_x^T diag(e) Q_y, both from the same
// staged tiles of Q_x and Q_y, one CTA per block.  The output tile is the
// smallest of 48, 64 and 80 wide that covers the block (OSV blocks are ~10-80
// wide; a fixed 64-wide tile would mostly compute padding), 80-wide tiles in a
// loop above that.  Every output's FMAs run in k order with the product
// e_a Q_x[a][mu] rounded first, as in a plain GEMM of the scaled operand.
constexpr int SF_TMAX = 80;
template <int R>
__device__ void sf_tiles(int nx, int ny, int nv, const double* __restrict__ qx, const double* __restrict__ qy,
                         const double* __restrict__ e_vir, double* S, double* F, double* sm) {
  constexpr int T = 16 * R;
  double* As = sm;                 // [TK][T]
  double* Bs = sm + TK * T;        // [TK][T]
  double* es = sm + 2 * TK * T;    // [TK]
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int m0 = 0; m0 < nx; m0 += T)
    for (int n0 = 0; n0 < ny; n0 += T) {
      double aS[R][R], aF[R][R];
#pragma unroll
      for (int u = 0; u < R; u++)
#pragma unroll
        for (int v = 0; v < R; v++) aS[u][v] = aF[u][v] = 0.0;
      for (int k0 = 0; k0 < nv; k0 += TK) {
        for (int e = tid; e < TK * T; e += NT) {
          const int k = e / T, m = e % T, gk = k0 + k;
          As[e] = (gk < nv && m0 + m < nx) ? qx[(size_t)gk * nx + m0 + m] : 0.0;
          Bs[e] = (gk < nv && n0 + m < ny) ? qy[(size_t)gk * ny + n0 + m] : 0.0;
        }
        if (tid < TK) es[tid] = (k0 + tid < nv) ? e_vir[k0 + tid] : 0.0;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < TK; k++) {
          double a[R], ea[R], b[R];
          const double ek = es[k];
#pragma unroll
          for (int u = 0; u < R; u++) {
            a[u] = As[k * T + ty + 16 * u];
            ea[u] = a[u] * ek;
          }
#pragma unroll
          for (int v = 0; v < R; v++) b[v] = Bs[k * T + tx + 16 * v];
#pragma unroll
          for (int u = 0; u < R; u++)
#pragma unroll
            for (int v = 0; v < R; v++) {
              aS[u][v] = fma(a[u], b[v], aS[u][v]);
              aF[u][v] = fma(ea[u], b[v], aF[u][v]);
            }
        }
        __syncthreads();
      }
#pragma unroll
      for (int u = 0; u < R; u++)
#pragma unroll
        for (int v = 0; v < R; v++) {
          const int r = m0 + ty + 16 * u, c = n0 + tx + 16 * v;
          if (r < nx && c < ny) {
            S[(size_t)r * ny + c] = aS[u][v];
            F[(size_t)r * ny + c] = aF[u][v];
          }
        }
    }
}

__global__ void __launch_bounds__(NT, 2) k_sf(Tables t, const double* __restrict__ e_vir,
                                           const SFJob* __restrict__ jobs) {
  __shared__ double sm[2 * TK * SF_TMAX + TK];
  const SFJob jb = jobs[blockIdx.x];
  const int nx = t.n_osv[jb.x], ny = t.n_osv[jb.y], nv = t.n_vir;
  const int w = max(nx, ny);
  if (w <= 48) sf_tiles<3>(nx, ny, nv, t.Q[jb.x], t.Q[jb.y], e_vir, jb.S, jb.F, sm);
  else if (w <= 64) sf_tiles<4>(nx, ny, nv, t.Q[jb.x], t.Q[jb.y], e_vir, jb.S, jb.F, sm);
  else sf_tiles<5>(nx, ny, nv, t.Q[jb.x], t.Q[jb.y], e_vir, jb.S, jb.F, sm);
}

void launch_sf(const Tables& t, const double* e_vir, const SFJob* jobs, int n_jobs, int max_n, cudaStream_t st) {
  if (n_jobs == 0) return;
  (void)max_n;
  k_sf<<<n_jobs, NT, 0, st>>>(t, e_vir, jobs);
  note_launch(1);
}

}  // namespace osv
