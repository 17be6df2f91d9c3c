// Mixed-form pair build in the orthonormal pair basis U_p = P_p X_p.
//
// X_p has entries up to ~1/sqrt(lambda_min(S_(ij,ij))), so a product formed in
// the raw OSV basis and then transformed (X^T K X, X^T S X) amplifies its
// rounding error by |X|^2.  The columns of U_p are orthonormal in the full
// virtual space (X^T S X = 1), so every low-precision product is formed with
// U_p directly:
//   U_p    = P_p X_p                           FP64 products, stored FP32 [n_vir][r]
//                                              and as four TF32 slices of U_p^T
//   G_p,x  = U_p^T B_x   (x = i, j)            split-precision tensor-core products
//                                              (gproj_tc.cu), stored FP32 [r][n_aux]
//   K~_p   = G_p,i G_p,j^T = X^T K_(ij,ij) X   FP32 products, stored FP64 [r][r]
// U_p must enter G with more than FP32 precision: its rounding error is the
// same for every aux function P, so it does not average out in the sum over P
// that forms K~, and it shifts every pair energy by ~eps_32 relative.  The
// rounding of G and of B, by contrast, is independent across P.
// The FP32 contractions sum each k-tile of sixteen products in FP32 and the
// tile sums in compensated FP32 (tile_mma_f32x64): long FP32 accumulations would leave
// errors of ~eps_32 sqrt(K) that add up over the thousands of pairs of an
// MBE(3) energy instead of averaging out.
// (Eqs. osv_imua and osv_close_k evaluated in the preconditioner basis of
// Eq. prec_eig.)
#include "pairview.cuh"
#include "tf32_split.cuh"

namespace osv {

// U_p = [Q_i Q_j] X_p in FP64 (per-CTA scratch [n_vir][max_r]), written as FP32
// [n_vir][r] and as the TF32 slices of U_p^T.  One CTA per pair (grid-stride).
__global__ void __launch_bounds__(NT) k_ubasis(Tables t, const UJob* __restrict__ jobs, int n_jobs,
                                               double* scratch, int max_r) {
  __shared__ double sm[GEMM_SMEM_DOUBLES];
  const int nv = t.n_vir;
  double* W = scratch + (size_t)blockIdx.x * nv * max_r;
  for (int jid = blockIdx.x; jid < n_jobs; jid += gridDim.x) {
    const UJob jb = jobs[jid];
    const int ni = t.n_osv[jb.i], nj = (jb.i == jb.j) ? 0 : t.n_osv[jb.j];
    const int m = ni + nj;
    const int pid = t.pair_id[jb.i * t.n_occ + jb.j];
    const int r = t.r[pid];
    View P;
    P.rows = nv; P.cols = m; P.rs = nv; P.cs = ni;
    P.b[0][0] = P.b[1][0] = Blk{t.Q[jb.i], ni, 0};
    P.b[0][1] = P.b[1][1] = Blk{nj ? t.Q[jb.j] : t.Q[jb.i], nj ? nj : ni, 0};
    cta_gemm(nv, r, m, 1.0, P, dense_view(t.X[pid], m, r, m), 0.0, W, r, sm);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nv * r; idx += NT) jb.U[idx] = (float)W[idx];
    const size_t sl = (size_t)r * jb.ldv;
    const int nch = (nv + tc::CHUNK - 1) / tc::CHUNK;
    const int lane = threadIdx.x & 31;
    for (int w = threadIdx.x >> 5; w < r * nch; w += NT / 32) {   // one (mu, chunk) per warp step
      const int mu = w / nch, a = (w - mu * nch) * tc::CHUNK + lane;
      float v[tc::NSL];
      tc::warp_fixed_slices(a < nv ? W[(size_t)a * r + mu] : 0.0, v);
      if (a < nv)
#pragma unroll
        for (int s = 0; s < tc::NSL; s++) jb.Us[s * sl + (size_t)mu * jb.ldv + a] = v[s];
    }
    __syncthreads();
  }
}

struct UtView {            // A(mu, a) = U[a][mu]
  const float* U;
  int r;
  __device__ __forceinline__ float get(int mu, int a) const { return U[(size_t)a * r + mu]; }
};
struct BView {             // B(a, P) = B[x, a, P]
  BSrc s;
  int x;
  __device__ __forceinline__ double get(int a, int P) const { return s.get(x, a, P); }
};

// G[mu][P] = sum_a U[a][mu] B[x,a,P].  grid: (job, P tile, mu tile)
__global__ void __launch_bounds__(NT) k_gproj(BSrc src, const GJob* __restrict__ jobs) {
  __shared__ float sm[GEMM_SMEM_DOUBLES];
  const GJob jb = jobs[blockIdx.x];
  const int m0 = blockIdx.z * TM, n0 = blockIdx.y * TN;
  if (m0 >= jb.r) return;
  double acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; u++)
#pragma unroll
    for (int v = 0; v < 4; v++) acc[u][v] = 0.0;
  tile_mma_f32x64(jb.r, src.n_aux, src.n_vir, m0, n0, UtView{jb.U, jb.r}, BView{src, jb.x}, acc, sm);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int u = 0; u < 4; u++)
#pragma unroll
    for (int v = 0; v < 4; v++) {
      const int rr = m0 + ty + 16 * u, c = n0 + tx + 16 * v;
      if (rr < jb.r && c < src.n_aux) jb.G[(size_t)rr * src.n_aux + c] = (float)acc[u][v];
    }
}

// K~ = G_i G_j^T (FP32 products, compensated accumulation over k-tiles of 16 aux
// functions: the aux sum is the final contraction of the energy and its FP32
// accumulation error would not average out).  grid: (job, tile r, tile c)
__global__ void __launch_bounds__(NT) k_ktilde_g(int n_aux, const KgJob* __restrict__ jobs) {
  __shared__ float sm[GEMM_SMEM_DOUBLES];
  const KgJob jb = jobs[blockIdx.x];
  const int m0 = blockIdx.y * TM, n0 = blockIdx.z * TN;
  if (m0 >= jb.r || n0 >= jb.r) return;
  double acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; u++)
#pragma unroll
    for (int v = 0; v < 4; v++) acc[u][v] = 0.0;
  tile_mma_f32x64(jb.r, jb.r, n_aux, m0, n0, ViewF{jb.Gi, n_aux, 0}, ViewF{jb.Gj, n_aux, 1}, acc, sm);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int u = 0; u < 4; u++)
#pragma unroll
    for (int v = 0; v < 4; v++) {
      const int rr = m0 + ty + 16 * u, c = n0 + tx + 16 * v;
      if (rr < jb.r && c < jb.r) jb.Kt[(size_t)rr * jb.r + c] = acc[u][v];
    }
}

void launch_ubasis(const Tables& t, const UJob* jobs, int n_jobs, int n_cta, double* scratch, int max_r,
                   cudaStream_t st) {
  if (!n_jobs) return;
  k_ubasis<<<n_cta, NT, 0, st>>>(t, jobs, n_jobs, scratch, max_r);
  note_launch(1);
}
void launch_gproj(const BSrc& src, const GJob* jobs, int n_jobs, int max_r, cudaStream_t st) {
  if (!n_jobs) return;
  dim3 grid(n_jobs, (src.n_aux + TN - 1) / TN, (max_r + TM - 1) / TM);
  k_gproj<<<grid, NT, 0, st>>>(src, jobs);
  note_launch(1);
}
void launch_ktilde_g(int n_aux, const KgJob* jobs, int n_jobs, int max_r, cudaStream_t st) {
  if (!n_jobs) return;
  const int nt = (max_r + TM - 1) / TM;
  dim3 grid(n_jobs, nt, nt);
  k_ktilde_g<<<grid, NT, 0, st>>>(n_aux, jobs);
  note_launch(1);
}

}  // namespace osv
