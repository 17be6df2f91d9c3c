// Mixed-form pair build in the orthonormal pair basis U_p = P_p X_p.
//
// X_p has entries up to ~1/sqrt(lambda_min(S_(ij,ij))), so a product formed in
// the raw OSV basis and then transformed (X^T K X, X^T S X) amplifies its
// rounding error by |X|^2.  The columns of U_p are orthonormal in the full
// virtual space (X^T S X = 1), so every low-precision product is formed with
// U_p directly:
//   U_p    = P_p X_p                           double-float products, stored FP32 [n_vir][r]
//                                              and as four TF32 slices of U_p^T
//   G_p,x  = U_p^T B_x   (x = i, j)            split-precision tensor-core products
//                                              (gproj_tc.cu), stored FP32 [r][n_aux]
//                                              and as the slices of G_p,x^T
//   K~_p   = G_p,i G_p,j^T = X^T K_(ij,ij) X   split-precision tensor-core products
//                                              of those slices, stored FP64 [r][r]
// U_p must enter G with more than FP32 precision: its rounding error is the
// same for every aux function P, so it does not average out in the sum over P
// that forms K~, and it shifts every pair energy by ~eps_32 relative.  For the
// same reason K~ is not formed from FP32 products of the rounded G.
// (Eqs. osv_imua and osv_close_k evaluated in the preconditioner basis of
// Eq. prec_eig.)
#include "pairview.cuh"
#include "tf32_split.cuh"

namespace osv {

// U_p = [Q_i Q_j] X_p in double-float arithmetic (~48 bits, above the ~36 bits
// its slices carry), formed transposed (U_p^T [r][n_vir] in the
// per-CTA scratch, so that the slices of U_p^T are cut from contiguous rows),
// written as FP32 [n_vir][r] through a shared-memory transpose and as the TF32
// slices of U_p^T.  One CTA per pair (grid-stride).
__global__ void __launch_bounds__(NT) k_ubasis(Tables t, const UJob* __restrict__ jobs, int n_jobs,
                                               double* scratch, int max_r) {
  __shared__ double sm[GEMM_SMEM_WIDE];   // GEMM tiles, then the transpose tiles
  constexpr int TW = (GEMM_SMEM_WIDE * 2) / (32 * 33);   // warps with a 32 x 33 float tile
  float (*tr)[32][33] = reinterpret_cast<float (*)[32][33]>(sm);
  const int nv = t.n_vir;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* Wt = scratch + (size_t)blockIdx.x * nv * max_r;
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
    cta_gemm_df(r, nv, m, 1.0, transpose(dense_view(t.X[pid], m, r, m)), transpose(P), 0.0, Wt, nv, sm);
    const size_t sl = (size_t)r * jb.ldv;
    const int nch = (nv + tc::CHUNK - 1) / tc::CHUNK;
    // slices of U^T: one (mu, 32-virtual chunk) per warp step, lanes along the virtuals
    for (int w = warp; w < r * nch; w += NT / 32) {
      const int mu = w / nch, a = (w - mu * nch) * tc::CHUNK + lane;
      float v[tc::NSL];
      tc::warp_fixed_slices(a < nv ? Wt[(size_t)mu * nv + a] : 0.0, v);
      if (a < nv)
#pragma unroll
        for (int s = 0; s < tc::NSL; s++) jb.Us[s * sl + (size_t)mu * jb.ldv + a] = v[s];
    }
    // U [a][mu] = U^T [mu][a], 32 x 32 tiles through shared memory (warps 0 .. TW-1)
    const int nta = (nv + 31) / 32, ntm = (r + 31) / 32;
    for (int tl = warp; warp < TW && tl < nta * ntm; tl += TW) {
      const int a0 = (tl % nta) * 32, m0 = (tl / nta) * 32;
      for (int q = 0; q < 32; q++) {
        const int mu = m0 + q, a = a0 + lane;
        tr[warp][q][lane] = (mu < r && a < nv) ? (float)Wt[(size_t)mu * nv + a] : 0.f;
      }
      __syncwarp();
      for (int q = 0; q < 32; q++) {
        const int a = a0 + q, mu = m0 + lane;
        if (a < nv && mu < r) jb.U[(size_t)a * r + mu] = tr[warp][lane][q];
      }
      __syncwarp();
    }
    __syncthreads();
  }
}

void launch_ubasis(const Tables& t, const UJob* jobs, int n_jobs, int n_cta, double* scratch, int max_r,
                   cudaStream_t st) {
  if (!n_jobs) return;
  k_ubasis<<<n_cta, NT, 0, st>>>(t, jobs, n_jobs, scratch, max_r);
  note_launch(1);
}
}  // namespace osv
