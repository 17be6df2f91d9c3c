// A3 with one warp per pair: the preconditioner F X = S X E~ (Eq. prec_eig) by
// canonical orthogonalisation of S and the eigen-decomposition of Y^T F Y,
// exactly as k_precond, but with many pairs in flight per SM so that the
// sequential parts (the Householder steps, the QR bulge chase) of different
// pairs overlap.  Matrices live in per-warp global scratch (L2-resident);
// vectors, the tridiagonal and the rotations in per-warp shared memory.
#include "eig.cuh"
#include "pairview.cuh"
#include "warp_eig.cuh"

namespace osv {

constexpr int PW_WARPS = 4;          // warps per CTA (static shared memory stays below 48 KB)

__global__ void __launch_bounds__(PW_WARPS * 32) k_precond_w(Tables t, double tau_s, const PJob* __restrict__ jobs,
                                                             int n_jobs, int max_m, double* scratch, int* err) {
  __shared__ WarpSm wsm[PW_WARPS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = blockIdx.x * PW_WARPS + warp, nw = gridDim.x * PW_WARPS;
  WarpSm& ws = wsm[warp];
  const size_t M2 = (size_t)max_m * max_m;
  double* base = scratch + (size_t)gw * (6 * M2 + 4 * (size_t)max_m);
  double* Sw = base;
  double* Fw = Sw + M2;
  double* Z = Fw + M2;
  double* Yw = Z + M2;
  double* W1 = Yw + M2;
  double* Fp = W1 + M2;
  double* tau = Fp + M2;
  double* wsv = tau + max_m;
  double* w2 = wsv + max_m;
  for (int jid = gw; jid < n_jobs; jid += nw) {
    const PJob jb = jobs[jid];
    const int m = pair_dim(t, jb.i, jb.j);
    const View Sv = pair_view(t, t.S, jb.i, jb.j, jb.i, jb.j);
    const View Fv = pair_view(t, t.F, jb.i, jb.j, jb.i, jb.j);
    for (int r = 0; r < m; r++)
      for (int c = lane; c < m; c += 32) {
        Sw[(size_t)r * m + c] = Sv.get(r, c);
        Fw[(size_t)r * m + c] = Fv.get(r, c);
      }
    __syncwarp();
    int rc = warp_syev(Sw, m, wsv, Z, tau, ws);
    int r = 0;
    if (lane == 0) {
      double smax = 0.0;
      for (int c = 0; c < m; c++) smax = fmax(smax, wsv[c]);
      for (int c = 0; c < m; c++)
        if (wsv[c] > tau_s * smax) ws.keep[r++] = c;
      if (rc) atomicOr(err, ERR_EIG);
    }
    r = __shfl_sync(0xffffffffu, r, 0);
    __syncwarp();
    for (int row = 0; row < m; row++)
      for (int c = lane; c < r; c += 32) {
        const int kc = ws.keep[c];
        Yw[(size_t)row * m + c] = Z[(size_t)row * m + kc] / sqrt(wsv[kc]);
      }
    __syncwarp();
    const View Yv = dense_view(Yw, m, r, m);
    warp_gemm(m, r, m, 1.0, dense_view(Fw, m, m, m), Yv, 0.0, W1, m);
    warp_gemm(r, r, m, 1.0, transpose(Yv), dense_view(W1, m, r, m), 0.0, Fp, r);
    rc = warp_syev(Fp, r, w2, Z, tau, ws);
    if (lane == 0 && rc) atomicOr(err, ERR_EIG);
    warp_gemm(m, r, r, 1.0, Yv, dense_view(Z, r, r, r), 0.0, jb.X, m);
    for (int c = lane; c < r; c += 32) {
      jb.et[c] = w2[c];
      if (!isfinite(w2[c])) atomicOr(err, ERR_NONFINITE);
    }
    if (lane == 0) *jb.r = r;
    __syncwarp();
  }
}

size_t precond_w_scratch_doubles(int max_m, int n_warps) {
  return (size_t)n_warps * (6 * (size_t)max_m * max_m + 4 * (size_t)max_m);
}

int launch_precond_w(const Tables& t, double tau_s, const PJob* jobs, int n_jobs, int max_m, double* scratch,
                     int n_warps, int* err, cudaStream_t st) {
  if (!n_jobs) return 0;
  if (max_m > PW_MAXN) return -1;
  const int n_cta = (n_warps + PW_WARPS - 1) / PW_WARPS;
  k_precond_w<<<n_cta, PW_WARPS * 32, 0, st>>>(t, tau_s, jobs, n_jobs, max_m, scratch, err);
  note_launch(1);
  return 0;
}

}  // namespace osv
