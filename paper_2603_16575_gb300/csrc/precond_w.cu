// A3 with one warp per pair: the preconditioner F X = S X E~ (Eq. prec_eig) by
// canonical orthogonalisation of S and the eigen-decomposition of Y^T F Y,
// exactly as k_precond, but with many pairs in flight per SM so that the
// sequential parts (the Householder steps, the QR bulge chase) of different
// pairs overlap.  Matrices live in per-warp global scratch (L2-resident);
// vectors, the tridiagonal and the rotations in per-warp shared memory.
#include "eig.cuh"
#include "pairview.cuh"

namespace osv {

constexpr int PW_WARPS = 4;          // warps per CTA (static shared memory stays below 48 KB)
constexpr int PW_MAXN = 192;         // largest pair order handled by the warp path

struct WarpSm {                      // per-warp shared scratch
  double v[PW_MAXN];
  double p[PW_MAXN];
  double d[PW_MAXN];
  double e[PW_MAXN];
  double cs[2 * PW_MAXN];
  int keep[PW_MAXN];
};

// C[MxN] (ld ldc) = alpha A B (+ beta C); lanes own columns, eight rows at a time.
template <class VA, class VB>
__device__ void warp_gemm(int M, int N, int K, double alpha, const VA& A, const VB& B, double beta, double* C,
                          int ldc) {
  const int lane = threadIdx.x & 31;
  for (int n0 = 0; n0 < N; n0 += 32) {
    const int n = n0 + lane;
    for (int m0 = 0; m0 < M; m0 += 8) {
      double acc[8];
#pragma unroll
      for (int i = 0; i < 8; i++) acc[i] = 0.0;
      if (n < N)
        for (int k = 0; k < K; k++) {
          const double b = B.get(k, n);
#pragma unroll
          for (int i = 0; i < 8; i++)
            if (m0 + i < M) acc[i] = fma(A.get(m0 + i, k), b, acc[i]);
        }
      if (n < N)
#pragma unroll
        for (int i = 0; i < 8; i++)
          if (m0 + i < M) {
            double* cp = C + (size_t)(m0 + i) * ldc + n;
            *cp = (beta == 0.0 ? 0.0 : beta * *cp) + alpha * acc[i];
          }
    }
  }
  __syncwarp();
}

// Householder tridiagonalisation (as cta_tridiag) with one warp.  p = tau A' v
// is formed column by column (A' symmetric): lanes own rows, no reductions.
__device__ void warp_tridiag(double* A, int n, int lda, double* d, double* e, double* tau, double* v, double* p) {
  const int lane = threadIdx.x & 31;
  for (int k = 0; k + 2 < n; k++) {
    const int L = n - k - 1;
    double* Ak = A + (size_t)(k + 1) * lda + (k + 1);
    double part = 0.0;
    for (int t = lane; t < L; t += 32) {
      const double x = A[(size_t)(k + 1 + t) * lda + k];
      v[t] = x;
      if (t > 0) part += x * x;
    }
    const double sigma = warp_sum(part);
    __syncwarp();
    double tk = 0.0, sc = 0.0;
    if (lane == 0) {
      const double alpha = v[0];
      double beta = alpha;
      if (sigma > 0.0) {
        const double mu = sqrt(alpha * alpha + sigma);
        beta = alpha <= 0.0 ? mu : -mu;
        tk = (beta - alpha) / beta;
        sc = 1.0 / (alpha - beta);
      }
      d[k] = A[(size_t)k * lda + k];
      e[k] = beta;
      tau[k] = tk;
    }
    tk = __shfl_sync(0xffffffffu, tk, 0);
    sc = __shfl_sync(0xffffffffu, sc, 0);
    if (tk != 0.0) {
      for (int t = lane; t < L; t += 32) v[t] = (t == 0) ? 1.0 : v[t] * sc;
      __syncwarp();
      for (int rb = 0; rb < L; rb += 128) {
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int c = 0; c < L; c++) {
          const double vc = v[c];
          const double* row = Ak + (size_t)c * lda;
#pragma unroll
          for (int j = 0; j < 4; j++) {
            const int r = rb + lane + 32 * j;
            if (r < L) acc[j] = fma(row[r], vc, acc[j]);
          }
        }
#pragma unroll
        for (int j = 0; j < 4; j++) {
          const int r = rb + lane + 32 * j;
          if (r < L) p[r] = tk * acc[j];
        }
      }
      __syncwarp();
      double pv = 0.0;
      for (int t = lane; t < L; t += 32) pv += p[t] * v[t];
      const double Kc = 0.5 * tk * warp_sum(pv);
      for (int t = lane; t < L; t += 32) p[t] -= Kc * v[t];
      __syncwarp();
      for (int c = 0; c < L; c++) {
        double* row = Ak + (size_t)c * lda;
        const double vc = v[c], wc = p[c];
        for (int r = lane; r < L; r += 32) row[r] -= vc * p[r] + wc * v[r];
      }
      for (int t = lane + 1; t < L; t += 32) A[(size_t)(k + 1 + t) * lda + k] = v[t];
    }
    __syncwarp();
  }
  if (lane == 0) {
    if (n >= 2) {
      d[n - 2] = A[(size_t)(n - 2) * lda + (n - 2)];
      e[n - 2] = A[(size_t)(n - 1) * lda + (n - 2)];
      if (n >= 3) tau[n - 2] = 0.0;
    }
    d[n - 1] = A[(size_t)(n - 1) * lda + (n - 1)];
    tau[n - 1] = 0.0;
  }
  __syncwarp();
}

// Z = H_0 ... H_{n-3} (row-major, ldz) by backward accumulation, one warp.
__device__ void warp_form_z(const double* A, int n, int lda, const double* tau, double* Z, int ldz, double* vs,
                            double* y) {
  const int lane = threadIdx.x & 31;
  for (int r = 0; r < n; r++)
    for (int c = lane; c < n; c += 32) Z[(size_t)r * ldz + c] = (r == c) ? 1.0 : 0.0;
  __syncwarp();
  for (int k = n - 3; k >= 0; k--) {
    const double tk = tau[k];
    if (tk == 0.0) continue;
    const int L = n - k - 1;
    for (int r = lane; r < L; r += 32) vs[r] = (r == 0) ? 1.0 : A[(size_t)(k + 1 + r) * lda + k];
    __syncwarp();
    for (int c = lane; c < L; c += 32) {
      double s = 0.0;
      for (int r = 0; r < L; r++) s = fma(vs[r], Z[(size_t)(k + 1 + r) * ldz + (k + 1 + c)], s);
      y[c] = tk * s;
    }
    __syncwarp();
    for (int r = 0; r < L; r++) {
      const double vr = vs[r];
      double* zr = Z + (size_t)(k + 1 + r) * ldz + (k + 1);
      for (int c = lane; c < L; c += 32) zr[c] -= vr * y[c];
    }
    __syncwarp();
  }
}

// Implicit symmetric QR with the Wilkinson shift (as cta_tridiag_qr), lane 0
// chasing the bulge in shared memory, all lanes rotating the rows of Z.
__device__ int warp_tridiag_qr(double* d, double* e, int n, double* Z, int ldz, double* cs) {
  const int lane = threadIdx.x & 31;
  const double eps = 2.220446049250313e-16;
  const int max_sweeps = 40 * n + 100;
  for (int sweeps = 0;; sweeps++) {
    int l = 0, h = 0, done = 0;
    if (lane == 0) {
      h = n - 1;
      while (h > 0) {
        if (fabs(e[h - 1]) <= eps * (fabs(d[h - 1]) + fabs(d[h]))) { e[h - 1] = 0.0; h--; }
        else break;
      }
      if (h == 0) done = 1;
      else {
        l = h - 1;
        while (l > 0) {
          if (fabs(e[l - 1]) <= eps * (fabs(d[l - 1]) + fabs(d[l]))) { e[l - 1] = 0.0; break; }
          l--;
        }
        const double delta = 0.5 * (d[h - 1] - d[h]);
        const double eh = e[h - 1];
        const double den = delta + copysign(sqrt(delta * delta + eh * eh), delta);
        const double mu = d[h] - (den != 0.0 ? eh * eh / den : 0.0);
        double x = d[l] - mu, z = e[l];
        for (int k = l; k < h; k++) {
          const double rr = sqrt(x * x + z * z);
          double c = 1.0, s = 0.0;
          if (rr != 0.0) {
            const double inv = 1.0 / rr;
            c = x * inv;
            s = z * inv;
          }
          if (k > l) e[k - 1] = rr;
          const double a = d[k], b = e[k], cc = d[k + 1];
          const double cs2 = c * s, c2 = c * c, s2 = s * s;
          d[k] = c2 * a + 2.0 * cs2 * b + s2 * cc;
          d[k + 1] = s2 * a - 2.0 * cs2 * b + c2 * cc;
          e[k] = cs2 * (cc - a) + (c2 - s2) * b;
          if (k + 1 < h) {
            x = e[k];
            z = s * e[k + 1];
            e[k + 1] = c * e[k + 1];
          }
          cs[2 * k] = c;
          cs[2 * k + 1] = s;
        }
      }
    }
    done = __shfl_sync(0xffffffffu, done, 0);
    l = __shfl_sync(0xffffffffu, l, 0);
    h = __shfl_sync(0xffffffffu, h, 0);
    __syncwarp();
    if (done) return 0;
    if (sweeps >= max_sweeps) return 1;
    for (int row = lane; row < n; row += 32) {
      double* zr = Z + (size_t)row * ldz;
      double carry = zr[l];
      for (int k = l; k < h; k++) {
        const double c = cs[2 * k], s = cs[2 * k + 1];
        const double y = zr[k + 1];
        zr[k] = c * carry + s * y;
        carry = -s * carry + c * y;
      }
      zr[h] = carry;
    }
    __syncwarp();
  }
}

// Full eigen-decomposition of A (n x n, destroyed) by one warp: eigenvalues in
// w (global), eigenvectors in the columns of Z.  Returns 0 on success.
__device__ int warp_syev(double* A, int n, double* w, double* Z, double* tau, WarpSm& ws) {
  const int lane = threadIdx.x & 31;
  if (n == 1) {
    if (lane == 0) { w[0] = A[0]; Z[0] = 1.0; }
    __syncwarp();
    return 0;
  }
  warp_tridiag(A, n, n, ws.d, ws.e, tau, ws.v, ws.p);
  warp_form_z(A, n, n, tau, Z, n, ws.v, ws.p);
  const int rc = warp_tridiag_qr(ws.d, ws.e, n, Z, n, ws.cs);
  for (int t = lane; t < n; t += 32) w[t] = ws.d[t];
  __syncwarp();
  return rc;
}

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
