// CTA-wide FP64 symmetric eigen-solvers used by the OSV build (Eq. osv_gen)
// and by the pair preconditioner (Eq. prec_eig).
//
//  * cta_tridiag     Householder reduction A = Z T Z^T to tridiagonal form
//                    (reflectors H_k = I - tau_k v_k v_k^T, v_k[0] = 1, stored
//                    below the sub-diagonal of A).
//  * cta_form_z      Z = H_0 H_1 ... H_{n-3} by backward accumulation.
//  * cta_tridiag_qr  implicit symmetric QR steps with the Wilkinson shift
//                    (Golub & Van Loan, Matrix Computations, Alg. 8.3.2/8.3.3),
//                    rotations accumulated into the columns of Z.
//  * sturm_count / multisection / inverse iteration + back-transformation for the
//    eigenpairs above a threshold, used when only a few OSVs out of a large
//    virtual space are kept.
// All routines are called by every thread of a CTA of NT threads.
#pragma once
#include "common.cuh"

namespace osv {

// Householder tridiagonalisation of the symmetric n x n matrix A (row-major,
// lda; global or shared memory), in place.  Outputs d[n], e[n-1] (any memory)
// and tau[n]; v and p are shared scratch of n elements each, red >= 33.
// T = double or float.
template <int NTH = NT, class T = double>
__device__ inline void cta_tridiag(T* A, int n, int lda, T* d, T* e, T* tau, T* v, T* p, T* red) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = NTH / 32;
  __shared__ T s_tau;
  for (int k = 0; k + 2 < n; k++) {
    const int L = n - k - 1;          // trailing block rows/cols k+1 .. n-1
    T* Ak = A + (size_t)(k + 1) * lda + (k + 1);   // trailing block origin
    T part = T(0.0);
    for (int t = tid; t < L; t += NTH) {
      const T x = A[(size_t)(k + 1 + t) * lda + k];
      v[t] = x;
      if (t > 0) part += x * x;
    }
    const T sigma = cta_sum(part, red);
    if (tid == 0) {
      const T alpha = v[0];
      T tu = T(0.0), beta = alpha;
      if (sigma > T(0.0)) {
        const T mu = sqrt(alpha * alpha + sigma);
        beta = alpha <= T(0.0) ? mu : -mu;
        tu = (beta - alpha) / beta;
        const T v0 = alpha - beta;
        red[0] = T(1.0) / v0;   // scale for v[1..]
      }
      s_tau = tu;
      d[k] = A[(size_t)k * lda + k];
      e[k] = beta;
      tau[k] = tu;
    }
    __syncthreads();
    const T tk = s_tau;
    if (tk != T(0.0)) {
      const T sc = red[0];
      for (int t = tid; t < L; t += NTH) v[t] = (t == 0) ? T(1.0) : v[t] * sc;
      __syncthreads();
      // p = tau * A' v  (warp per row, lanes over columns)
      for (int r = warp; r < L; r += nwarp) {
        const T* row = Ak + (size_t)r * lda;
        T s0 = T(0.0), s1 = T(0.0), s2 = T(0.0), s3 = T(0.0);
        int c = lane;
        for (; c + 96 < L; c += 128) {       // four independent loads in flight per lane
          const T a0 = row[c], a1 = row[c + 32], a2 = row[c + 64], a3 = row[c + 96];
          s0 += a0 * v[c];
          s1 += a1 * v[c + 32];
          s2 += a2 * v[c + 64];
          s3 += a3 * v[c + 96];
        }
        for (; c < L; c += 32) s0 += row[c] * v[c];
        const T s = warp_sum((s0 + s1) + (s2 + s3));
        if (lane == 0) p[r] = tk * s;
      }
      __syncthreads();
      T pv = T(0.0);
      for (int t = tid; t < L; t += NTH) pv += p[t] * v[t];
      const T Kc = T(0.5) * tk * cta_sum(pv, red);
      for (int t = tid; t < L; t += NTH) p[t] -= Kc * v[t];   // p becomes w
      __syncthreads();
      // A' -= v w^T + w v^T
      for (int r = warp; r < L; r += nwarp) {
        T* row = Ak + (size_t)r * lda;
        const T vr = v[r], wr = p[r];
        int c = lane;
        for (; c + 96 < L; c += 128) {
          const T a0 = row[c], a1 = row[c + 32], a2 = row[c + 64], a3 = row[c + 96];
          row[c] = a0 - (vr * p[c] + wr * v[c]);
          row[c + 32] = a1 - (vr * p[c + 32] + wr * v[c + 32]);
          row[c + 64] = a2 - (vr * p[c + 64] + wr * v[c + 64]);
          row[c + 96] = a3 - (vr * p[c + 96] + wr * v[c + 96]);
        }
        for (; c < L; c += 32) row[c] -= vr * p[c] + wr * v[c];
      }
      // keep the reflector below the sub-diagonal of column k
      for (int t = tid + 1; t < L; t += NTH) A[(size_t)(k + 1 + t) * lda + k] = v[t];
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (n >= 2) {
      d[n - 2] = A[(size_t)(n - 2) * lda + (n - 2)];
      e[n - 2] = A[(size_t)(n - 1) * lda + (n - 2)];
      if (n >= 3) tau[n - 2] = T(0.0);
    }
    d[n - 1] = A[(size_t)(n - 1) * lda + (n - 1)];
    tau[n - 1] = T(0.0);
  }
  __syncthreads();
}

// Householder tridiagonalisation as cta_tridiag, for large n with A in global
// memory: the symmetric matvec p = tau A' v is formed column-wise (thread c
// owns column c and walks the rows, so every load instruction of a warp is
// coalesced and a thread keeps many independent loads in flight), and the
// rank-2 update is applied the same way.  Reflector k is also stored
// contiguously in row k to the right of the diagonal (A[k][k+1+t] = v_t,
// v_0 = 1; that part of the upper triangle is not read again), for the
// back-transformation.
template <int NTH = NT>
__device__ inline void cta_tridiag_col(double* A, int n, int lda, double* d, double* e, double* tau, double* v,
                                       double* p, double* red) {
  const int tid = threadIdx.x;
  __shared__ double s_tc, s_sc;
  for (int k = 0; k + 2 < n; k++) {
    const int L = n - k - 1;
    double* Ak = A + (size_t)(k + 1) * lda + (k + 1);
    double part = 0.0;
    for (int t = tid; t < L; t += NTH) {
      const double x = A[(size_t)(k + 1 + t) * lda + k];
      v[t] = x;
      if (t > 0) part += x * x;
    }
    const double sigma = cta_sum(part, red);
    if (tid == 0) {
      const double alpha = v[0];
      double tu = 0.0, beta = alpha, sc = 0.0;
      if (sigma > 0.0) {
        const double mu = sqrt(alpha * alpha + sigma);
        beta = alpha <= 0.0 ? mu : -mu;
        tu = (beta - alpha) / beta;
        sc = 1.0 / (alpha - beta);
      }
      s_tc = tu;
      s_sc = sc;
      d[k] = A[(size_t)k * lda + k];
      e[k] = beta;
      tau[k] = tu;
    }
    __syncthreads();
    const double tk = s_tc;
    if (tk != 0.0) {
      const double sc = s_sc;
      for (int t = tid; t < L; t += NTH) v[t] = (t == 0) ? 1.0 : v[t] * sc;
      __syncthreads();
      // p_c = tau sum_r A'[r][c] v_r   (A' symmetric)
      for (int c = tid; c < L; c += NTH) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int r = 0;
        for (; r + 3 < L; r += 4) {
          const double a0 = Ak[(size_t)r * lda + c], a1 = Ak[(size_t)(r + 1) * lda + c];
          const double a2 = Ak[(size_t)(r + 2) * lda + c], a3 = Ak[(size_t)(r + 3) * lda + c];
          s0 = fma(a0, v[r], s0);
          s1 = fma(a1, v[r + 1], s1);
          s2 = fma(a2, v[r + 2], s2);
          s3 = fma(a3, v[r + 3], s3);
        }
        for (; r < L; r++) s0 = fma(Ak[(size_t)r * lda + c], v[r], s0);
        p[c] = tk * ((s0 + s1) + (s2 + s3));
      }
      __syncthreads();
      double pv = 0.0;
      for (int t = tid; t < L; t += NTH) pv += p[t] * v[t];
      const double Kc = 0.5 * tk * cta_sum(pv, red);
      for (int t = tid; t < L; t += NTH) p[t] -= Kc * v[t];
      __syncthreads();
      // A'[r][c] -= v_r w_c + w_r v_c
      for (int c = tid; c < L; c += NTH) {
        const double vc = v[c], wc = p[c];
        int r = 0;
        for (; r + 3 < L; r += 4) {
          double* a = Ak + (size_t)r * lda + c;
          const double a0 = a[0], a1 = a[lda], a2 = a[2 * (size_t)lda], a3 = a[3 * (size_t)lda];
          a[0] = a0 - (v[r] * wc + p[r] * vc);
          a[lda] = a1 - (v[r + 1] * wc + p[r + 1] * vc);
          a[2 * (size_t)lda] = a2 - (v[r + 2] * wc + p[r + 2] * vc);
          a[3 * (size_t)lda] = a3 - (v[r + 3] * wc + p[r + 3] * vc);
        }
        for (; r < L; r++) Ak[(size_t)r * lda + c] -= v[r] * wc + p[r] * vc;
      }
      for (int t = tid + 1; t < L; t += NTH) A[(size_t)(k + 1 + t) * lda + k] = v[t];
      for (int t = tid; t < L; t += NTH) A[(size_t)k * lda + (k + 1 + t)] = v[t];
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (n >= 2) {
      d[n - 2] = A[(size_t)(n - 2) * lda + (n - 2)];
      e[n - 2] = A[(size_t)(n - 1) * lda + (n - 2)];
      if (n >= 3) tau[n - 2] = 0.0;
    }
    d[n - 1] = A[(size_t)(n - 1) * lda + (n - 1)];
    tau[n - 1] = 0.0;
  }
  __syncthreads();
}

// Householder tridiagonalisation of the symmetric A (row-major, lda, global
// memory) keeping only its lower triangle, for the OSV eigenproblem.  Each
// step fuses the rank-2 update of the previous reflector with the symmetric
// matvec of the current one, in one pass over the lower triangle of the
// trailing block: per stored element two FMAs of the update and two of the
// matvec (its column sum and, through a shared-memory tile, its row sum),
// against three FMAs per element of the full matrix and three passes over it
// in cta_tridiag_col.  The trailing block is cut into 32 x 32 tiles, handled
// by ntw warps in a fixed order; their partial sums go to gpart and are added
// in a fixed order, so the result is deterministic.
// Outputs as cta_tridiag_col: d, e, tau, and reflector k in row k to the right
// of the diagonal (A[k][k+1+t] = v_t, v_0 = 1).
// sm: 4 n + 64 doubles (vp, wp, vk, p, red) + ntw * 32 * 33 doubles of tiles;
// gpart: nb (nb + 1) / 2 * 64 doubles, nb = ceil((n - 1) / 32).
template <int NTH>
__device__ inline void cta_tridiag_sym(double* A, int n, int lda, double* d, double* e, double* tau, double* sm,
                                       int ntw, double* gpart) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double* vp = sm;            // previous reflector v_{k-1}, by global index (0 outside its range)
  double* wp = vp + n;        // previous w_{k-1}
  double* vk = wp + n;        // current reflector v_k
  double* p = vk + n;         // A_k v_k, then w_k
  double* red = p + n;        // 64
  double* tiles = red + 64;   // ntw x 32 x 33
  __shared__ double s_tc, s_sc;
  for (int t = tid; t < n; t += NTH) { vp[t] = 0.0; wp[t] = 0.0; }
  __syncthreads();
  for (int k = 0; k + 2 < n; k++) {
    const int L = n - k - 1, k1 = k + 1;
    // (a) column k (rows k..n-1) receives the previous update
    double part = 0.0;
    for (int r = k + tid; r < n; r += NTH) {
      double a = A[(size_t)r * lda + k];
      if (k > 0) a = fma(-wp[r], vp[k], fma(-vp[r], wp[k], a));
      if (r == k) d[k] = a;
      else {
        vk[r] = a;
        if (r > k1) part += a * a;
      }
    }
    // (b) Householder reflector of column k below the diagonal
    const double sigma = cta_sum(part, red);
    if (tid == 0) {
      const double alpha = vk[k1];
      double tu = 0.0, beta = alpha, sc = 0.0;
      if (sigma > 0.0) {
        const double mu = sqrt(alpha * alpha + sigma);
        beta = alpha <= 0.0 ? mu : -mu;
        tu = (beta - alpha) / beta;
        sc = 1.0 / (alpha - beta);
      }
      s_tc = tu;
      s_sc = sc;
      e[k] = beta;
      tau[k] = tu;
    }
    __syncthreads();
    const double tk = s_tc, sc = s_sc;
    for (int r = k1 + tid; r < n; r += NTH) {
      const double v = (r == k1) ? 1.0 : vk[r] * sc;
      vk[r] = (tk != 0.0) ? v : 0.0;
      A[(size_t)k * lda + r] = v;                 // reflector, row storage
    }
    for (int t = tid; t < k1; t += NTH) vk[t] = 0.0;
    __syncthreads();
    // (c) fused sweep over the lower triangle of the trailing block
    const int nb = (L + 31) >> 5;
    const int ntile = nb * (nb + 1) / 2;
    if (warp < ntw) {
      double* tb = tiles + (size_t)warp * 32 * 33;
      for (int tl = warp; tl < ntile; tl += ntw) {
        int bi = 0;
        while ((bi + 1) * (bi + 2) / 2 <= tl) bi++;
        const int bj = tl - bi * (bi + 1) / 2;
        const int r0 = k1 + 32 * bi, c0 = k1 + 32 * bj;
        const int c = c0 + lane;
        const bool cin = c < n;
        const double vpc = cin ? vp[c] : 0.0, wpc = cin ? wp[c] : 0.0;
        double colsum = 0.0;
        for (int i0 = 0; i0 < 32; i0 += 8) {   // eight rows' loads in flight before their arithmetic
          double av[8];
#pragma unroll
          for (int u = 0; u < 8; u++) {
            const int r = r0 + i0 + u;
            av[u] = (cin && r < n && r >= c) ? A[(size_t)r * lda + c] : 0.0;
          }
#pragma unroll
          for (int u = 0; u < 8; u++) {
            const int r = r0 + i0 + u;
            double a = 0.0;
            if (cin && r < n && r >= c) {
              a = av[u];
              if (k > 0) {
                a = fma(-wp[r], vpc, fma(-vp[r], wpc, a));
                A[(size_t)r * lda + c] = a;
              }
              colsum = fma(a, vk[r], colsum);
            }
            tb[(i0 + u) * 33 + lane] = (r > c) ? a : 0.0;   // the row sums take the strictly lower part
          }
        }
        __syncwarp();
        double rowsum = 0.0;
        for (int j = 0; j < 32; j++) rowsum = fma(tb[lane * 33 + j], vk[min(c0 + j, n - 1)], rowsum);   // tb = 0 past n
        double* gp = gpart + (size_t)tl * 64;
        gp[lane] = colsum;
        gp[32 + lane] = rowsum;
        __syncwarp();
      }
    }
    __syncthreads();
    // (d) p = A_k v_k from the partial sums (fixed order), then w_k
    double pv = 0.0;
    for (int c = k1 + tid; c < n; c += NTH) {
      const int b = (c - k1) >> 5, o = (c - k1) & 31;
      double s = 0.0;
      for (int bi = b; bi < nb; bi++) s += gpart[(size_t)(bi * (bi + 1) / 2 + b) * 64 + o];        // column sums
      for (int bj = 0; bj <= b; bj++) s += gpart[(size_t)(b * (b + 1) / 2 + bj) * 64 + 32 + o];   // row sums
      s *= tk;
      p[c] = s;
      pv += s * vk[c];
    }
    const double Kc = 0.5 * tk * cta_sum(pv, red);
    for (int c = tid; c < n; c += NTH) {
      const double w = (c >= k1) ? p[c] - Kc * vk[c] : 0.0;
      wp[c] = w;
      vp[c] = vk[c];
    }
    __syncthreads();
  }
  // the trailing 2 x 2 block receives the last update
  if (tid == 0) {
    if (n >= 2) {
      const int a0 = n - 2, a1 = n - 1;
      double x00 = A[(size_t)a0 * lda + a0], x10 = A[(size_t)a1 * lda + a0], x11 = A[(size_t)a1 * lda + a1];
      if (n >= 3) {
        x00 -= 2.0 * vp[a0] * wp[a0];
        x10 -= vp[a1] * wp[a0] + wp[a1] * vp[a0];
        x11 -= 2.0 * vp[a1] * wp[a1];
        tau[n - 2] = 0.0;
      }
      d[a0] = x00;
      e[a0] = x10;
      d[a1] = x11;
    } else {
      d[0] = A[0];
    }
    tau[n - 1] = 0.0;
  }
  __syncthreads();
}

// ---------------------------------------------------------------- double-float
// (arithmetic in common.cuh)
// CTA sum in double-float (fixed order); red: >= 66 floats of shared memory.
__device__ inline dfl cta_sum_df(dfl v, float* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = df_add(v, df_shfl_xor(v, o));
  __syncthreads();
  if (lane == 0) { red[2 * w] = v.h; red[2 * w + 1] = v.l; }
  __syncthreads();
  if (threadIdx.x == 0) {
    dfl s{0.f, 0.f};
    for (int k = 0; k < nw; k++) s = df_add(s, dfl{red[2 * k], red[2 * k + 1]});
    red[64] = s.h;
    red[65] = s.l;
  }
  __syncthreads();
  return dfl{red[64], red[65]};
}

// cta_tridiag_sym in double-float arithmetic, for the mixed-form OSV build
// (whose T_ii carries ~35 significant bits, so the ~48 bits here do not limit
// it): the same fused sweep over the lower triangle, with A held as (hi, lo)
// FP32 pairs in place of its FP64 elements (converted on the first step).
// Outputs in FP64: d, e, tau, and reflector k in row k to the right of the
// diagonal (A[k][k+1+t] = v_t, v_0 = 1), as cta_tridiag_sym.
// sm: 4 n + 64 doubles (vp, wp, vk, p as pairs; reductions) + ntw * 16 * 33 doubles of staging
// tiles (each 32 x 32 tile goes through them in two halves of 16 rows, so that every warp of
// the CTA fits one).
// refl_df: reflector k stored as (hi, lo) pairs instead of FP64 (read by k_eig_back_df).
template <int NTH>
__device__ inline void cta_tridiag_sym_df(double* A, int n, int lda, double* d, double* e, double* tau, double* sm,
                                          int ntw, double* gpart_d, bool refl_df) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  dfl* vp = reinterpret_cast<dfl*>(sm);   // previous reflector v_{k-1}
  dfl* wp = vp + n;                        // previous w_{k-1}
  dfl* vk = wp + n;                        // current reflector v_k
  dfl* p = vk + n;                         // A_k v_k, then w_k
  float* red = reinterpret_cast<float*>(p + n);   // 64 doubles of room
  dfl* tiles = reinterpret_cast<dfl*>(sm + 4 * n + 64);   // ntw x 16 x 33 pairs
  dfl* gpart = reinterpret_cast<dfl*>(gpart_d);
  dfl* Ad = reinterpret_cast<dfl*>(A);     // element (r, c) of the lower triangle at Ad[r * lda + c]
  __shared__ double s_tc, s_sc;
  // the lower triangle to (hi, lo) pairs, in place
  for (int r = warp; r < n; r += NTH / 32)
    for (int c = lane; c <= r; c += 32) Ad[(size_t)r * lda + c] = df_from(A[(size_t)r * lda + c]);
  for (int t = tid; t < n; t += NTH) { vp[t] = dfl{0.f, 0.f}; wp[t] = dfl{0.f, 0.f}; }
  __syncthreads();
  for (int k = 0; k + 2 < n; k++) {
    const int L = n - k - 1, k1 = k + 1;
    // (a) column k (rows k..n-1) receives the previous update
    dfl part{0.f, 0.f};
    const dfl vpk = vp[k], wpk = wp[k];
    for (int r = k + tid; r < n; r += NTH) {
      dfl a = Ad[(size_t)r * lda + k];
      if (k > 0) a = df_fma(df_neg(wp[r]), vpk, df_fma(df_neg(vp[r]), wpk, a));
      if (r == k) d[k] = df_to(a);
      else {
        vk[r] = a;
        if (r > k1) part = df_fma(a, a, part);
      }
    }
    // (b) Householder reflector of column k below the diagonal (scalars in FP64)
    const double sigma = df_to(cta_sum_df(part, red));
    if (tid == 0) {
      const double alpha = df_to(vk[k1]);
      double tu = 0.0, beta = alpha, sc = 0.0;
      if (sigma > 0.0) {
        const double mu = sqrt(alpha * alpha + sigma);
        beta = alpha <= 0.0 ? mu : -mu;
        tu = (beta - alpha) / beta;
        sc = 1.0 / (alpha - beta);
      }
      s_tc = tu;
      s_sc = sc;
      e[k] = beta;
      tau[k] = tu;
    }
    __syncthreads();
    const double tk = s_tc;
    const dfl scd = df_from(s_sc);
    for (int r = k1 + tid; r < n; r += NTH) {
      const dfl v = (r == k1) ? dfl{1.f, 0.f} : df_mul(vk[r], scd);
      vk[r] = (tk != 0.0) ? v : dfl{0.f, 0.f};
      if (refl_df) Ad[(size_t)k * lda + r] = v;    // reflector, row storage (not read again by this sweep)
      else A[(size_t)k * lda + r] = df_to(v);
    }
    for (int t = tid; t < k1; t += NTH) vk[t] = dfl{0.f, 0.f};
    __syncthreads();
    // (c) fused sweep over the lower triangle of the trailing block
    const int nb = (L + 31) >> 5;
    const int ntile = nb * (nb + 1) / 2;
    if (warp < ntw) {
      dfl* tb = tiles + (size_t)warp * 16 * 33;
      for (int tl = warp; tl < ntile; tl += ntw) {
        int bi = 0;
        while ((bi + 1) * (bi + 2) / 2 <= tl) bi++;
        const int bj = tl - bi * (bi + 1) / 2;
        const int r0 = k1 + 32 * bi, c0 = k1 + 32 * bj;
        const int c = c0 + lane;
        const bool cin = c < n;
        const dfl nvpc = cin ? df_neg(vp[c]) : dfl{0.f, 0.f}, nwpc = cin ? df_neg(wp[c]) : dfl{0.f, 0.f};
        dfl* gp = gpart + (size_t)tl * 64;
        float csh = 0.f, csl = 0.f;   // column sum, unnormalised pair
        for (int h = 0; h < 32; h += 16) {
          for (int i0 = h; i0 < h + 16; i0 += 8) {   // eight rows' loads in flight before their arithmetic
            dfl av[8];
#pragma unroll
            for (int u = 0; u < 8; u++) {
              const int r = r0 + i0 + u;
              av[u] = (cin && r < n && r >= c) ? Ad[(size_t)r * lda + c] : dfl{0.f, 0.f};
            }
#pragma unroll
            for (int u = 0; u < 8; u++) {
              const int r = r0 + i0 + u;
              dfl a{0.f, 0.f};
              if (cin && r < n && r >= c) {
                a = av[u];
                if (k > 0) {
                  a = df_fma2(vp[r], nwpc, wp[r], nvpc, a);
                  Ad[(size_t)r * lda + c] = a;
                }
                df_acc(csh, csl, a, vk[r]);
              }
              tb[(i0 - h + u) * 33 + lane] = (r > c) ? a : dfl{0.f, 0.f};   // the row sums take the strictly lower part
            }
          }
          __syncwarp();
          // row sums of these 16 rows: lane (g, rho) sums row rho over column half g, and the
          // two halves are added in a fixed order
          const int rho = lane & 15, g = lane >> 4;
          float rsh = 0.f, rsl = 0.f;
#pragma unroll 8
          for (int j = 16 * g; j < 16 * g + 16; j++) df_acc(rsh, rsl, tb[rho * 33 + j], vk[min(c0 + j, n - 1)]);
          const float oh = __shfl_xor_sync(0xffffffffu, rsh, 16), ol = __shfl_xor_sync(0xffffffffu, rsl, 16);
          if (g == 0) {
            float sh, st;
            two_sum_f(rsh, oh, sh, st);
            gp[32 + h + rho] = df_norm(sh, (rsl + ol) + st);
          }
          __syncwarp();
        }
        gp[lane] = df_norm(csh, csl);
      }
    }
    __syncthreads();
    // (d) p = A_k v_k from the partial sums (fixed order), then w_k
    const dfl tkd = df_from(tk);
    dfl pv{0.f, 0.f};
    for (int c = k1 + tid; c < n; c += NTH) {
      const int b = (c - k1) >> 5, o = (c - k1) & 31;
      dfl s2{0.f, 0.f};
      for (int bi = b; bi < nb; bi++) s2 = df_add(s2, gpart[(size_t)(bi * (bi + 1) / 2 + b) * 64 + o]);
      for (int bj = 0; bj <= b; bj++) s2 = df_add(s2, gpart[(size_t)(b * (b + 1) / 2 + bj) * 64 + 32 + o]);
      s2 = df_mul(s2, tkd);
      p[c] = s2;
      pv = df_fma(s2, vk[c], pv);
    }
    const dfl Kc = df_mul(df_from(0.5 * tk), cta_sum_df(pv, red));
    const dfl nKc = df_neg(Kc);
    for (int c = tid; c < n; c += NTH) {
      const dfl w = (c >= k1) ? df_fma(nKc, vk[c], p[c]) : dfl{0.f, 0.f};
      wp[c] = w;
      vp[c] = vk[c];
    }
    __syncthreads();
  }
  // the trailing 2 x 2 block receives the last update
  if (tid == 0) {
    if (n >= 2) {
      const int a0 = n - 2, a1 = n - 1;
      double x00 = df_to(Ad[(size_t)a0 * lda + a0]), x10 = df_to(Ad[(size_t)a1 * lda + a0]);
      double x11 = df_to(Ad[(size_t)a1 * lda + a1]);
      if (n >= 3) {
        const double v0 = df_to(vp[a0]), v1 = df_to(vp[a1]), w0 = df_to(wp[a0]), w1 = df_to(wp[a1]);
        x00 -= 2.0 * v0 * w0;
        x10 -= v1 * w0 + w1 * v0;
        x11 -= 2.0 * v1 * w1;
        tau[n - 2] = 0.0;
      }
      d[a0] = x00;
      e[a0] = x10;
      d[a1] = x11;
    } else {
      d[0] = df_to(Ad[0]);
    }
    tau[n - 1] = 0.0;
  }
  __syncthreads();
}

// Z (n x n, row-major, ldz) = H_0 H_1 ... H_{n-3} from the reflectors left in A.
// y, vs: shared scratch of n doubles each.
template <int NTH = NT>
__device__ inline void cta_form_z(const double* A, int n, int lda, const double* tau, double* Z, int ldz,
                                  double* y, double* vs) {
  const int tid = threadIdx.x;
  for (int t = tid; t < n * n; t += NTH) Z[(size_t)(t / n) * ldz + (t % n)] = (t / n == t % n) ? 1.0 : 0.0;
  __syncthreads();
  for (int k = n - 3; k >= 0; k--) {
    const double tk = tau[k];
    if (tk == 0.0) continue;
    const int L = n - k - 1;
    for (int r = tid; r < L; r += NTH) vs[r] = (r == 0) ? 1.0 : A[(size_t)(k + 1 + r) * lda + k];
    __syncthreads();
    // y_c = tau * sum_r v_r Z[k+1+r][k+1+c]
    for (int c = tid; c < L; c += NTH) {
      double s = 0.0;
      for (int r = 0; r < L; r++) s += vs[r] * Z[(size_t)(k + 1 + r) * ldz + (k + 1 + c)];
      y[c] = tk * s;
    }
    __syncthreads();
    for (int t = tid; t < L * L; t += NTH) {
      const int r = t / L, c = t % L;
      Z[(size_t)(k + 1 + r) * ldz + (k + 1 + c)] -= vs[r] * y[c];
    }
    __syncthreads();
  }
}

// Implicit symmetric QR on the tridiagonal (d[n], e[n-1]) with rotations
// accumulated into the columns of Z (n x n, row-major, ldz).  d, e must be in
// shared or global memory visible to thread 0; cs is shared scratch of 2n
// elements.  Returns 0 on convergence (d holds the eigenvalues, columns of Z the
// eigenvectors), 1 otherwise.  Every thread returns the same value.
// ZCM: Z stored column-major (Z[r][c] at Z[c * ldz + r]), so that the threads,
// one per row, rotate it with coalesced accesses.  T = double or float.
template <int NTH = NT, bool ZCM = false, class T = double>
__device__ inline int cta_tridiag_qr(T* d, T* e, int n, T* Z, int ldz, T* cs) {
  __shared__ int s_l, s_h, s_done;
  const int tid = threadIdx.x;
  const T eps = sizeof(T) == 8 ? T(2.220446049250313e-16) : T(1.1920929e-07);
  int sweeps = 0;
  const int max_sweeps = 40 * n + 100;
  while (true) {
    if (tid == 0) {
      int h = n - 1, l = 0, done = 0;
      // deflate negligible couplings from the bottom
      while (h > 0) {
        if (fabs(e[h - 1]) <= eps * (fabs(d[h - 1]) + fabs(d[h]))) { e[h - 1] = T(0.0); h--; }
        else break;
      }
      if (h == 0) done = 1;
      else {
        l = h - 1;
        while (l > 0) {
          if (fabs(e[l - 1]) <= eps * (fabs(d[l - 1]) + fabs(d[l]))) { e[l - 1] = T(0.0); break; }
          l--;
        }
        // Wilkinson shift from the trailing 2x2 of the unreduced block [l, h]
        const T delta = T(0.5) * (d[h - 1] - d[h]);
        const T eh = e[h - 1];
        const T den = delta + copysign(hypot(delta, eh), delta);
        const T mu = d[h] - (den != T(0.0) ? eh * eh / den : T(0.0));
        T x = d[l] - mu, z = e[l];
        for (int k = l; k < h; k++) {
          const T r = hypot(x, z);
          T c = T(1.0), s = T(0.0);
          if (r != T(0.0)) { c = x / r; s = z / r; }
          if (k > l) e[k - 1] = r;
          const T a = d[k], b = e[k], cc = d[k + 1];
          d[k] = c * c * a + T(2.0) * c * s * b + s * s * cc;
          d[k + 1] = s * s * a - T(2.0) * c * s * b + c * c * cc;
          e[k] = c * s * (cc - a) + (c * c - s * s) * b;
          if (k + 1 < h) {
            x = e[k];
            z = s * e[k + 1];
            e[k + 1] = c * e[k + 1];
          }
          cs[2 * k] = c;
          cs[2 * k + 1] = s;
        }
      }
      s_l = l; s_h = h; s_done = done;
    }
    __syncthreads();
    if (s_done) return 0;
    if (++sweeps > max_sweeps) return 1;
    const int l = s_l, h = s_h;
    // Z <- Z R_l^T R_{l+1}^T ... : column pair (k, k+1) rotated for k = l..h-1
    for (int row = tid; row < n; row += NTH) {
      T* zr = ZCM ? Z + row : Z + (size_t)row * ldz;
      const size_t zs = ZCM ? (size_t)ldz : 1;   // stride between the columns of one row
      T carry = zr[l * zs];
      for (int k = l; k < h; k++) {
        const T c = cs[2 * k], s = cs[2 * k + 1];
        const T y = zr[(k + 1) * zs];
        zr[k * zs] = c * carry + s * y;
        carry = -s * carry + c * y;
      }
      zr[h * zs] = carry;
    }
    __syncthreads();
  }
}

// Full symmetric eigen-decomposition of A (n x n, row-major lda, destroyed).
// On return w[0..n) holds the eigenvalues and column t of Z the eigenvector
// of w[t] (unordered).  d/e/tau: n doubles each (any memory visible to the
// CTA); sm: shared scratch of >= 4n + 33 doubles.  Returns 0 on success.
template <int NTH = NT>
__device__ inline int cta_syev(double* A, int n, int lda, double* w, double* Z, int ldz, double* e,
                               double* tau, double* sm) {
  double* v = sm;
  double* p = sm + n;
  double* cs = sm + 2 * n;      // 2n
  double* red = sm + 4 * n;     // 33
  if (n == 1) {
    if (threadIdx.x == 0) { w[0] = A[0]; Z[0] = 1.0; }
    __syncthreads();
    return 0;
  }
  cta_tridiag<NTH>(A, n, lda, w, e, tau, v, p, red);
  cta_form_z<NTH>(A, n, lda, tau, Z, ldz, v, p);
  // the bulge chase is sequential: run it on shared-memory copies of d and e
  for (int t = threadIdx.x; t < n; t += NTH) {
    v[t] = w[t];
    p[t] = (t + 1 < n) ? e[t] : 0.0;
  }
  __syncthreads();
  const int rc = cta_tridiag_qr<NTH>(v, p, n, Z, ldz, cs);
  for (int t = threadIdx.x; t < n; t += NTH) w[t] = v[t];
  __syncthreads();
  return rc;
}

// Z = H_0 H_1 ... H_{n-3} from the reflectors left in A, stored column-major
// (Z[r][c] at Z[c * ldz + r]); a warp per column forms the dot products along
// contiguous memory.  y, vs: shared scratch of n elements each.
// T = double or float.  ROWV: reflector k in row k to the right of the diagonal
// (cta_tridiag_sym) instead of below the sub-diagonal of column k (cta_tridiag).
template <int NTH = NT, class T, bool ROWV = false>
__device__ inline void cta_form_z_cm(const T* A, int n, int lda, const T* tau, T* Z, int ldz, T* y, T* vs) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = NTH / 32;
  for (int t = tid; t < n * n; t += NTH) Z[(size_t)(t / n) * ldz + (t % n)] = (t / n == t % n) ? T(1.0) : T(0.0);
  __syncthreads();
  for (int k = n - 3; k >= 0; k--) {
    const T tk = tau[k];
    if (tk == T(0.0)) continue;
    const int L = n - k - 1;
    for (int r = tid; r < L; r += NTH)
      vs[r] = (r == 0) ? T(1.0) : (ROWV ? A[(size_t)k * lda + k + 1 + r] : A[(size_t)(k + 1 + r) * lda + k]);
    __syncthreads();
    // y_c = tau * sum_r v_r Z[k+1+r][k+1+c]: column k+1+c is contiguous
    for (int c = warp; c < L; c += NW) {
      const T* zc = Z + (size_t)(k + 1 + c) * ldz + (k + 1);
      T s = T(0.0);
      for (int r = lane; r < L; r += 32) s = fma(vs[r], zc[r], s);
      s = warp_sum(s);
      if (lane == 0) y[c] = tk * s;
    }
    __syncthreads();
    for (int t = tid; t < L * L; t += NTH) {
      const int c = t / L, r = t % L;
      Z[(size_t)(k + 1 + c) * ldz + (k + 1 + r)] -= vs[r] * y[c];
    }
    __syncthreads();
  }
}

// Full symmetric eigen-decomposition as cta_syev with Z column-major: on
// return w[0..n) holds the eigenvalues and Z[t * ldz + a] is component a of
// the eigenvector of w[t] (unordered).  A (row-major, lda) is destroyed; e,
// tau: n elements each (any memory visible to the CTA); sm: shared scratch of
// >= 4n + 33 elements.  Returns 0 on success.  T = double or float.
template <int NTH = NT, class T>
__device__ inline int cta_syev_cm(T* A, int n, int lda, T* w, T* Z, int ldz, T* e, T* tau, T* sm) {
  T* v = sm;
  T* p = sm + n;
  T* cs = sm + 2 * n;      // 2n
  T* red = sm + 4 * n;     // 33
  if (n == 1) {
    if (threadIdx.x == 0) { w[0] = A[0]; Z[0] = T(1.0); }
    __syncthreads();
    return 0;
  }
  cta_tridiag<NTH>(A, n, lda, w, e, tau, v, p, red);
  cta_form_z_cm<NTH>(A, n, lda, tau, Z, ldz, v, p);
  for (int t = threadIdx.x; t < n; t += NTH) {   // the bulge chase runs on shared copies of d and e
    v[t] = w[t];
    p[t] = (t + 1 < n) ? e[t] : T(0.0);
  }
  __syncthreads();
  const int rc = cta_tridiag_qr<NTH, true>(v, p, n, Z, ldz, cs);
  for (int t = threadIdx.x; t < n; t += NTH) w[t] = v[t];
  __syncthreads();
  return rc;
}

// ---------------------------------------------------------------- batched QR
// The bulge chase of the implicit QR (as cta_tridiag_qr) is sequential; run by
// one thread of a CTA it leaves the rest of the CTA idle and, in FP64, uses a
// thirty-second of the FP64 pipe for every instruction.  These two routines
// split cta_tridiag_qr into (a) the chase of one tridiagonal per THREAD, many
// problems per warp, recording the sweeps (l, h) and their rotations, and (b)
// the application of the recorded rotations to the rows of Z by a CTA.  The
// sweeps are those of cta_tridiag_qr; the rotations are formed with fewer
// FP64 operations (chase_rotation).

// (a) One thread: chase (d[n], e[n-1]) to diagonal form, appending each sweep
// to swp (l, h pairs, capacity cap_s sweeps) and its rotations (c, s pairs,
// capacity cap_r) to rot.  Returns 0 on convergence (*n_sw sweeps recorded, d
// holds the eigenvalues), 1 if the sweep limit was reached, 2 if a record
// would overflow.  With partial, the overflow return also sets *n_sw to the
// sweeps recorded so far (d, e are then those after them, so a later call
// continues the chase).
// Givens rotation (c, s) with c x + s z = r >= 0, -s x + c z = 0.  FP64: one
// reciprocal square root; FP32: a correctly rounded square root and one
// division (unbiased rounding, so the accumulated rotations stay orthogonal
// to the FP32 rounding level).  hypot and two divisions where x^2 + z^2 could
// leave the normal range.
__device__ __forceinline__ void chase_rotation(double x, double z, double& c, double& s, double& r) {
  const double q = x * x + z * z;
  if (q > 1e-280 && q < 1e280) {
    const double inv = rsqrt(q);
    c = x * inv;
    s = z * inv;
    r = q * inv;
  } else {
    r = hypot(x, z);
    c = 1.0;
    s = 0.0;
    if (r != 0.0) { c = x / r; s = z / r; }
  }
}
__device__ __forceinline__ void chase_rotation(float x, float z, float& c, float& s, float& r) {
  const float q = x * x + z * z;
  if (q > 1e-36f && q < 1e36f) {
    r = sqrtf(q);
    const float inv = 1.f / r;
    c = x * inv;
    s = z * inv;
  } else {
    r = hypotf(x, z);
    c = 1.f;
    s = 0.f;
    if (r != 0.f) { c = x / r; s = z / r; }
  }
}

template <class T>
__device__ inline int tridiag_qr_record(T* __restrict__ d, T* __restrict__ e, int n, int* __restrict__ swp, int cap_s,
                                        T* __restrict__ rot, int cap_r, int* n_sw, bool partial = false) {
  const T eps = sizeof(T) == 8 ? T(2.220446049250313e-16) : T(1.1920929e-07);
  const int max_sweeps = 40 * n + 100;
  int ns = 0, nr = 0;
  *n_sw = 0;
  for (int sweeps = 0;; sweeps++) {
    int h = n - 1;
    while (h > 0) {
      if (fabs(e[h - 1]) <= eps * (fabs(d[h - 1]) + fabs(d[h]))) { e[h - 1] = T(0.0); h--; }
      else break;
    }
    if (h == 0) { *n_sw = ns; return 0; }
    if (sweeps >= max_sweeps) return 1;
    int l = h - 1;
    while (l > 0) {
      if (fabs(e[l - 1]) <= eps * (fabs(d[l - 1]) + fabs(d[l]))) { e[l - 1] = T(0.0); break; }
      l--;
    }
    if (ns >= cap_s || nr + (h - l) > cap_r) {
      if (partial) *n_sw = ns;
      return 2;
    }
    swp[2 * ns] = l;
    swp[2 * ns + 1] = h;
    ns++;
    T* cs = rot + 2 * (size_t)nr;
    nr += h - l;
    const T delta = T(0.5) * (d[h - 1] - d[h]);
    const T eh = e[h - 1];
    const T den = delta + copysign(hypot(delta, eh), delta);
    const T mu = d[h] - (den != T(0.0) ? eh * eh / den : T(0.0));
    // d[k] and e[k] as updated by the previous rotation stay in registers
    T dk = d[l], ek = e[l];
    T x = dk - mu, z = ek;
    for (int k = l; k < h; k++) {
      const T cc = d[k + 1];
      const T en = (k + 1 < h) ? e[k + 1] : T(0.0);
      T c, s, r;
      chase_rotation(x, z, c, s, r);
      if (k > l) e[k - 1] = r;
      const T a = dk, b = ek;
      d[k] = c * c * a + T(2.0) * c * s * b + s * s * cc;
      dk = s * s * a - T(2.0) * c * s * b + c * c * cc;
      const T ekn = c * s * (cc - a) + (c * c - s * s) * b;
      e[k] = ekn;
      if (k + 1 < h) {
        x = ekn;
        z = s * en;
        ek = c * en;
      }
      cs[2 * (k - l)] = c;
      cs[2 * (k - l) + 1] = s;
    }
    d[h] = dk;
  }
}

// (b) The CTA: apply the n_sw recorded sweeps to Z (n x n, column-major, ldz;
// a thread per row, coalesced).
template <int NTH = NT, class T>
__device__ inline void apply_qr_record_cm(T* Z, int ldz, int n, const int* swp, int n_sw, const T* rot) {
  for (int row = threadIdx.x; row < n; row += NTH) {
    T* zr = Z + row;
    const T* cs = rot;
    for (int q = 0; q < n_sw; q++) {
      const int l = swp[2 * q], h = swp[2 * q + 1];
      T carry = zr[(size_t)l * ldz];
      for (int k = l; k < h; k++, cs += 2) {
        const T c = cs[0], s = cs[1];
        const T y = zr[(size_t)(k + 1) * ldz];
        zr[(size_t)k * ldz] = c * carry + s * y;
        carry = -s * carry + c * y;
      }
      zr[(size_t)h * ldz] = carry;
    }
  }
  __syncthreads();
}

// Full symmetric eigen-decomposition as cta_syev_cm (FP64, Z column-major), with the
// implicit QR split as in the batched routines above: thread 0 chases the tridiagonal
// and records its rotations into the storage of A (no longer needed once Z is formed;
// lda == n), and the CTA applies each full record to the rows of Z, so the CTA waits
// once per record instead of once per rotation.  With ntw >= 2 warps of tiles in sm
// (after its 4 n + 64 doubles) the tridiagonalisation is the fused sweep cta_tridiag_sym,
// its partial sums in gpart.  Returns 0 on success, 1 otherwise.
template <int NTH = NT>
__device__ inline int cta_syev_cm_rec(double* A, int n, double* w, double* Z, int ldz, double* e, double* tau,
                                      double* sm, int ntw, double* gpart) {
  double* v = sm;
  double* p = sm + n;
  double* red = sm + 4 * n;
  __shared__ int s_rc, s_ns;
  if (n == 1) {
    if (threadIdx.x == 0) { w[0] = A[0]; Z[0] = 1.0; }
    __syncthreads();
    return 0;
  }
  if (ntw >= 2) {
    cta_tridiag_sym<NTH>(A, n, n, w, e, tau, sm, ntw, gpart);
    cta_form_z_cm<NTH, double, true>(A, n, n, tau, Z, ldz, v, p);
  } else {
    cta_tridiag<NTH>(A, n, n, w, e, tau, v, p, red);
    cta_form_z_cm<NTH>(A, n, n, tau, Z, ldz, v, p);
  }
  for (int t = threadIdx.x; t < n; t += NTH) {   // the chase runs on shared copies of d and e
    v[t] = w[t];
    p[t] = (t + 1 < n) ? e[t] : 0.0;
  }
  __syncthreads();
  const size_t room = (size_t)n * n;                       // doubles of A
  const int cap_s = (int)(room / 8 > 16 ? room / 8 : 16);  // sweeps: two ints (one double) each
  int* swp = reinterpret_cast<int*>(A);
  double* rot = A + cap_s;
  const int cap_r = (int)((room - (size_t)cap_s) / 2);     // rotations: (c, s) pairs
  int rc = 1;
  for (int chunk = 0; chunk < 64; chunk++) {
    if (threadIdx.x == 0) {
      int ns = 0;
      s_rc = tridiag_qr_record(v, p, n, swp, cap_s, rot, cap_r, &ns, true);
      s_ns = ns;
    }
    __syncthreads();
    apply_qr_record_cm<NTH>(Z, ldz, n, swp, s_ns, rot);   // ends with a barrier
    const int r = s_rc;
    __syncthreads();                                      // every thread has read s_rc
    if (r != 2) { rc = r; break; }
  }
  for (int t = threadIdx.x; t < n; t += NTH) w[t] = v[t];
  __syncthreads();
  return rc;
}

// ---------------------------------------------------------------- top-k
// Number of eigenvalues of the tridiagonal (d, e) strictly below x
// (Sturm sequence of the LDL^T pivots).
__device__ inline int sturm_count(const double* d, const double* e, int n, double x, double pivmin) {
  int cnt = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  cnt += q < 0.0;
  for (int i = 1; i < n; i++) {
    q = d[i] - x - e[i - 1] * e[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    cnt += q < 0.0;
  }
  return cnt;
}

// sturm_count with the squared off-diagonal e2[i] = e[i]^2 given.
__device__ inline int sturm_count_sq(const double* d, const double* e2, int n, double x, double pivmin) {
  int cnt = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  cnt += q < 0.0;
  for (int i = 1; i < n; i++) {
    q = d[i] - x - e2[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    cnt += q < 0.0;
  }
  return cnt;
}

// Eigenvalues with ascending indices n-1-t, t < k, of (d, e) by multisection
// on the Sturm count, called by one warp that handles t = t0, t0 + tstride, ...
// (at most tcount of them):
// g = lane / L lanes per eigenvalue split its interval at L points per step
// (log2(L+1) bits per Sturm sequence instead of one), until the interval is
// below 2 eps |lambda| or atol (the eigenvalues of the tridiagonal are only
// determined to ~eps ||T|| by its rounding).  e2 holds the squared
// off-diagonal.  w[t] receives the eigenvalue.
__device__ inline void multisect_eigs(const double* d, const double* e2, int n, int k, int t0, int tstride,
                                      int tcount, double lo0, double hi0, double pivmin, double atol, double* w) {
  const int lane = threadIdx.x & 31;
  const int ng = min(tcount, (k - t0 + tstride - 1) / tstride);   // eigenvalues of this warp
  if (ng <= 0) return;
  const int L = max(1, 32 / ng);
  const int gmax = 32 / L;                                  // groups per pass
  const double eps = 2.220446049250313e-16;
  for (int gb = 0; gb < ng; gb += gmax) {
    const int g = gb + lane / L, q = lane % L;
    const int t = t0 + g * tstride;
    const bool mine = (lane / L < gmax) && (g < ng) && (t < k);
    const int j = n - 1 - t;
    double lo = lo0, hi = hi0;
    bool done = !mine;
    for (int it = 0; it < 200; it++) {
      if (!__any_sync(0xffffffffu, !done)) break;
      const double x = lo + (hi - lo) * (double)(q + 1) / (double)(L + 1);
      bool above = false;   // more than j eigenvalues below x: eigenvalue j lies below x
      if (!done) above = sturm_count_sq(d, e2, n, x, pivmin) > j;
      const unsigned bal = __ballot_sync(0xffffffffu, above);
      if (!done) {
        const unsigned bits = (bal >> ((lane / L) * L)) & ((L == 32) ? 0xffffffffu : ((1u << L) - 1u));
        const int qs = bits ? (__ffs(bits) - 1) : L;        // first split point above eigenvalue j
        const double nlo = (qs == 0) ? lo : lo + (hi - lo) * (double)qs / (double)(L + 1);
        const double nhi = (qs == L) ? hi : lo + (hi - lo) * (double)(qs + 1) / (double)(L + 1);
        if (!(nlo > lo || nhi < hi)) done = true;           // no progress at this precision
        lo = nlo;
        hi = nhi;
        if (hi - lo <= fmax(2.0 * eps * fmax(fabs(lo), fabs(hi)), atol) + pivmin) done = true;
      }
    }
    if (mine && q == 0) w[t] = 0.5 * (lo + hi);
  }
  __syncwarp();
}

// a / b in double-float: an FP32 quotient corrected once with the exact
// remainder (~2^-46 relative).
__device__ __forceinline__ dfl df_div(dfl a, dfl b) {
  const float q1 = __fdividef(a.h, b.h);
  const dfl r = df_add(a, df_neg(df_mul(dfl{q1, 0.f}, b)));
  const float q2 = __fdividef(r.h, b.h);
  return df_fast2(q1, q2);
}
// sturm_count_sq in double-float: d and e^2 as (hi, lo) pairs, x converted once;
// pivmin in FP32 range.
__device__ inline int sturm_count_df(const dfl* d, const dfl* e2, int n, double x, float pivmin) {
  const dfl nx = df_neg(df_from(x));
  int cnt = 0;
  dfl q = df_add(d[0], nx);
  if (fabsf(q.h) < pivmin) q = dfl{-pivmin, 0.f};
  cnt += q.h < 0.f;
  for (int i = 1; i < n; i++) {
    q = df_add(df_add(d[i], nx), df_neg(df_div(e2[i - 1], q)));
    if (fabsf(q.h) < pivmin) q = dfl{-pivmin, 0.f};
    cnt += q.h < 0.f;
  }
  return cnt;
}
// multisect_eigs with the Sturm counts in double-float (FP32 pipes): the
// intervals stop at ~2^-44 of ||T|| (atol) or 2^-45 relative.  Meant for all the
// warps of a CTA at once (t0 = warp, tstride = warps), so each eigenvalue gets
// several lanes and rounds are few.
__device__ inline void multisect_eigs_df(const dfl* d, const dfl* e2, int n, int k, int t0, int tstride,
                                         double lo0, double hi0, float pivmin, double atol, double* w) {
  const int lane = threadIdx.x & 31;
  const int ng = (k - t0 + tstride - 1) / tstride;          // eigenvalues of this warp
  if (ng <= 0) return;
  const int L = max(1, 32 / ng);
  const int gmax = 32 / L;
  const double eps = 2.842170943040401e-14;                 // 2^-45
  for (int gb = 0; gb < ng; gb += gmax) {
    const int g = gb + lane / L, q = lane % L;
    const int t = t0 + g * tstride;
    const bool mine = (lane / L < gmax) && (g < ng) && (t < k);
    const int j = n - 1 - t;
    double lo = lo0, hi = hi0;
    bool done = !mine;
    for (int it = 0; it < 200; it++) {
      if (!__any_sync(0xffffffffu, !done)) break;
      const double x = lo + (hi - lo) * (double)(q + 1) / (double)(L + 1);
      bool above = false;
      if (!done) above = sturm_count_df(d, e2, n, x, pivmin) > j;
      const unsigned bal = __ballot_sync(0xffffffffu, above);
      if (!done) {
        const unsigned bits = (bal >> ((lane / L) * L)) & ((L == 32) ? 0xffffffffu : ((1u << L) - 1u));
        const int qs = bits ? (__ffs(bits) - 1) : L;
        const double nlo = (qs == 0) ? lo : lo + (hi - lo) * (double)qs / (double)(L + 1);
        const double nhi = (qs == L) ? hi : lo + (hi - lo) * (double)(qs + 1) / (double)(L + 1);
        if (!(nlo > lo || nhi < hi)) done = true;
        lo = nlo;
        hi = nhi;
        if (hi - lo <= fmax(2.0 * eps * fmax(fabs(lo), fabs(hi)), atol)) done = true;
      }
    }
    if (mine && q == 0) w[t] = 0.5 * (lo + hi);
  }
  __syncwarp();
}

// One solve (T - lam I) x = y by Gaussian elimination with partial pivoting on
// the tridiagonal; y is overwritten by x.  u0,u1,u2,mul: n doubles; piv: n ints.
__device__ inline void tri_factor(const double* d, const double* e, int n, double lam, double small,
                                  double* u0, double* u1, double* u2, double* mul, int* piv) {
  double wa = d[0] - lam, wb = (n > 1) ? e[0] : 0.0;     // working row (col i, col i+1)
  for (int i = 0; i + 1 < n; i++) {
    const double c = e[i], a1 = d[i + 1] - lam, b1 = (i + 2 < n) ? e[i + 1] : 0.0;
    if (fabs(wa) >= fabs(c)) {
      double a = wa;
      if (a == 0.0) a = small;
      u0[i] = a; u1[i] = wb; u2[i] = 0.0;
      const double m = c / a;
      mul[i] = m; piv[i] = 0;
      wa = a1 - m * wb;
      wb = b1;
    } else {
      u0[i] = c; u1[i] = a1; u2[i] = b1;
      const double m = wa / c;
      mul[i] = m; piv[i] = 1;
      const double na = wb - m * a1, nb = -m * b1;
      wa = na; wb = nb;
    }
  }
  u0[n - 1] = (wa == 0.0) ? small : wa;
}
__device__ inline void tri_solve(int n, const double* u0, const double* u1, const double* u2,
                                 const double* mul, const int* piv, double* y) {
  for (int i = 0; i + 1 < n; i++) {
    if (piv[i]) { const double t = y[i]; y[i] = y[i + 1]; y[i + 1] = t; }
    y[i + 1] -= mul[i] * y[i];
  }
  for (int i = n - 1; i >= 0; i--) {
    double s = y[i];
    if (i + 1 < n) s -= u1[i] * y[i + 1];
    if (i + 2 < n) s -= u2[i] * y[i + 2];
    y[i] = s / u0[i];
  }
}

// The same factorisation and solve for many shifts at once, one per lane of a
// warp: element i of a lane's arrays at [i * 32] from the lane's base pointer,
// so a warp's accesses are coalesced.  Branch-free, one division per row
// (the inverse pivot ui = 1 / u0 is kept), so the lanes do not diverge.
__device__ inline void tri_factor_lanes(const double* d, const double* e, int n, double lam, double small,
                                        double* ui, double* u1, double* u2, double* mul, int* piv) {
  double wa = d[0] - lam, wb = (n > 1) ? e[0] : 0.0;
  for (int i = 0; i + 1 < n; i++) {
    const double c = e[i], a1 = d[i + 1] - lam, b1 = (i + 2 < n) ? e[i + 1] : 0.0;
    const bool keep = fabs(wa) >= fabs(c);
    const double a = keep ? (wa == 0.0 ? small : wa) : c;
    const double inv = 1.0 / a;
    const double m = (keep ? c : wa) * inv;
    ui[32 * i] = inv;
    u1[32 * i] = keep ? wb : a1;
    u2[32 * i] = keep ? 0.0 : b1;
    mul[32 * i] = m;
    piv[32 * i] = keep ? 0 : 1;
    const double na = keep ? a1 - m * wb : wb - m * a1;
    wb = keep ? b1 : -m * b1;
    wa = na;
  }
  ui[32 * (n - 1)] = 1.0 / ((wa == 0.0) ? small : wa);
  u1[32 * (n - 1)] = 0.0;
  u2[32 * (n - 1)] = 0.0;
}
// y <- (T - lam I)^{-1} (sc y) for each lane's vector, returning |x|^2 of the
// result.  The element loads of each sweep are issued eight rows ahead of the
// recurrence (the arrays live in L2), so their latency is not paid per row.
__device__ inline double tri_solve_lanes(int n, double sc, const double* ui, const double* u1, const double* u2,
                                         const double* mul, const int* piv, double* y) {
  constexpr int U = 8;
  double cur = sc * y[0];
  int i = 0;
  for (; i + U < n; i += U) {
    double nx[U], mu[U];
    int pv[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      nx[u] = y[32 * (i + 1 + u)];
      mu[u] = mul[32 * (i + u)];
      pv[u] = piv[32 * (i + u)];
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
      const double v = sc * nx[u];
      const bool sw = pv[u] != 0;
      const double lo = sw ? v : cur, hi = sw ? cur : v;
      y[32 * (i + u)] = lo;
      cur = hi - mu[u] * lo;
    }
  }
  for (; i + 1 < n; i++) {
    const double v = sc * y[32 * (i + 1)];
    const bool sw = piv[32 * i] != 0;
    const double lo = sw ? v : cur, hi = sw ? cur : v;
    y[32 * i] = lo;
    cur = hi - mul[32 * i] * lo;
  }
  y[32 * (n - 1)] = cur;
  double y1 = 0.0, y2 = 0.0, nn = 0.0;   // x[i + 1], x[i + 2]
  i = n - 1;
  for (; i - U + 1 >= 0; i -= U) {
    double yv[U], a1[U], a2[U], iv[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      yv[u] = y[32 * (i - u)];
      a1[u] = u1[32 * (i - u)];
      a2[u] = u2[32 * (i - u)];
      iv[u] = ui[32 * (i - u)];
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
      const double x = (yv[u] - a1[u] * y1 - a2[u] * y2) * iv[u];
      y[32 * (i - u)] = x;
      nn += x * x;
      y2 = y1;
      y1 = x;
    }
  }
  for (; i >= 0; i--) {
    const double x = (y[32 * i] - u1[32 * i] * y1 - u2[32 * i] * y2) * ui[32 * i];
    y[32 * i] = x;
    nn += x * x;
    y2 = y1;
    y1 = x;
  }
  return nn;
}

// 1/a in double-float: the rounded FP32 reciprocal refined by one Newton step
// (the residual 1 - a_h r is exact in an FMA), ~47 bits.
__device__ __forceinline__ dfl df_rcp(dfl a) {
  const float r = 1.0f / a.h;
  float e = fmaf(-a.h, r, 1.0f);
  e = fmaf(-a.l, r, e);
  return df_fast2(r, r * e);
}
// tri_factor_lanes in double-float arithmetic (the mixed-form OSV build): d and e
// as (hi, lo) pairs, the factors stored as pairs in the same lane-interleaved
// slots, so the recurrence runs on the FP32 pipes.
__device__ inline void tri_factor_lanes_df(const dfl* d, const dfl* e, int n, dfl lam, float small, dfl* ui,
                                           dfl* u1, dfl* u2, dfl* mul, int* piv) {
  const dfl z{0.f, 0.f}, nl = df_neg(lam);
  dfl wa = df_add(d[0], nl), wb = (n > 1) ? e[0] : z;
  for (int i = 0; i + 1 < n; i++) {
    const dfl c = e[i], a1 = df_add(d[i + 1], nl), b1 = (i + 2 < n) ? e[i + 1] : z;
    const bool keep = fabsf(wa.h) >= fabsf(c.h);
    const dfl a = keep ? (wa.h == 0.f ? dfl{small, 0.f} : wa) : c;
    const dfl inv = df_rcp(a);
    const dfl m = df_mul(keep ? c : wa, inv);
    ui[32 * i] = inv;
    u1[32 * i] = keep ? wb : a1;
    u2[32 * i] = keep ? z : b1;
    mul[32 * i] = m;
    piv[32 * i] = keep ? 0 : 1;
    const dfl nm = df_neg(m);
    const dfl na = keep ? df_fma1(nm, wb, a1) : df_fma1(nm, a1, wb);
    wb = keep ? b1 : df_mul(nm, b1);
    wa = na;
  }
  ui[32 * (n - 1)] = df_rcp(wa.h == 0.f ? dfl{small, 0.f} : wa);
  u1[32 * (n - 1)] = z;
  u2[32 * (n - 1)] = z;
}
// tri_solve_lanes in double-float: y <- (T - lam I)^{-1} (sc y), returning max |x|
// (the next solve's scale; the vectors are normalised in FP64 afterwards).
__device__ inline float tri_solve_lanes_df(int n, float sc, const dfl* ui, const dfl* u1, const dfl* u2,
                                           const dfl* mul, const int* piv, dfl* y) {
  constexpr int U = 4;
  const dfl s{sc, 0.f};
  dfl cur = df_mul(y[0], s);
  int i = 0;
  for (; i + U < n; i += U) {
    dfl nx[U], mu[U];
    int pv[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      nx[u] = y[32 * (i + 1 + u)];
      mu[u] = mul[32 * (i + u)];
      pv[u] = piv[32 * (i + u)];
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
      const dfl v = df_mul(nx[u], s);
      const bool sw = pv[u] != 0;
      const dfl lo = sw ? v : cur, hi = sw ? cur : v;
      y[32 * (i + u)] = lo;
      cur = df_fma1(df_neg(mu[u]), lo, hi);
    }
  }
  for (; i + 1 < n; i++) {
    const dfl v = df_mul(y[32 * (i + 1)], s);
    const bool sw = piv[32 * i] != 0;
    const dfl lo = sw ? v : cur, hi = sw ? cur : v;
    y[32 * i] = lo;
    cur = df_fma1(df_neg(mul[32 * i]), lo, hi);
  }
  y[32 * (n - 1)] = cur;
  const dfl z{0.f, 0.f};
  dfl y1 = z, y2 = z;   // x[i + 1], x[i + 2]
  float amax = 0.f;
  i = n - 1;
  for (; i - U + 1 >= 0; i -= U) {
    dfl yv[U], a1[U], a2[U], iv[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      yv[u] = y[32 * (i - u)];
      a1[u] = u1[32 * (i - u)];
      a2[u] = u2[32 * (i - u)];
      iv[u] = ui[32 * (i - u)];
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
      const dfl x = df_mul(df_fma2(df_neg(a1[u]), y1, df_neg(a2[u]), y2, yv[u]), iv[u]);
      y[32 * (i - u)] = x;
      amax = fmaxf(amax, fabsf(x.h));
      y2 = y1;
      y1 = x;
    }
  }
  for (; i >= 0; i--) {
    const dfl x = df_mul(df_fma2(df_neg(u1[32 * i]), y1, df_neg(u2[32 * i]), y2, y[32 * i]), ui[32 * i]);
    y[32 * i] = x;
    amax = fmaxf(amax, fabsf(x.h));
    y2 = y1;
    y1 = x;
  }
  return amax;
}

}  // namespace osv
