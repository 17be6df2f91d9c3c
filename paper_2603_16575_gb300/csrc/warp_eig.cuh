// One-warp dense symmetric eigen-solvers (FP64 or FP32), used by the pair
// preconditioners (Eq. prec_eig): Householder tridiagonalisation, backward
// accumulation of Z, implicit QR with the Wilkinson shift (Golub & Van Loan,
// Matrix Computations, Alg. 8.3.2/8.3.3) with lane 0 chasing the bulge and all
// lanes rotating the rows of Z, and a warp GEMM.  All routines are called by
// every lane of one warp.
#pragma once
#include "common.cuh"

namespace osv {

constexpr int PW_MAXN = 192;         // largest order handled by the one-warp routines

template <class T>
struct WarpSmT {                     // per-warp shared scratch
  T v[PW_MAXN];
  T p[PW_MAXN];
  T d[PW_MAXN];
  T e[PW_MAXN];
  T cs[2 * PW_MAXN];
  int keep[PW_MAXN];
};
using WarpSm = WarpSmT<double>;

// C[MxN] (ld ldc) = alpha A B (+ beta C); lanes own columns, eight rows at a time.
template <class T, class VA, class VB>
__device__ void warp_gemm(int M, int N, int K, T alpha, const VA& A, const VB& B, T beta, T* C, int ldc) {
  const int lane = threadIdx.x & 31;
  for (int n0 = 0; n0 < N; n0 += 32) {
    const int n = n0 + lane;
    for (int m0 = 0; m0 < M; m0 += 8) {
      T acc[8];
#pragma unroll
      for (int i = 0; i < 8; i++) acc[i] = T(0);
      if (n < N)
        for (int k = 0; k < K; k++) {
          const T b = static_cast<T>(B.get(k, n));
#pragma unroll
          for (int i = 0; i < 8; i++)
            if (m0 + i < M) acc[i] = fma(static_cast<T>(A.get(m0 + i, k)), b, acc[i]);
        }
      if (n < N)
#pragma unroll
        for (int i = 0; i < 8; i++)
          if (m0 + i < M) {
            T* cp = C + (size_t)(m0 + i) * ldc + n;
            *cp = (beta == T(0) ? T(0) : beta * *cp) + alpha * acc[i];
          }
    }
  }
  __syncwarp();
}

// Householder tridiagonalisation (as cta_tridiag) with one warp.  p = tau A' v
// is formed column by column (A' symmetric): lanes own rows, no reductions.
template <class T>
__device__ void warp_tridiag(T* A, int n, int lda, T* d, T* e, T* tau, T* v, T* p) {
  const int lane = threadIdx.x & 31;
  for (int k = 0; k + 2 < n; k++) {
    const int L = n - k - 1;
    T* Ak = A + (size_t)(k + 1) * lda + (k + 1);
    T part = T(0.0);
    for (int t = lane; t < L; t += 32) {
      const T x = A[(size_t)(k + 1 + t) * lda + k];
      v[t] = x;
      if (t > 0) part += x * x;
    }
    const T sigma = warp_sum(part);
    __syncwarp();
    T tk = T(0.0), sc = T(0.0);
    if (lane == 0) {
      const T alpha = v[0];
      T beta = alpha;
      if (sigma > T(0.0)) {
        const T mu = sqrt(alpha * alpha + sigma);
        beta = alpha <= T(0.0) ? mu : -mu;
        tk = (beta - alpha) / beta;
        sc = T(1.0) / (alpha - beta);
      }
      d[k] = A[(size_t)k * lda + k];
      e[k] = beta;
      tau[k] = tk;
    }
    tk = __shfl_sync(0xffffffffu, tk, 0);
    sc = __shfl_sync(0xffffffffu, sc, 0);
    if (tk != T(0.0)) {
      for (int t = lane; t < L; t += 32) v[t] = (t == 0) ? T(1.0) : v[t] * sc;
      __syncwarp();
      for (int rb = 0; rb < L; rb += 128) {
        T acc[4] = {T(0.0), T(0.0), T(0.0), T(0.0)};
        for (int c = 0; c < L; c++) {
          const T vc = v[c];
          const T* row = Ak + (size_t)c * lda;
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
      T pv = T(0.0);
      for (int t = lane; t < L; t += 32) pv += p[t] * v[t];
      const T Kc = T(0.5) * tk * warp_sum(pv);
      for (int t = lane; t < L; t += 32) p[t] -= Kc * v[t];
      __syncwarp();
      for (int c = 0; c < L; c++) {
        T* row = Ak + (size_t)c * lda;
        const T vc = v[c], wc = p[c];
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
      if (n >= 3) tau[n - 2] = T(0.0);
    }
    d[n - 1] = A[(size_t)(n - 1) * lda + (n - 1)];
    tau[n - 1] = T(0.0);
  }
  __syncwarp();
}

// Z = H_0 ... H_{n-3} (row-major, ldz) by backward accumulation, one warp.
template <class T>
__device__ void warp_form_z(const T* A, int n, int lda, const T* tau, T* Z, int ldz, T* vs, T* y) {
  const int lane = threadIdx.x & 31;
  for (int r = 0; r < n; r++)
    for (int c = lane; c < n; c += 32) Z[(size_t)r * ldz + c] = (r == c) ? T(1.0) : T(0.0);
  __syncwarp();
  for (int k = n - 3; k >= 0; k--) {
    const T tk = tau[k];
    if (tk == T(0.0)) continue;
    const int L = n - k - 1;
    for (int r = lane; r < L; r += 32) vs[r] = (r == 0) ? T(1.0) : A[(size_t)(k + 1 + r) * lda + k];
    __syncwarp();
    for (int c = lane; c < L; c += 32) {
      T s = T(0.0);
      for (int r = 0; r < L; r++) s = fma(vs[r], Z[(size_t)(k + 1 + r) * ldz + (k + 1 + c)], s);
      y[c] = tk * s;
    }
    __syncwarp();
    for (int r = 0; r < L; r++) {
      const T vr = vs[r];
      T* zr = Z + (size_t)(k + 1 + r) * ldz + (k + 1);
      for (int c = lane; c < L; c += 32) zr[c] -= vr * y[c];
    }
    __syncwarp();
  }
}

// Implicit symmetric QR with the Wilkinson shift (as cta_tridiag_qr), lane 0
// chasing the bulge in shared memory, all lanes rotating the rows of Z.
template <class T>
__device__ int warp_tridiag_qr(T* d, T* e, int n, T* Z, int ldz, T* cs) {
  const int lane = threadIdx.x & 31;
  const T eps = (sizeof(T) == 8) ? T(2.220446049250313e-16) : T(1.1920929e-07);
  const int max_sweeps = 40 * n + 100;
  for (int sweeps = 0;; sweeps++) {
    int l = 0, h = 0, done = 0;
    if (lane == 0) {
      h = n - 1;
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
        const T delta = T(0.5) * (d[h - 1] - d[h]);
        const T eh = e[h - 1];
        const T den = delta + copysign(sqrt(delta * delta + eh * eh), delta);
        const T mu = d[h] - (den != T(0.0) ? eh * eh / den : T(0.0));
        T x = d[l] - mu, z = e[l];
        for (int k = l; k < h; k++) {
          const T rr = sqrt(x * x + z * z);
          T c = T(1.0), s = T(0.0);
          if (rr != T(0.0)) {
            const T inv = T(1.0) / rr;
            c = x * inv;
            s = z * inv;
          }
          if (k > l) e[k - 1] = rr;
          const T a = d[k], b = e[k], cc = d[k + 1];
          const T cs2 = c * s, c2 = c * c, s2 = s * s;
          d[k] = c2 * a + T(2.0) * cs2 * b + s2 * cc;
          d[k + 1] = s2 * a - T(2.0) * cs2 * b + c2 * cc;
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
      T* zr = Z + (size_t)row * ldz;
      T carry = zr[l];
      for (int k = l; k < h; k++) {
        const T c = cs[2 * k], s = cs[2 * k + 1];
        const T y = zr[k + 1];
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
template <class T>
__device__ int warp_syev(T* A, int n, T* w, T* Z, T* tau, WarpSmT<T>& ws) {
  const int lane = threadIdx.x & 31;
  if (n == 1) {
    if (lane == 0) { w[0] = A[0]; Z[0] = T(1.0); }
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

}  // namespace osv
