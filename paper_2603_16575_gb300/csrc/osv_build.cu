// A0: OSV generation.  T_ii from the RI integrals (Eq. mp2_tkk, positive
// denominator e_a + e_b - 2 f_ii), its eigen-decomposition (Eq. osv_gen; FP64, or
// double-float for the mixed form)
// and the selection omega >= l_osv of Algorithm 3, all on the GPU.
#include <algorithm>

#include "eig.cuh"
#include "internal.h"

namespace osv {

// A(a, P) = B[i,a,P] and its transpose, read straight from the source (stored
// or regenerated).
struct BiRows {
  BSrc s;
  int i;
  __device__ __forceinline__ double get(int a, int P) const { return s.get(i, a, P); }
};
struct BiCols {
  BSrc s;
  int i;
  __device__ __forceinline__ double get(int P, int b) const { return s.get(i, b, P); }
};

// One 64x64 tile (tr >= tc) of T_i = (B_i B_i^T) / (e_a + e_b - 2 f_ii); the
// mirror tile is written from the same accumulators.
__global__ void __launch_bounds__(NT) k_tii(BSrc src, const double* __restrict__ e_vir,
                                            const double* __restrict__ f_occ, int n_occ, int i0,
                                            double* __restrict__ T) {
  __shared__ double sm[GEMM_SMEM_DOUBLES];
  const int nv = src.n_vir, nx = src.n_aux;
  const int b = blockIdx.y, i = i0 + b;
  int t = blockIdx.x, tr = 0;
  while ((tr + 1) * (tr + 2) / 2 <= t) tr++;
  const int tc = t - tr * (tr + 1) / 2;
  double acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; u++)
#pragma unroll
    for (int v = 0; v < 4; v++) acc[u][v] = 0.0;
  tile_mma(nv, nv, nx, tr * TM, tc * TN, BiRows{src, i}, BiCols{src, i}, acc, sm);
  const double f2 = 2.0 * f_occ[(size_t)i * n_occ + i];
  double* Ti = T + (size_t)b * nv * nv;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int u = 0; u < 4; u++)
#pragma unroll
    for (int v = 0; v < 4; v++) {
      const int a = tr * TM + ty + 16 * u, c = tc * TN + tx + 16 * v;
      if (a < nv && c < nv) {
        const double val = acc[u][v] / (e_vir[a] + e_vir[c] - f2);
        Ti[(size_t)a * nv + c] = val;
        Ti[(size_t)c * nv + a] = val;
      }
    }
}

void launch_tii(const BSrc& src, const double* e_vir, const double* f_occ, int n_occ, int i0, int nb,
                double* T, cudaStream_t st) {
  const int nt = (src.n_vir + TM - 1) / TM;
  dim3 grid(nt * (nt + 1) / 2, nb);
  k_tii<<<grid, NT, 0, st>>>(src, e_vir, f_occ, n_occ, i0, T);
  note_launch(1);
}

// ---------------------------------------------------------------- eigen
constexpr int ZSMEM_MAX = 160;   // Z kept in shared memory up to this order
constexpr int NT_EIG = 1024;     // threads of the OSV eigen kernel (more loads in flight)
constexpr int INV_GROUPS = 4;    // warps running the lane-batched inverse iteration (176 n doubles each)
constexpr int EB_DF_MAXN = 1536; // double-float back-transformation: the vector in registers up to this order

// Sign eigenvector t (V[t][0..n), eigenvector-major) so that its largest-magnitude
// entry (lowest index on ties) is positive.  One warp per vector.
__device__ inline void sign_vectors(double* V, int n, int k) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int t = warp; t < k; t += NT_EIG / 32) {
    double* x = V + (size_t)t * n;
    double best = -1.0;
    int bi = 0x7fffffff;
    for (int r = lane; r < n; r += 32) {
      const double a = fabs(x[r]);
      if (a > best) { best = a; bi = r; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (x[bi] < 0.0)
      for (int r = lane; r < n; r += 32) x[r] = -x[r];
  }
  __syncthreads();
}

// Full decomposition path (n <= ZSMEM_MAX with Z in shared memory, or any n
// with Z in global scratch): eigenvalues sorted descending, then selection.
// zcm: Z column-major (eigenvector-major), for Z in global memory, where the rotations of the
// QR sweeps then touch contiguous columns; row-major otherwise (Z in shared memory).
// ntw (zcm only): warps of tiles after the 4 n + 64 doubles of sm for the fused sweep, whose
// partial sums go to V (written only at the end); 0 for the plain tridiagonalisation.
__device__ void eig_full_select(double* A, int n, double thr, int kmax, double* V, double* w, int* kout,
                                double* scr, int* err, double* Zs, int ldz, double* sm, bool zcm, int ntw = 0) {
  double* e = scr;
  double* tau = scr + n;
  double* ww = scr + 2 * n;
  const int nbt = (n - 1 + 31) / 32;
  if ((size_t)nbt * (nbt + 1) / 2 * 64 > (size_t)kmax * n) ntw = 0;   // the partial sums must fit V
  int rc = zcm ? cta_syev_cm_rec<NT_EIG>(A, n, ww, Zs, ldz, e, tau, sm, ntw, V)
               : cta_syev<NT_EIG>(A, n, n, ww, Zs, ldz, e, tau, sm);
  __shared__ int s_k;
  int* perm = reinterpret_cast<int*>(sm);   // sm reused: n ints (n <= 4n doubles)
  if (threadIdx.x == 0) {
    for (int t = 0; t < n; t++) perm[t] = t;
    for (int t = 1; t < n; t++) {           // insertion sort, descending, stable
      const int pv = perm[t];
      const double x = ww[pv];
      int u = t - 1;
      while (u >= 0 && ww[perm[u]] < x) { perm[u + 1] = perm[u]; u--; }
      perm[u + 1] = pv;
    }
    int k = 0;
    if (thr > 0.0) { while (k < n && ww[perm[k]] >= thr) k++; }
    else k = n;
    if (k > kmax) { k = kmax; atomicOr(err, ERR_SIZE); }
    bool bad = rc != 0;
    for (int t = 0; t < n; t++) bad |= !isfinite(ww[t]);
    if (bad) atomicOr(err, rc ? ERR_EIG : ERR_NONFINITE);
    s_k = k;
    *kout = k;
    for (int t = 0; t < k; t++) w[t] = ww[perm[t]];
  }
  __syncthreads();
  const int k = s_k;
  for (int idx = threadIdx.x; idx < n * k; idx += NT_EIG) {
    const int t = idx / n, r = idx % n;
    V[(size_t)t * n + r] = zcm ? Zs[(size_t)perm[t] * ldz + r] : Zs[(size_t)r * ldz + perm[t]];
  }
  __syncthreads();
  sign_vectors(V, n, k);
}

// Eigenpairs with eigenvalue >= thr only: tridiagonalise, count by Sturm
// sequence, multisection for the kept eigenvalues, inverse iteration with
// Gram-Schmidt inside clusters of close eigenvalues, back-transformation.
__device__ void eig_topk(double* A, int n, double thr, int kmax, double* V, double* w, int* kout,
                         double* scr, int* err, double* sm, int ntw, int dfl_tridiag) {
  double* d = scr;
  double* e = scr + n;
  double* tau = scr + 2 * n;
  double* v = sm;
  double* p = sm + n;
  double* red = sm + 2 * n;
  __shared__ int s_k, s_nclu;
  __shared__ double s_lo, s_hi, s_piv, s_norm;
  if (ntw >= 2 && dfl_tridiag)
    cta_tridiag_sym_df<NT_EIG>(A, n, n, d, e, tau, sm, ntw, scr + 3 * n, n <= EB_DF_MAXN);   // partial sums in the Z room
  else if (ntw >= 2)
    cta_tridiag_sym<NT_EIG>(A, n, n, d, e, tau, sm, ntw, scr + 3 * n);
  else cta_tridiag_col<NT_EIG>(A, n, n, d, e, tau, v, p, red);
  // Gershgorin bounds and a pivot floor
  double glo = 1e300, ghi = -1e300, nrm = 0.0, emax = 0.0;
  for (int t = threadIdx.x; t < n; t += NT_EIG) {
    const double off = (t > 0 ? fabs(e[t - 1]) : 0.0) + (t + 1 < n ? fabs(e[t]) : 0.0);
    glo = fmin(glo, d[t] - off);
    ghi = fmax(ghi, d[t] + off);
    nrm = fmax(nrm, fabs(d[t]) + off);
    if (t + 1 < n) emax = fmax(emax, e[t] * e[t]);
  }
  glo = -cta_max(-glo, red);
  ghi = cta_max(ghi, red);
  nrm = cta_max(nrm, red);
  emax = cta_max(emax, red);
  int* clu = reinterpret_cast<int*>(p);     // cluster starts (reuses p)
  if (threadIdx.x == 0) {
    const double piv = 1e-290 * fmax(1.0, emax);
    const double span = ghi - glo;
    s_lo = glo - 1e-14 * span - piv;
    s_hi = ghi + 1e-14 * span + piv;
    s_piv = piv;
    s_norm = nrm;
    int k = n - sturm_count(d, e, n, thr, piv);
    if (k > kmax) { k = kmax; atomicOr(err, ERR_SIZE); }
    s_k = k;
    *kout = k;
  }
  __syncthreads();
  const int k = s_k;
  // kept eigenvalues by multisection: warps 0-3 (one per SM sub-partition, whose
  // FP64 pipes work in parallel), several lanes per eigenvalue
  // (shared copies of d and e^2)
  double* ds = p;
  double* e2s = v;
  for (int t = threadIdx.x; t < n; t += NT_EIG) {
    ds[t] = d[t];
    e2s[t] = (t + 1 < n) ? e[t] * e[t] : 0.0;
  }
  __syncthreads();
  // Many kept eigenvalues (k >= 64): whole warps of one eigenvalue per lane (pure
  // bisection, the fewest Sturm counts), so fewer warp instructions feed the FP64
  // pipe; otherwise four warps, several lanes per eigenvalue.  The mixed-form
  // build counts in double-float on every warp (its tridiagonal is double-float).
  const double atol = 4.0 * 2.220446049250313e-16 * s_norm;
  if (dfl_tridiag) {
    dfl* dd = reinterpret_cast<dfl*>(ds);
    dfl* de = reinterpret_cast<dfl*>(e2s);
    for (int t = threadIdx.x; t < n; t += NT_EIG) {
      dd[t] = df_from(ds[t]);
      de[t] = df_from(e2s[t]);
    }
    __syncthreads();
    const float pivf = 1e-30f * (float)fmax(1.0, emax);
    multisect_eigs_df(dd, de, n, k, threadIdx.x >> 5, NT_EIG / 32, s_lo, s_hi, pivf, 5.7e-14 * s_norm, w);
  } else if (k >= 64) {
    const int wv = threadIdx.x >> 5;
    if (32 * wv < k) multisect_eigs(ds, e2s, n, k, 32 * wv, 1, 32, s_lo, s_hi, s_piv, atol, w);
  } else if ((threadIdx.x >> 5) < 4) {
    multisect_eigs(ds, e2s, n, k, threadIdx.x >> 5, 4, k, s_lo, s_hi, s_piv, atol, w);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double ortol = 1e-3 * s_norm;
    int nc = 0;
    for (int t = 0; t < k; t++)
      if (t == 0 || w[t - 1] - w[t] > ortol) clu[nc++] = t;
    clu[nc] = k;
    s_nclu = nc;
    for (int t = 0; t < k; t++)
      if (!isfinite(w[t])) atomicOr(err, ERR_NONFINITE);
  }
  __syncthreads();
  // inverse iteration, parallel over the kept vectors, one vector per LANE
  // (lane-interleaved factorisations, so every instruction of a warp works for 32
  // vectors): two solves from a seeded start, Gram-Schmidt inside each cluster of
  // close eigenvalues (FP64: a warp per cluster; mixed form: the whole CTA per
  // cluster, below), then one more
  // solve per vector and the Gram-Schmidt again.  With shifts accurate to
  // ~eps ||T||, one solve leaves a vector contaminated by an eigenvector at
  // distance g at ~eps ||T|| / g, so the vectors separate without
  // orthogonalising between every solve; the passes take care of
  // (near-)degenerate groups.  Warps 0-3 (one per SM sub-partition) take the
  // groups of 32 vectors; group slot w uses 176 n doubles of the scratch from
  // scr + 3n (the tridiagonalisation's partial sums are no longer needed).
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double small = 2.220446049250313e-16 * fmax(s_norm, 1e-300);
  // The mixed-form build solves in double-float arithmetic (FP32 pipes; its
  // tridiagonal carries ~48 bits): d and e (and the Gram-Schmidt dots) as pairs in
  // the tridiagonalisation's tile room, when it holds them and the scales stay
  // well inside FP32 range.
  const bool inv_df = dfl_tridiag && ntw >= 2 && 2 * n + k <= ntw * 16 * 33 && s_norm > 1e-12 && s_norm < 1e12;
  dfl* ddf = reinterpret_cast<dfl*>(sm + 4 * n + 64);
  dfl* edf = ddf + n;
  dfl* Vd = reinterpret_cast<dfl*>(scr + 3 * n + eig_osv_work_doubles(n));   // kept vectors, pairs [k][n]
  dfl* gsd = edf + n;                                                          // -dots of one Gram-Schmidt step [k]
  if (inv_df) {
    for (int t = threadIdx.x; t < n; t += NT_EIG) {
      ddf[t] = df_from(d[t]);
      edf[t] = (t + 1 < n) ? df_from(e[t]) : dfl{0.f, 0.f};
    }
    __syncthreads();
  }
  for (int pass = 0; pass < 2; pass++) {
    if (inv_df && warp < INV_GROUPS) {
      double* base = scr + 3 * n + (size_t)warp * 176 * n;
      dfl* ui = reinterpret_cast<dfl*>(base) + lane;
      dfl* u1 = reinterpret_cast<dfl*>(base + 32 * (size_t)n) + lane;
      dfl* u2 = reinterpret_cast<dfl*>(base + 64 * (size_t)n) + lane;
      dfl* mul = reinterpret_cast<dfl*>(base + 96 * (size_t)n) + lane;
      dfl* y = reinterpret_cast<dfl*>(base + 128 * (size_t)n) + lane;
      int* piv = reinterpret_cast<int*>(base + 160 * (size_t)n) + lane;
      for (int g = warp; 32 * g < k; g += INV_GROUPS) {
        const int t = 32 * g + lane;
        if (t < k) {
          if (pass == 0 || k > 32 * INV_GROUPS)
            tri_factor_lanes_df(ddf, edf, n, df_from(w[t]), (float)small, ui, u1, u2, mul, piv);
          if (pass == 0) {
#pragma unroll 4
            for (int r = 0; r < n; r++) {
              const uint64_t h = draw(0x5eedull + (uint64_t)t, (uint64_t)r);
              y[32 * r] = dfl{(float)(uint32_t)(h >> 40) * 0x1p-24f - 0.5f, 0.f};
            }
          } else {
#pragma unroll 4
            for (int r = 0; r < n; r++) y[32 * r] = Vd[(size_t)t * n + r];
          }
          float sc = 1.f;   // scale of the previous solve, applied on the next read
          for (int it = 0; it < 2 - pass; it++) {
            const float am = tri_solve_lanes_df(n, sc, ui, u1, u2, mul, piv, y);
            sc = am > 0.f ? 1.f / am : 0.f;
          }
          const dfl s{sc, 0.f};
#pragma unroll 4
          for (int r = 0; r < n; r++) Vd[(size_t)t * n + r] = df_mul(y[32 * r], s);
        }
      }
    } else if (warp < INV_GROUPS) {
      double* base = scr + 3 * n + (size_t)warp * 176 * n;
      double* ui = base + lane;
      double* u1 = base + 32 * (size_t)n + lane;
      double* u2 = base + 64 * (size_t)n + lane;
      double* mul = base + 96 * (size_t)n + lane;
      double* y = base + 128 * (size_t)n + lane;
      int* piv = reinterpret_cast<int*>(base + 160 * (size_t)n) + lane;
      for (int g = warp; 32 * g < k; g += INV_GROUPS) {
        const int t = 32 * g + lane;
        if (t < k) {
          // the second pass reuses the first pass's factorisation when every group kept its slot
          if (pass == 0 || k > 32 * INV_GROUPS) tri_factor_lanes(d, e, n, w[t], small, ui, u1, u2, mul, piv);
          if (pass == 0) {
#pragma unroll 4
            for (int r = 0; r < n; r++) {
              const uint64_t h = draw(0x5eedull + (uint64_t)t, (uint64_t)r);
              y[32 * r] = (double)(h >> 11) * 0x1p-53 - 0.5;
            }
          } else {
#pragma unroll 8
            for (int r = 0; r < n; r++) y[32 * r] = V[(size_t)t * n + r];
          }
          double sc = 1.0;   // normalisation of the previous solve, applied on the next read
          for (int it = 0; it < 2 - pass; it++) {
            const double nn = tri_solve_lanes(n, sc, ui, u1, u2, mul, piv, y);
            sc = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
          }
#pragma unroll 8
          for (int r = 0; r < n; r++) V[(size_t)t * n + r] = sc * y[32 * r];
        }
      }
    }
    __syncthreads();
    if (inv_df) {
      // Mixed form: the clusters one after another with the whole CTA, each vector
      // orthogonalised against the earlier ones of its cluster by classical
      // Gram-Schmidt applied twice (the dots one warp each, the update one thread
      // per row), so the loads of a cluster's vectors overlap instead of one warp
      // waiting on each in turn.  Double-float arithmetic on the pairs in Vd.
      float* redf = reinterpret_cast<float*>(red);
      for (int c = 0; c < s_nclu; c++) {
        const int t0 = clu[c], t1 = clu[c + 1];
        for (int t = t0; t < t1; t++) {
          dfl* Vt = Vd + (size_t)t * n;
          for (int rep = 0; rep < 2 && t > t0; rep++) {
            for (int q = t0 + warp; q < t; q += NT_EIG / 32) {
              const dfl* Vq = Vd + (size_t)q * n;
              float dh = 0.f, dl = 0.f;
              for (int r0 = lane; r0 < n; r0 += 32 * 4) {
                dfl x[4], y2[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                  const int r = r0 + 32 * u;
                  x[u] = r < n ? Vt[r] : dfl{0.f, 0.f};
                  y2[u] = r < n ? Vq[r] : dfl{0.f, 0.f};
                }
#pragma unroll
                for (int u = 0; u < 4; u++) df_acc(dh, dl, x[u], y2[u]);
              }
              dfl dot = df_norm(dh, dl);
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) dot = df_add(dot, df_shfl_xor(dot, o));
              if (lane == 0) gsd[q - t0] = df_neg(dot);
            }
            __syncthreads();
            for (int r = threadIdx.x; r < n; r += NT_EIG) {
              dfl acc = Vt[r];
              int q = t0;
              for (; q + 4 <= t; q += 4) {
                dfl vq[4];
#pragma unroll
                for (int u = 0; u < 4; u++) vq[u] = Vd[(size_t)(q + u) * n + r];
#pragma unroll
                for (int u = 0; u < 4; u++) acc = df_fma1(gsd[q + u - t0], vq[u], acc);
              }
              for (; q < t; q++) acc = df_fma1(gsd[q - t0], Vd[(size_t)q * n + r], acc);
              Vt[r] = acc;
            }
            __syncthreads();
          }
          float nh = 0.f, nl = 0.f;
          for (int r = threadIdx.x; r < n; r += NT_EIG) df_acc(nh, nl, Vt[r], Vt[r]);
          const double nnd = df_to(cta_sum_df(df_norm(nh, nl), redf));
          const dfl sc = df_from(nnd > 0.0 ? 1.0 / sqrt(nnd) : 0.0);
          for (int r = threadIdx.x; r < n; r += NT_EIG) Vt[r] = df_mul(Vt[r], sc);
          __syncthreads();
        }
      }
    }
    for (int c = warp; !inv_df && c < s_nclu; c += NT_EIG / 32) {   // Gram-Schmidt within clusters
      const int t0 = clu[c], t1 = clu[c + 1];
      for (int t = t0; t < t1; t++) {
        double* Vt = V + (size_t)t * n;
        for (int s = t0; s < t; s++) {
          const double* Vs = V + (size_t)s * n;
          double dot = 0.0;
          for (int r = lane; r < n; r += 32) dot += Vt[r] * Vs[r];
          dot = warp_sum(dot);
          for (int r = lane; r < n; r += 32) Vt[r] -= dot * Vs[r];
          __syncwarp();
        }
        double nn = 0.0;
        for (int r = lane; r < n; r += 32) nn += Vt[r] * Vt[r];
        nn = warp_sum(nn);
        const double sc = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
        for (int r = lane; r < n; r += 32) Vt[r] *= sc;
        __syncwarp();
      }
    }
    __syncthreads();
  }
  if (inv_df) {   // the kept vectors to FP64
    for (size_t idx = threadIdx.x; idx < (size_t)k * n; idx += NT_EIG) V[idx] = df_to(Vd[idx]);
    __syncthreads();
  }
  // the back-transformation to the virtual basis is k_eig_back
}

// Back-transformation of the kept eigenvectors of eig_topk, one warp per
// (orbital, vector) over the whole GPU (the vectors are independent, and
// orbitals keep different numbers of them): x <- H_0 ... H_{n-3} x with the
// reflectors stored contiguously in the rows of A and tau in the scratch, then
// the sign convention of sign_vectors.
constexpr int EB_WARPS = 8;

// The same back-transformation in double-float for the mixed-form build (its
// reflectors are stored as (hi, lo) pairs by cta_tridiag_sym_df): the vector
// lives in registers, NJ elements per lane (n <= 32 NJ), and every reflector
// costs FP32 instructions only.
template <int NJ>
__global__ void __launch_bounds__(EB_WARPS * 32) k_eig_back_df(const double* T, int n, int kmax, double* V,
                                                              const int* kout, const double* scratch,
                                                              size_t scr_stride) {
  __shared__ dfl s_tau[EB_DF_MAXN];   // tau as pairs: no global load or FP64 work per reflector
  const int b = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.y * EB_WARPS + warp;
  const int kb = kout[b];
  if ((int)blockIdx.y * EB_WARPS >= kb) return;   // CTA-uniform
  const double* tau = scratch + (size_t)b * scr_stride + 2 * n;
  for (int i = threadIdx.x; i < n; i += EB_WARPS * 32) s_tau[i] = df_from(tau[i]);
  __syncthreads();
  if (t >= kb) return;   // warp-uniform
  const dfl* Ad = reinterpret_cast<const dfl*>(T + (size_t)b * n * n);
  double* x = V + (size_t)b * n * kmax + (size_t)t * n;
  dfl xr[NJ];
#pragma unroll
  for (int j = 0; j < NJ; j++) {
    const int r = 32 * j + lane;
    xr[j] = r < n ? df_from(x[r]) : dfl{0.f, 0.f};
  }
  for (int kk = n - 3; kk >= 0; kk--) {
    const dfl tk = s_tau[kk];
    if (tk.h == 0.f) continue;
    const dfl* vr = Ad + (size_t)kk * n;   // v at columns kk+1 .. n-1 of row kk
    const int j0 = (kk + 1) >> 5;          // register blocks below j0 hold no row > kk
    float sh = 0.f, sl = 0.f;
#pragma unroll
    for (int j = 0; j < NJ; j++) {
      if (j < j0) continue;   // warp-uniform
      const int r = 32 * j + lane;
      if (r > kk && r < n) df_acc(sh, sl, vr[r], xr[j]);
    }
    dfl s = df_norm(sh, sl);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = df_add(s, df_shfl_xor(s, o));
    const dfl ns = df_neg(df_mul(s, tk));
#pragma unroll
    for (int j = 0; j < NJ; j++) {
      if (j < j0) continue;
      const int r = 32 * j + lane;
      if (r > kk && r < n) xr[j] = df_fma1(ns, vr[r], xr[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < NJ; j++) {
    const int r = 32 * j + lane;
    if (r < n) x[r] = df_to(xr[j]);
  }
  __syncwarp();
  double best = -1.0;
  int bi = 0x7fffffff;
  for (int r = lane; r < n; r += 32) {
    const double a = fabs(x[r]);
    if (a > best) { best = a; bi = r; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  if (x[bi] < 0.0)
    for (int r = lane; r < n; r += 32) x[r] = -x[r];
}
__global__ void __launch_bounds__(EB_WARPS * 32) k_eig_back(const double* T, int n, int kmax, double* V,
                                                           const int* kout, const double* scratch,
                                                           size_t scr_stride) {
  const int b = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.y * EB_WARPS + warp;
  if (t >= kout[b]) return;   // warp-uniform
  const double* A = T + (size_t)b * n * n;
  const double* tau = scratch + (size_t)b * scr_stride + 2 * n;
  double* x = V + (size_t)b * n * kmax + (size_t)t * n;
  for (int kk = n - 3; kk >= 0; kk--) {
    const double tk = tau[kk];
    if (tk == 0.0) continue;
    const int L = n - kk - 1;
    const double* vr = A + (size_t)kk * n + kk + 1;
    double* xs = x + kk + 1;
    double s = 0.0;
    for (int r = lane; r < L; r += 32) s = fma(vr[r], xs[r], s);
    s = tk * warp_sum(s);
    for (int r = lane; r < L; r += 32) xs[r] = fma(-vr[r], s, xs[r]);
    __syncwarp();
  }
  double best = -1.0;
  int bi = 0x7fffffff;
  for (int r = lane; r < n; r += 32) {
    const double a = fabs(x[r]);
    if (a > best) { best = a; bi = r; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  if (x[bi] < 0.0)
    for (int r = lane; r < n; r += 32) x[r] = -x[r];
}

__global__ void __launch_bounds__(NT_EIG) k_eig_osv(double* T, int nv, double thr, int kmax, double* V, double* w,
                                                int* kout, double* scratch, int* err, int zsmem, int ntw,
                                                int dfl_tridiag) {
  extern __shared__ double dyn[];
  const int b = blockIdx.x;
  double* A = T + (size_t)b * nv * nv;
  double* Vb = V + (size_t)b * nv * kmax;
  double* wb = w + (size_t)b * kmax;
  double* scr = scratch + (size_t)b * eig_osv_scratch_doubles(nv, kmax);
  if (zsmem) {
    const int ldz = nv + 1;
    double* Zs = dyn;
    double* sm = dyn + (size_t)nv * ldz;
    eig_full_select(A, nv, thr, kmax, Vb, wb, kout + b, scr, err, Zs, ldz, sm, false);
  } else if (thr > 0.0) {
    eig_topk(A, nv, thr, kmax, Vb, wb, kout + b, scr, err, dyn, ntw, dfl_tridiag);
  } else {
    double* Zg = scr + 3 * nv;
    eig_full_select(A, nv, thr, kmax, Vb, wb, kout + b, scr, err, Zg, nv, dyn, true, ntw);
  }
}

// Warps of rows x 33-double staging tiles in the shared memory of the top-k path's
// symmetric tridiagonalisation (0 when fewer than two fit): 32 rows in FP64, 16 in
// double-float (whose sweep stages each tile in two halves).
static int eig_tile_rows(bool dfl_tridiag) { return dfl_tridiag ? 16 : 32; }
static int eig_tile_warps(int nv, double thr, int rows) {
  (void)thr;   // the top-k path and the full path with Z in global memory both sweep in tiles
  if (nv <= ZSMEM_MAX) return 0;
  const size_t cap = (size_t)224 * 1024 / sizeof(double), base = (size_t)4 * nv + 64, tile = (size_t)rows * 33;
  const int ntw = cap > base ? (int)std::min<size_t>(NT_EIG / 32, (cap - base) / tile) : 0;
  return ntw >= 2 ? ntw : 0;
}

void launch_eig_osv(double* T, int nb, int nv, double thr, int kmax, double* V, double* w, int* k,
                    double* scratch, int* err, bool dfl_tridiag, cudaStream_t st) {
  const int zsmem = nv <= ZSMEM_MAX;
  size_t smem = (size_t)(4 * nv + 64) * sizeof(double);
  // the full path (thr <= 0) sweeps in FP64 tiles whatever dfl_tridiag says
  const int rows = (thr > 0.0) ? eig_tile_rows(dfl_tridiag) : eig_tile_rows(false);
  const int ntw = eig_tile_warps(nv, thr, rows);
  if (zsmem) smem += (size_t)nv * (nv + 1) * sizeof(double);
  else if (ntw >= 2) smem += (size_t)ntw * rows * 33 * sizeof(double);
  cudaFuncSetAttribute(k_eig_osv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_eig_osv<<<nb, NT_EIG, smem, st>>>(T, nv, thr, kmax, V, w, k, scratch, err, zsmem, ntw, dfl_tridiag ? 1 : 0);
  note_launch(1);
}

void launch_eig_back(double* T, int nb, int nv, double thr, int kmax, double* V, const int* k, double* scratch,
                     bool dfl_tridiag, cudaStream_t st) {
  if (nv <= ZSMEM_MAX || !(thr > 0.0)) return;   // the other paths form the eigenvectors in k_eig_osv
  const int ntw = eig_tile_warps(nv, thr, eig_tile_rows(dfl_tridiag));
  dim3 grid(nb, (std::min(kmax, nv) + EB_WARPS - 1) / EB_WARPS);
  const size_t ss = eig_osv_scratch_doubles(nv, kmax);
  if (dfl_tridiag && ntw >= 2 && nv <= EB_DF_MAXN) {   // reflectors stored as pairs
    if (nv <= 640) k_eig_back_df<20><<<grid, EB_WARPS * 32, 0, st>>>(T, nv, kmax, V, k, scratch, ss);
    else if (nv <= 1280) k_eig_back_df<40><<<grid, EB_WARPS * 32, 0, st>>>(T, nv, kmax, V, k, scratch, ss);
    else k_eig_back_df<48><<<grid, EB_WARPS * 32, 0, st>>>(T, nv, kmax, V, k, scratch, ss);
  } else {
    k_eig_back<<<grid, EB_WARPS * 32, 0, st>>>(T, nv, kmax, V, k, scratch, ss);
  }
  note_launch(1);
}

__global__ void k_pack_q(const double* V, const double* w, int nv, int kmax, const int* k,
                         double* const* Qdst, double* const* wdst) {
  const int b = blockIdx.y;
  const int kb = k[b];
  const double* Vb = V + (size_t)b * nv * kmax;
  double* Q = Qdst[b];
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nv * kb; idx += gridDim.x * blockDim.x) {
    const int r = idx / kb, t = idx % kb;
    Q[idx] = Vb[(size_t)t * nv + r];
  }
  if (blockIdx.x == 0)
    for (int t = threadIdx.x; t < kb; t += blockDim.x) wdst[b][t] = w[(size_t)b * kmax + t];
}

void launch_pack_q(const double* V, const double* w, int nb, int nv, int kmax, const int* k,
                   double* const* Qdst, double* const* wdst, cudaStream_t st) {
  dim3 grid(32, nb);
  k_pack_q<<<grid, 256, 0, st>>>(V, w, nv, kmax, k, Qdst, wdst);
  note_launch(1);
}

}  // namespace osv
