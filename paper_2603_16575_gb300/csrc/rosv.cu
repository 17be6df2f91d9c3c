// Randomized OSV generation (Algorithm 3; Eqs. rsvd_z, tsub, tii_rsvd, back_q,
// rsvd_za), per orbital batch, replacing the full eigen-decomposition of T_ii:
//   Ybar = [G; Gbar] T_ii      r + n_max Gaussian rows (counter-based draws)
//   range finder              rows of Ybar taken in order, each orthogonalised
//                             against Z (Eq. rsvd_za), until the r look-ahead
//                             rows all have norm <= l_osv / (10 sqrt(2/pi))
//   T~ = Z T_ii               (Eq. tsub)
//   T~ = Q~ omega V~^T        (Eq. tii_rsvd) through the eigen-decomposition of
//                             T~ T~^T (omega^2, Q~)
//   Q = Z^T Q~                (Eq. back_q), kept where omega >= l_osv
// The two GEMMs run in FP64 (FP64 form) or as split-TF32 tensor-core
// contractions with FP64 results (mixed form); the range finder and the small
// eigen-decomposition are FP64 in both.
#include "internal.h"
#include "eig.cuh"
#include "tc_tf32x3.cuh"

namespace osv {

__device__ __forceinline__ double gauss_draw(uint64_t key, int i, int k, int nv, int a) {
  return ih12(key, ((uint64_t)i * ROSV_ROWS_PER_ORBITAL + (uint64_t)k) * (uint64_t)nv + (uint64_t)a);
}

struct GaussRows {        // A(k, a) = Gaussian draw k of orbital i
  uint64_t key;
  int i, nv;
  __device__ __forceinline__ double get(int k, int a) const { return gauss_draw(key, i, k, nv, a); }
};
struct Rows64 {           // A(r, c) = p[r * ld + c]
  const double* p;
  int ld;
  __device__ __forceinline__ double get(int r, int c) const { return p[(size_t)r * ld + c]; }
};

// FP64 form: out[u] (rows x nv) = A_u T_u, A_u the Gaussian rows (mode 0) or Z_u (mode 1,
// rows limited to nrows[u]).  grid: (orbital, row tile, column tile).
__global__ void __launch_bounds__(NT) k_rosv_gemm64(int mode, const double* __restrict__ T, int nv, int i0,
                                                    uint64_t key, const double* __restrict__ Z, const int* nrows,
                                                    int rows, double* out) {
  __shared__ double sm[GEMM_SMEM_DOUBLES];
  const int u = blockIdx.x;
  const int M = mode == 0 ? rows : min(rows, nrows[u]);
  const int m0 = blockIdx.y * TM, n0 = blockIdx.z * TN;
  if (m0 >= M) return;
  const double* Tu = T + (size_t)u * nv * nv;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; a++)
#pragma unroll
    for (int b = 0; b < 4; b++) acc[a][b] = 0.0;
  if (mode == 0) tile_mma(M, nv, nv, m0, n0, GaussRows{key, i0 + u, nv}, Rows64{Tu, nv}, acc, sm);
  else tile_mma(M, nv, nv, m0, n0, Rows64{Z + (size_t)u * rows * nv, nv}, Rows64{Tu, nv}, acc, sm);
  double* o = out + (size_t)u * rows * nv;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int a = 0; a < 4; a++)
#pragma unroll
    for (int b = 0; b < 4; b++) {
      const int rr = m0 + ty + 16 * a, cc = n0 + tx + 16 * b;
      if (rr < M && cc < nv) o[(size_t)rr * nv + cc] = acc[a][b];
    }
}

// Mixed form: TF32 slices along K = n_vir of T_u rows (part 0), of the Gaussian
// rows (part 1) or of Z_u rows (part 2) into the store of orbital u:
//   T   slice s row a : base_u + s * nv + a
//   G/Z slice s row k : base_u + NSL * nv + s * rows + k,  base_u = u * NSL * (nv + rows)
// One warp per (row, 32-wide chunk); rows past nrows[u] (part 2) are written as zeros.
__global__ void __launch_bounds__(256) k_rosv_slices(int part, const double* __restrict__ T, int nv, int i0,
                                                     uint64_t key, const double* __restrict__ Z, int z_rows,
                                                     const int* nrows, int rows, float* __restrict__ S, int ldk) {
  const int u = blockIdx.y;
  const int nch = (nv + tc::CHUNK - 1) / tc::CHUNK;
  const int nr = (part == 0 || part == 3) ? nv : rows;   // parts 2, 3 write zeros for rows >= nrows[u]
  const long long w = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (w >= (long long)nr * nch) return;   // warp-uniform
  const int row = (int)(w / nch), k = (int)(w % nch) * tc::CHUNK + (threadIdx.x & 31);
  double x = 0.0;
  if (k < nv) {
    if (part == 0) x = T[((size_t)u * nv + row) * nv + k];
    else if (part == 1) x = gauss_draw(key, i0 + u, row, nv, k);
    else if (row < nrows[u]) x = Z[((size_t)u * z_rows + row) * nv + k];   // Z or T~: [orbital][z_rows][nv]
  }
  float v[tc::NSL];
  tc::warp_fixed_slices(x, v);
  if (k < nv) {
    const size_t base = (size_t)u * tc::NSL * (nv + rows);
    const bool treg = part == 0 || part == 3;   // T region (T, then T~) or G region (G, then Z)
    const size_t r0 = treg ? base + row : base + (size_t)tc::NSL * nv + row;
    const size_t ss = treg ? (size_t)nv : (size_t)rows;
#pragma unroll
    for (int s = 0; s < tc::NSL; s++) S[(r0 + s * ss) * ldk + k] = v[s];
  }
}

// out[q] = rows[q] . v for q < count (rows nv apart), v in shared memory; each warp
// takes groups of eight rows with eight partial sums per lane in flight, then the
// shuffle tree (fixed order).
constexpr int NT_F = 1024;   // threads of the range-finder CTA

__device__ void block_dots(const double* rows, int count, const double* v, int nv, double* out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int NW = NT_F / 32;
  for (int q0 = warp * 8; q0 < count; q0 += NW * 8) {
    double acc[8];
#pragma unroll
    for (int t = 0; t < 8; t++) acc[t] = 0.0;
    for (int a = lane; a < nv; a += 32) {
      const double va = v[a];
#pragma unroll
      for (int t = 0; t < 8; t++)
        if (q0 + t < count) acc[t] = fma(rows[(size_t)(q0 + t) * nv + a], va, acc[t]);
    }
#pragma unroll
    for (int t = 0; t < 8; t++) {
      const double sum = warp_sum(acc[t]);
      if (lane == 0 && q0 + t < count) out[q0 + t] = sum;
    }
  }
}

// The adaptive range finder of one orbital per CTA.  Y (r + n_max rows of the
// orbital's Ybar) is updated in place: before step s (0-based) the look-ahead
// window is rows s .. s+r-1.  Z receives the orthonormal rows, nrows the count.
// Shared memory: the vector being orthogonalised (nv), the dots (n_max + r).
// v - sum_{q < s} c_q Z_q at entry a: four independent chains (q mod 4), combined in a fixed order.
__device__ __forceinline__ double project_out(double v, const double* c, const double* Z, int s, int nv, int a) {
  double p0 = 0.0, p1 = 0.0, p2 = 0.0, p3 = 0.0;
  int q = 0;
  for (; q + 3 < s; q += 4) {
    p0 = fma(c[q], Z[(size_t)q * nv + a], p0);
    p1 = fma(c[q + 1], Z[(size_t)(q + 1) * nv + a], p1);
    p2 = fma(c[q + 2], Z[(size_t)(q + 2) * nv + a], p2);
    p3 = fma(c[q + 3], Z[(size_t)(q + 3) * nv + a], p3);
  }
  for (; q < s; q++) p0 = fma(c[q], Z[(size_t)q * nv + a], p0);
  return v - ((p0 + p1) + (p2 + p3));
}

__global__ void __launch_bounds__(NT_F) k_rosv_finder(double* Yall, int nv, int r, int n_max, double thr, double* Zall,
                                                    int* nrows, double* wmax, int* err) {
  extern __shared__ double dyn[];
  double* vec = dyn;               // nv
  double* c = dyn + nv;            // n_max dot products
  double* nrm = c + n_max;         // r window norms / dots
  __shared__ double s_scale;
  const int u = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int NW = NT_F / 32;
  double* Y = Yall + (size_t)u * (r + n_max) * nv;
  double* Z = Zall + (size_t)u * n_max * nv;
  int s = 0;
  double mx = 0.0;
  for (;;) {
    for (int w = warp; w < r; w += NW) {
      const double* y = Y + (size_t)(s + w) * nv;
      double d = 0.0;
      for (int a = lane; a < nv; a += 32) d = fma(y[a], y[a], d);
      d = warp_sum(d);
      if (lane == 0) nrm[w] = sqrt(d);
    }
    __syncthreads();
    mx = 0.0;
    for (int w = 0; w < r; w++) mx = fmax(mx, nrm[w]);
    if (!(mx > thr) || s >= n_max) break;
    // z^(s) = y^(s) (1 - Z^T Z) / norm   (Eq. rsvd_za)
    const double* y = Y + (size_t)s * nv;
    for (int a = threadIdx.x; a < nv; a += NT_F) vec[a] = y[a];
    __syncthreads();
    block_dots(Z, s, vec, nv, c);
    __syncthreads();
    double* z = Z + (size_t)s * nv;
    for (int a = threadIdx.x; a < nv; a += NT_F) z[a] = project_out(vec[a], c, Z, s, nv, a);
    __syncthreads();
    if (warp == 0) {
      double d = 0.0;
      for (int a = lane; a < nv; a += 32) d = fma(z[a], z[a], d);
      d = warp_sum(d);
      if (lane == 0) s_scale = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
    }
    __syncthreads();
    const double sc = s_scale;
    for (int a = threadIdx.x; a < nv; a += NT_F) z[a] *= sc;
    // the fresh row g-bar^(s) T, projected against Z^(s-1) (rows 0 .. s-1 of Z)
    double* yn = Y + (size_t)(s + r) * nv;
    for (int a = threadIdx.x; a < nv; a += NT_F) vec[a] = yn[a];
    __syncthreads();
    block_dots(Z, s, vec, nv, c);
    __syncthreads();
    for (int a = threadIdx.x; a < nv; a += NT_F) yn[a] = project_out(vec[a], c, Z, s, nv, a);
    // window rows s+1 .. s+r lose their z^(s) component
    for (int a = threadIdx.x; a < nv; a += NT_F) vec[a] = z[a];
    __syncthreads();
    block_dots(Y + (size_t)(s + 1) * nv, r, vec, nv, nrm);
    __syncthreads();
    for (int idx = threadIdx.x; idx < r * nv; idx += NT_F) {
      const int w = idx / nv, a = idx % nv;
      Y[(size_t)(s + 1 + w) * nv + a] = fma(-nrm[w], vec[a], Y[(size_t)(s + 1 + w) * nv + a]);
    }
    __syncthreads();
    s++;
  }
  if (threadIdx.x == 0) {
    nrows[u] = s;
    wmax[u] = mx;
    if (mx > thr) atomicOr(err, ERR_SIZE);   // the row budget ran out before the window vanished
  }
}

// FP64 form: M[u] (nb x nb padded, zeros outside n = nrows[u]) = T~ T~^T.
__global__ void __launch_bounds__(NT) k_rosv_gram64(const double* Ttall, const int* nrows, int nv, int n_max, int ldm,
                                                    double* Mall) {
  __shared__ double sm[GEMM_SMEM_DOUBLES];
  const int u = blockIdx.x;
  const int n = nrows[u];
  double* M = Mall + (size_t)u * ldm * ldm;
  for (int e = threadIdx.x; e < ldm * ldm; e += NT) M[e] = 0.0;
  __syncthreads();
  const View Tv = dense_view(Ttall + (size_t)u * n_max * nv, n, nv, nv);
  cta_gemm(n, n, nv, 1.0, Tv, transpose(Tv), 0.0, M, ldm, sm);
}

// Q (k x nv) = Q~^T Z from the eigenvectors Q~ of M (eigenvector-major [kmax][ldm],
// descending eigenvalues omega^2), omega = sqrt; each vector signed so that its
// largest-magnitude entry (the first on ties) is positive.
__global__ void __launch_bounds__(NT) k_rosv_backq(const double* Vsall, const double* wsall, const int* ks,
                                                   const double* Zall, const int* nrows, int nv, int n_max, int ldm,
                                                   int kmax, double* Vall, double* wall, int* kout) {
  __shared__ double sm[GEMM_SMEM_DOUBLES];
  const int u = blockIdx.x;
  const int n = nrows[u], k = ks[u];
  const double* Vs = Vsall + (size_t)u * ldm * ldm;
  double* V = Vall + (size_t)u * kmax * nv;
  cta_gemm(k, nv, n, 1.0, dense_view(Vs, k, n, ldm), dense_view(Zall + (size_t)u * n_max * nv, n, nv, nv), 0.0, V,
           nv, sm);
  for (int t = threadIdx.x; t < k; t += NT) wall[(size_t)u * kmax + t] = sqrt(fmax(wsall[(size_t)u * ldm + t], 0.0));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int t = warp; t < k; t += NT / 32) {
    double* v = V + (size_t)t * nv;
    double best = -1.0;
    int bi = nv;
    for (int a = lane; a < nv; a += 32) {
      const double m = fabs(v[a]);
      if (m > best) { best = m; bi = a; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    const bool neg = v[bi] < 0.0;
    __syncwarp();
    if (neg)
      for (int a = lane; a < nv; a += 32) v[a] = -v[a];
  }
  if (threadIdx.x == 0) kout[u] = k;
}

RosvLayout rosv_layout(int nb, int nv, int r, int n_max, int kmax) {
  RosvLayout L;
  L.rows = r + n_max;
  L.y = 0;
  L.z = L.y + (size_t)nb * L.rows * nv;
  L.tt = L.z + (size_t)nb * n_max * nv;
  L.svd = L.tt + (size_t)nb * n_max * nv;
  (void)kmax;
  L.svd_per = 2 * (size_t)n_max * n_max + 2 * (size_t)n_max + eig_osv_scratch_doubles(n_max, n_max);
  L.wmax = L.svd + (size_t)nb * L.svd_per;
  L.nrows = L.wmax + nb;
  L.total = L.nrows + (size_t)nb + 64;
  L.ldk = (nv + 3) & ~3;
  L.store_rows = (long long)nb * tc::NSL * (nv + L.rows);
  return L;
}

void launch_rosv_gemm64(int mode, const double* T, int nb, int nv, int i0, uint64_t key, const double* Z,
                        const int* nrows, int rows, double* out, cudaStream_t st) {
  dim3 g(nb, (rows + TM - 1) / TM, (nv + TN - 1) / TN);
  k_rosv_gemm64<<<g, NT, 0, st>>>(mode, T, nv, i0, key, Z, nrows, rows, out);
  note_launch(1);
}

void launch_rosv_slices(int part, const double* T, int nb, int nv, int i0, uint64_t key, const double* Z,
                        int z_rows, const int* nrows, int rows, float* slices, int ldk, cudaStream_t st) {
  const int nch = (nv + tc::CHUNK - 1) / tc::CHUNK;
  const long long nr = part == 0 ? nv : rows;
  dim3 g((unsigned)((nr * nch + 7) / 8), nb);
  k_rosv_slices<<<g, 256, 0, st>>>(part, T, nv, i0, key, Z, z_rows, nrows, rows, slices, ldk);
  note_launch(1);
}

void launch_rosv_finder(double* Y, int nb, int nv, int r, int n_max, double l_osv, double* Z, int* nrows,
                        double* wmax, int* err, cudaStream_t st) {
  const double thr = l_osv / (10.0 * 0.7978845608028654);   // l_osv / (10 sqrt(2/pi))
  const size_t smem = (size_t)(nv + n_max + r) * sizeof(double);
  cudaFuncSetAttribute(k_rosv_finder, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_rosv_finder<<<nb, NT_F, smem, st>>>(Y, nv, r, n_max, thr, Z, nrows, wmax, err);
  note_launch(1);
}

void launch_rosv_gram64(const double* Tt, const int* nrows, int nb, int nv, int n_max, int ldm, double* M,
                        cudaStream_t st) {
  k_rosv_gram64<<<nb, NT, 0, st>>>(Tt, nrows, nv, n_max, ldm, M);
  note_launch(1);
}

void launch_rosv_backq(const double* Vs, const double* ws, const int* ks, const double* Z, const int* nrows, int nb,
                       int nv, int n_max, int ldm, int kmax, double* V, double* w, int* k, cudaStream_t st) {
  k_rosv_backq<<<nb, NT, 0, st>>>(Vs, ws, ks, Z, nrows, nv, n_max, ldm, kmax, V, w, k);
  note_launch(1);
}

}  // namespace osv
