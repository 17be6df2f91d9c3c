// Occupied-orbital localization (Section 3.2, Algorithm 2): Pipek-Mezey with
// Loewdin charges by Jacobi sweeps.
//   P^A_ij = sum_{alpha in A} C~_alpha,i C~_alpha,j
//   per pair i < j in order: a_ij = sum_A (P^A_ij)^2 - (P^A_ii - P^A_jj)^2 / 4,
//   b_ij = sum_A P^A_ij (P^A_ii - P^A_jj), theta = atan2(b, -a) / 4 (Eq. loc_theta,
//   the branch that maximises L), skipped when |sin theta| < 1e-10; otherwise
//   dL += sqrt(a^2 + b^2)(1 - cos 4 theta) and columns i, j of U and both MO
//   indices of every P^A are rotated.  Sweeps until dL <= l_loc.
// The pairs are sequential (each rotation uses the previous one's P); every
// rotation is spread over the CTA's threads by (k, atom), as in the paper.
// Layout: P [n][n][n_atom] (atom index innermost), U [n][n] row-major.
#include "internal.h"

namespace osv {

constexpr int NT_LOC = 1024;

__global__ void k_pm_charges(const double* __restrict__ C, int n_ao, int n, const int* __restrict__ atom_ao,
                             int n_atom, double* __restrict__ P) {
  const long long tot = (long long)n * n * n_atom;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int A = (int)(e % n_atom);
    const long long ij = e / n_atom;
    const int i = (int)(ij / n), j = (int)(ij % n);
    double s = 0.0;
    for (int al = atom_ao[A]; al < atom_ao[A + 1]; al++) s = fma(C[(size_t)al * n + i], C[(size_t)al * n + j], s);
    P[e] = s;
  }
}

// Deterministic CTA sum over NT_LOC threads (shuffle tree, then the warps in order).
__device__ double loc_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < NT_LOC / 32; k++) s += red[k];
    red[32] = s;
  }
  __syncthreads();
  const double r = red[32];
  __syncthreads();
  return r;
}

// out[0] = L, out[1] = dL of the last sweep; status[0] = sweeps, status[1] = 1 if converged.
__global__ void __launch_bounds__(NT_LOC) k_pm_sweeps(double* __restrict__ P, double* __restrict__ U, int n, int n_atom,
                                                      double l_loc, int max_sweeps, double* out, int* status) {
  __shared__ double red[33];
  __shared__ double s_c, s_s;
  __shared__ int s_skip;
  const int tid = threadIdx.x;
  for (int k = tid; k < n * n; k += NT_LOC) U[k] = (k / n == k % n) ? 1.0 : 0.0;
  __syncthreads();
  double dL = 0.0;   // meaningful on thread 0
  int sweeps = 0, conv = 0;
  while (sweeps < max_sweeps) {
    sweeps++;
    dL = 0.0;
    for (int i = 0; i < n; i++)
      for (int j = i + 1; j < n; j++) {
        double pa = 0.0, pb = 0.0;
        const double* Pij = P + ((size_t)i * n + j) * n_atom;
        const double* Pii = P + ((size_t)i * n + i) * n_atom;
        const double* Pjj = P + ((size_t)j * n + j) * n_atom;
        for (int A = tid; A < n_atom; A += NT_LOC) {
          const double x = Pij[A], d = Pii[A] - Pjj[A];
          pa += x * x - 0.25 * d * d;
          pb += x * d;
        }
        const double a = loc_sum(pa, red);
        const double b = loc_sum(pb, red);
        if (tid == 0) {
          const double th = 0.25 * atan2(b, -a);
          double sn, cs;
          sincos(th, &sn, &cs);
          s_skip = fabs(sn) < 1e-10;
          s_c = cs;
          s_s = sn;
          if (!s_skip) dL += sqrt(a * a + b * b) * (1.0 - cos(4.0 * th));
        }
        __syncthreads();
        if (s_skip) continue;
        const double c = s_c, s = s_s;
        for (int k = tid; k < n; k += NT_LOC) {
          const double ui = U[(size_t)k * n + i], uj = U[(size_t)k * n + j];
          U[(size_t)k * n + i] = c * ui + s * uj;
          U[(size_t)k * n + j] = c * uj - s * ui;
        }
        // rows i, j against every other k (the first index), mirrored into the columns
        for (long long e = tid; e < (long long)n * n_atom; e += NT_LOC) {
          const int k = (int)(e / n_atom), A = (int)(e % n_atom);
          if (k == i || k == j) continue;
          double* pik = P + ((size_t)i * n + k) * n_atom + A;
          double* pjk = P + ((size_t)j * n + k) * n_atom + A;
          const double x = *pik, y = *pjk;
          const double nx = c * x + s * y, ny = c * y - s * x;
          *pik = nx;
          *pjk = ny;
          P[((size_t)k * n + i) * n_atom + A] = nx;
          P[((size_t)k * n + j) * n_atom + A] = ny;
        }
        // the (i, j) block: first index, then second index
        for (int A = tid; A < n_atom; A += NT_LOC) {
          double* qii = P + ((size_t)i * n + i) * n_atom + A;
          double* qij = P + ((size_t)i * n + j) * n_atom + A;
          double* qji = P + ((size_t)j * n + i) * n_atom + A;
          double* qjj = P + ((size_t)j * n + j) * n_atom + A;
          const double ri0 = c * *qii + s * *qji, ri1 = c * *qij + s * *qjj;   // row i after the first rotation
          const double rj0 = c * *qji - s * *qii, rj1 = c * *qjj - s * *qij;   // row j
          *qii = c * ri0 + s * ri1;
          *qij = c * ri1 - s * ri0;
          *qji = c * rj0 + s * rj1;
          *qjj = c * rj1 - s * rj0;
        }
        __syncthreads();
      }
    __shared__ int s_done;
    if (tid == 0) s_done = !(dL > l_loc);
    __syncthreads();
    if (s_done) {
      conv = 1;
      break;
    }
  }
  double lsum = 0.0;
  for (long long e = tid; e < (long long)n * n_atom; e += NT_LOC) {
    const int i = (int)(e / n_atom), A = (int)(e % n_atom);
    const double d = P[((size_t)i * n + i) * n_atom + A];
    lsum += d * d;
  }
  const double L = loc_sum(lsum, red);
  if (tid == 0) {
    out[0] = L;
    out[1] = dL;
    status[0] = sweeps;
    status[1] = conv;
  }
}

// ---------------------------------------------------------------- whole-GPU form
// The same sweeps with the atoms spread over a cooperative grid: CTA c owns the
// charge matrices of atoms [c apc, (c+1) apc) (atom-major [A][n][n], in shared
// memory when they fit).  Per rotation every CTA writes its partial (a, b), one
// grid barrier, and every CTA adds the G partials in the same fixed order, so all
// CTAs take the same angle, the same skip decision and the same dL, and rotate
// their own atoms; CTA 0 also rotates U.  The barrier is a counter and a
// generation word with a bounded wait: a CTA that waits too long sets ERR_TIMEOUT
// and leaves, and the others then time out at their next barrier.
constexpr int NT_G = 256;
constexpr long long PM_WAIT_LIMIT = 1ll << 22;   // polls (with a short sleep) before giving up

__device__ bool pm_grid_sync(unsigned* bar, unsigned nblocks) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
      s_ok = 1;
    } else {
      long long it = 0;
      while (*gen == g && it < PM_WAIT_LIMIT) {
        __nanosleep(32);
        it++;
      }
      s_ok = *gen != g;
    }
    __threadfence();
  }
  __syncthreads();
  return s_ok != 0;
}

__global__ void k_pm_charges_am(const double* __restrict__ C, int n, const int* __restrict__ atom_ao, int n_atom,
                                double* __restrict__ P) {
  const long long tot = (long long)n_atom * n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int A = (int)(e / ((long long)n * n));
    const int ij = (int)(e % ((long long)n * n)), i = ij / n, j = ij % n;
    double s = 0.0;
    for (int al = atom_ao[A]; al < atom_ao[A + 1]; al++) s = fma(C[(size_t)al * n + i], C[(size_t)al * n + j], s);
    P[e] = s;
  }
}

__device__ double pm_block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < NT_G / 32; k++) s += red[k];
    red[32] = s;
  }
  __syncthreads();
  const double r = red[32];
  __syncthreads();
  return r;
}

// sum of x[0], x[stride], ... x[(G-1) stride] by warp 0 in a fixed order (lane stride, then the shuffle tree)
__device__ double pm_sum_parts(const double* x, int G, int stride) {
  double s = 0.0;
  for (int q = threadIdx.x & 31; q < G; q += 32) s += __ldcg(x + (size_t)q * stride);
  return warp_sum(s);
}

template <bool SMEM>
__global__ void __launch_bounds__(NT_G) k_pm_grid(double* __restrict__ Pg, double* __restrict__ U, int n, int n_atom,
                                                  int apc, double l_loc, int max_sweeps, double* part, unsigned* bar,
                                                  double* out, int* status, int* err) {
  extern __shared__ double dyn[];
  __shared__ double red[33];
  __shared__ double s_c, s_s;
  __shared__ int s_skip;
  const int cb = blockIdx.x, G = gridDim.x, tid = threadIdx.x;
  const int A0 = cb * apc, na = max(0, min(n_atom, A0 + apc) - A0);
  const size_t NN = (size_t)n * n;
  double* P = SMEM ? dyn : Pg + (size_t)A0 * NN;
  if (SMEM)
    for (size_t e = tid; e < (size_t)na * NN; e += NT_G) dyn[e] = Pg[(size_t)A0 * NN + e];
  if (cb == 0)
    for (int k = tid; k < n * n; k += NT_G) U[k] = (k / n == k % n) ? 1.0 : 0.0;
  __syncthreads();
  double dL = 0.0;
  int sweeps = 0, conv = 0;
  long long rot = 0;
  while (sweeps < max_sweeps) {
    sweeps++;
    dL = 0.0;
    for (int i = 0; i < n; i++)
      for (int j = i + 1; j < n; j++, rot++) {
        double pa = 0.0, pb = 0.0;
        for (int t = tid; t < na; t += NT_G) {
          const double* Pa = P + (size_t)t * NN;
          const double x = Pa[(size_t)i * n + j], d = Pa[(size_t)i * n + i] - Pa[(size_t)j * n + j];
          pa += x * x - 0.25 * d * d;
          pb += x * d;
        }
        pa = pm_block_sum(pa, red);
        pb = pm_block_sum(pb, red);
        double* pp = part + (size_t)(rot & 1) * 2 * G;
        if (tid == 0) {
          pp[2 * cb] = pa;
          pp[2 * cb + 1] = pb;
        }
        if (!pm_grid_sync(bar, (unsigned)G)) {
          if (tid == 0) atomicOr(err, ERR_TIMEOUT);
          return;
        }
        if (tid < 32) {
          const double a = pm_sum_parts(pp, G, 2);
          const double b = pm_sum_parts(pp + 1, G, 2);
          if (tid == 0) {
            const double th = 0.25 * atan2(b, -a);
            double sn, cs;
            sincos(th, &sn, &cs);
            s_skip = fabs(sn) < 1e-10;
            s_c = cs;
            s_s = sn;
            if (!s_skip) dL += sqrt(a * a + b * b) * (1.0 - cos(4.0 * th));
          }
        }
        __syncthreads();
        if (s_skip) continue;
        const double c = s_c, s = s_s;
        if (cb == 0)
          for (int k = tid; k < n; k += NT_G) {
            const double ui = U[(size_t)k * n + i], uj = U[(size_t)k * n + j];
            U[(size_t)k * n + i] = c * ui + s * uj;
            U[(size_t)k * n + j] = c * uj - s * ui;
          }
        for (int e = tid; e < na * n; e += NT_G) {
          const int t = e / n, k = e % n;
          if (k == i || k == j) continue;
          double* Pa = P + (size_t)t * NN;
          const double x = Pa[(size_t)i * n + k], y = Pa[(size_t)j * n + k];
          const double nx = c * x + s * y, ny = c * y - s * x;
          Pa[(size_t)i * n + k] = nx;
          Pa[(size_t)j * n + k] = ny;
          Pa[(size_t)k * n + i] = nx;
          Pa[(size_t)k * n + j] = ny;
        }
        for (int t = tid; t < na; t += NT_G) {
          double* Pa = P + (size_t)t * NN;
          const double qii = Pa[(size_t)i * n + i], qij = Pa[(size_t)i * n + j];
          const double qji = Pa[(size_t)j * n + i], qjj = Pa[(size_t)j * n + j];
          const double ri0 = c * qii + s * qji, ri1 = c * qij + s * qjj;
          const double rj0 = c * qji - s * qii, rj1 = c * qjj - s * qij;
          Pa[(size_t)i * n + i] = c * ri0 + s * ri1;
          Pa[(size_t)i * n + j] = c * ri1 - s * ri0;
          Pa[(size_t)j * n + i] = c * rj0 + s * rj1;
          Pa[(size_t)j * n + j] = c * rj1 - s * rj0;
        }
        __syncthreads();
      }
    if (!(dL > l_loc)) {   // the same value in every CTA (thread 0 of each holds it)
      conv = 1;
    }
    __shared__ int s_conv;
    if (tid == 0) s_conv = conv;
    __syncthreads();
    if (s_conv) break;
  }
  // L = sum_{A, i} (P^A_ii)^2
  double ls = 0.0;
  for (int e = tid; e < na * n; e += NT_G) {
    const double d = P[(size_t)(e / n) * NN + (size_t)(e % n) * n + (e % n)];
    ls += d * d;
  }
  ls = pm_block_sum(ls, red);
  double* pl = part + (size_t)(rot & 1) * 2 * G;
  if (tid == 0) pl[2 * cb] = ls;
  if (!pm_grid_sync(bar, (unsigned)G)) {
    if (tid == 0) atomicOr(err, ERR_TIMEOUT);
    return;
  }
  if (cb == 0 && tid < 32) {
    const double L = pm_sum_parts(pl, G, 2);
    if (tid == 0) {
      out[0] = L;
      out[1] = dL;
      status[0] = sweeps;
      status[1] = conv;
    }
  }
}

// Cooperative whole-GPU launch when every CTA can be resident; returns false if not
// possible (the caller then uses the one-CTA form).  scratch: 4 * max CTAs doubles.
bool launch_pm_localize_grid(const double* C, int n, const int* atom_ao, int n_atom, double l_loc, int max_sweeps,
                             double* P, double* U, double* out, int* status, double* part, unsigned* bar, int* err,
                             int num_sms, cudaStream_t st) {
  const size_t nn = (size_t)n * n;
  int G = std::min(n_atom, num_sms);
  int apc = (n_atom + G - 1) / G;
  G = (n_atom + apc - 1) / apc;
  const size_t smem = (size_t)apc * nn * sizeof(double);
  const bool use_smem = smem <= 200 * 1024;
  void* fn = use_smem ? (void*)k_pm_grid<true> : (void*)k_pm_grid<false>;
  const size_t dsm = use_smem ? smem : 0;
  if (use_smem && cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NT_G, dsm) != cudaSuccess || per_sm < 1 ||
      per_sm * num_sms < G) {
    cudaGetLastError();
    return false;
  }
  const long long tot = (long long)n_atom * nn;
  k_pm_charges_am<<<(int)std::min<long long>((tot + 255) / 256, 8LL * num_sms), 256, 0, st>>>(C, n, atom_ao, n_atom, P);
  cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st);
  void* args[] = {&P, &U, const_cast<int*>(&n), const_cast<int*>(&n_atom), &apc, &l_loc, &max_sweeps, &part, &bar, &out,
                  &status, &err};
  if (cudaLaunchCooperativeKernel(fn, dim3(G), dim3(NT_G), args, dsm, st) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  note_launch(2);
  return true;
}

void launch_pm_localize(const double* C, int n_ao, int n, const int* atom_ao, int n_atom, double l_loc, int max_sweeps,
                        double* P, double* U, double* out, int* status, int num_sms, cudaStream_t st) {
  const long long tot = (long long)n * n * n_atom;
  const int grid = (int)std::min<long long>((tot + 255) / 256, 8LL * num_sms);
  k_pm_charges<<<grid, 256, 0, st>>>(C, n_ao, n, atom_ao, n_atom, P);
  k_pm_sweeps<<<1, NT_LOC, 0, st>>>(P, U, n, n_atom, l_loc, max_sweeps, out, status);
  note_launch(2);
}

}  // namespace osv
