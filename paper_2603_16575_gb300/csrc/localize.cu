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

void launch_pm_localize(const double* C, int n_ao, int n, const int* atom_ao, int n_atom, double l_loc, int max_sweeps,
                        double* P, double* U, double* out, int* status, int num_sms, cudaStream_t st) {
  const long long tot = (long long)n * n * n_atom;
  const int grid = (int)std::min<long long>((tot + 255) / 256, 8LL * num_sms);
  k_pm_charges<<<grid, 256, 0, st>>>(C, n_ao, n, atom_ao, n_atom, P);
  k_pm_sweeps<<<1, NT_LOC, 0, st>>>(P, U, n, n_atom, l_loc, max_sweeps, out, status);
  note_launch(2);
}

}  // namespace osv
