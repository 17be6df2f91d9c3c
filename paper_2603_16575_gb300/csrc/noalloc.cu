// Allocation-free variant of the pair preconditioner (the k_precond kernel of
// precond.cu): the same canonical orthogonalisation of S followed by the
// eigen-decomposition of Y^T F Y, for ONE pair whose S and F the caller passes
// as dense matrices, with all scratch in a file-scope device array instead of
// cudaMalloc'd workspace.
//
// Who needs this: callers that must not allocate device memory while they run
// -- a process that hands all GPU memory to its own pool allocator at start-up
// and forbids further driver allocations, a plug-in running inside another
// application's CUDA context under that application's memory budget, or a
// latency-critical loop in which a cudaMalloc (which may synchronise the
// device) is unacceptable.
#include <cstdio>

#include "osvmp2.h"
#include "eig.cuh"
#include "internal.h"

namespace osv {

constexpr int NOALLOC_ZMAX = 144;  // eigenvector matrix kept in shared memory up to this order

// Scratch of one preconditioner solve: S, F copies, Z, Y, F Y, Y^T F Y
// (6 m^2) plus e, tau, eigenvalues of S and of Y^T F Y (4 m).  Sized for
// m <= OSVMP2_NOALLOC_MAX_M; every GPU that loads the library holds it
// (about 3.2 MB) until the process exits.
constexpr size_t NOALLOC_SCRATCH =
    6 * (size_t)OSVMP2_NOALLOC_MAX_M * OSVMP2_NOALLOC_MAX_M + 4 * (size_t)OSVMP2_NOALLOC_MAX_M + 64;
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH];

__global__ void __launch_bounds__(NT) k_precond_dense(const double* __restrict__ S, const double* __restrict__ F,
                                                      int m, double tau_s, double* X, double* et, int* r_out,
                                                      double* scratch) {
  extern __shared__ double dyn[];
  __shared__ int s_r;
  double* gsm = dyn;
  double* esm = dyn + GEMM_SMEM_DOUBLES;
  double* zsm = esm + 4 * OSVMP2_NOALLOC_MAX_M + 64;
  int* keep = reinterpret_cast<int*>(esm);
  const size_t M2 = (size_t)m * m;
  // every scratch element below is written before it is read, so nothing
  // left by an earlier call needs clearing
  double* Sw = scratch;
  double* Fw = Sw + M2;
  double* Zg = Fw + M2;
  double* Yw = Zg + M2;
  double* W1 = Yw + M2;
  double* Fp = W1 + M2;
  double* e = Fp + M2;
  double* tau = e + m;
  double* ws = tau + m;
  double* w2 = ws + m;
  int bad = 0;
  for (int idx = threadIdx.x; idx < m * m; idx += NT) {
    const double sv = S[idx], fv = F[idx];
    bad |= !isfinite(sv) || !isfinite(fv);
    Sw[idx] = sv;
    Fw[idx] = fv;
  }
  // a NaN or Inf in S or F is refused up front: the eigen-solver's scalings
  // (fmax over magnitudes) would otherwise drop it silently
  if (__syncthreads_or(bad)) {
    if (threadIdx.x == 0) *r_out = -1;
    return;
  }
  double* Z = (m <= NOALLOC_ZMAX) ? zsm : Zg;
  const int ldz = (m <= NOALLOC_ZMAX) ? m + 1 : m;
  int rc = cta_syev(Sw, m, m, ws, Z, ldz, e, tau, esm);
  if (threadIdx.x == 0) {
    double smax = 0.0;
    bool finite = true;
    for (int c = 0; c < m; c++) {
      finite = finite && isfinite(ws[c]);
      smax = fmax(smax, ws[c]);
    }
    int r = 0;
    for (int c = 0; c < m; c++)
      if (ws[c] > tau_s * smax) keep[r++] = c;
    s_r = (rc != 0 || !finite) ? -1 : r;
  }
  __syncthreads();
  const int r = s_r;
  if (r <= 0) {
    // r == 0: S has no eigenvalue above tau_s * max (e.g. S = 0); nothing to
    // diagonalise, X and e~ are left untouched
    if (threadIdx.x == 0) *r_out = r;
    return;
  }
  for (int idx = threadIdx.x; idx < m * r; idx += NT) {
    const int row = idx / r, c = idx % r;
    const int kc = keep[c];
    Yw[(size_t)row * m + c] = Z[(size_t)row * ldz + kc] / sqrt(ws[kc]);
  }
  __syncthreads();
  const View Yv = dense_view(Yw, m, r, m);
  cta_gemm(m, r, m, 1.0, dense_view(Fw, m, m, m), Yv, 0.0, W1, m, gsm);
  cta_gemm(r, r, m, 1.0, transpose(Yv), dense_view(W1, m, r, m), 0.0, Fp, r, gsm);
  double* Z2 = (r <= NOALLOC_ZMAX) ? zsm : Zg;
  const int ldz2 = (r <= NOALLOC_ZMAX) ? r + 1 : r;
  rc = cta_syev(Fp, r, r, w2, Z2, ldz2, e, tau, esm);
  cta_gemm(m, r, r, 1.0, Yv, dense_view(Z2, r, r, ldz2), 0.0, X, m, gsm);
  for (int c = threadIdx.x; c < r; c += NT) et[c] = w2[c];
  if (threadIdx.x == 0) {
    bool finite = true;
    for (int c = 0; c < r; c++) finite = finite && isfinite(w2[c]);
    *r_out = (rc == 0 && finite) ? r : -1;
  }
}

}  // namespace osv

extern "C" int osvmp2_precond_noalloc(const double* S, const double* F, int32_t m, double tau_s, double* X,
                                      double* et, int32_t* r_dev, void* cuda_stream, char* err, int32_t err_len) {
  auto msg = [&](const char* text) {
    if (err && err_len > 0) snprintf(err, (size_t)err_len, "%s", text);
  };
  if (!S || !F || !X || !et || !r_dev || !(tau_s >= 0.0)) {
    msg("osvmp2_precond_noalloc: null pointer or negative tau_s");
    return OSVMP2_E_ARG;
  }
  if (m < 1 || m > OSVMP2_NOALLOC_MAX_M) {
    char b[160];
    snprintf(b, sizeof b, "osvmp2_precond_noalloc: m = %d is outside 1..%d (the size of its static scratch)", m,
             OSVMP2_NOALLOC_MAX_M);
    msg(b);
    return OSVMP2_E_ARG;
  }
  // Set-up, done on every call with the caller's device and context current:
  // the device address of the static scratch in this context (host code only
  // sees a host-side stand-in for the array; a kernel given that stand-in
  // would read the wrong memory) and the kernel's shared-memory limit.  Both
  // are look-ups that allocate nothing once the library's module is loaded in
  // the context; the first call in a context may load it (lazy module
  // loading), which is why that call should come before any stream capture.
  // Nothing is cached across calls, so a context that was reset or replaced
  // (cudaDeviceReset, a plug-in's own context) never sees a stale address.
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, osv::g_noalloc_scratch) != cudaSuccess || !p) {
    cudaGetLastError();
    msg("osvmp2_precond_noalloc: cudaGetSymbolAddress of the static scratch failed (no usable CUDA device?)");
    return OSVMP2_E_CUDA;
  }
  double* scratch = static_cast<double*>(p);
  const size_t smem = (size_t)(osv::GEMM_SMEM_DOUBLES + 4 * OSVMP2_NOALLOC_MAX_M + 64 +
                               osv::NOALLOC_ZMAX * (osv::NOALLOC_ZMAX + 1)) * sizeof(double);
  if (cudaFuncSetAttribute(osv::k_precond_dense, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess) {
    cudaGetLastError();
    msg("osvmp2_precond_noalloc: cudaFuncSetAttribute failed");
    return OSVMP2_E_CUDA;
  }
  osv::k_precond_dense<<<1, osv::NT, smem, (cudaStream_t)cuda_stream>>>(S, F, m, tau_s, X, et, r_dev, scratch);
  osv::note_launch(1);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    msg(cudaGetErrorString(e));
    return OSVMP2_E_CUDA;
  }
  return OSVMP2_OK;
}
