// On-device regeneration of the RI integrals B[i,a,P] = env[i,a] * z(seed,i,a,P)
// from the counter-based generator (SplitMix64 draws, Irwin-Hall(12) normal).
#include "osvmp2.h"
#include "internal.h"

namespace osv {

__global__ void k_generate_B(BSrc src, int i0, int n_i, double* __restrict__ out) {
  const size_t per = (size_t)src.n_vir * src.n_aux;
  const size_t total = per * n_i;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(idx / per);
    const size_t rem = idx % per;
    const int a = (int)(rem / src.n_aux), P = (int)(rem % src.n_aux);
    out[idx] = src.get(i0 + b, a, P);
  }
}

}  // namespace osv

extern "C" int osvmp2_generate_B(int32_t n_occ, int32_t n_vir, int32_t n_aux, uint64_t seed, const double* env,
                                 int32_t i0, int32_t n_i, double* out, void* cuda_stream) {
  if (n_occ <= 0 || n_vir <= 0 || n_aux <= 0 || !env || !out || i0 < 0 || n_i < 0 || i0 + n_i > n_occ)
    return OSVMP2_E_ARG;
  if (n_i == 0) return OSVMP2_OK;
  const uint64_t key = osv::mix64(seed ^ (5ull * 0xD1B54A32D192ED03ull));
  osv::BSrc src{nullptr, env, key, n_vir, n_aux};
  osv::k_generate_B<<<1184, 256, 0, (cudaStream_t)cuda_stream>>>(src, i0, n_i, out);
  osv::note_launch(1);
  return cudaGetLastError() == cudaSuccess ? OSVMP2_OK : OSVMP2_E_CUDA;
}
