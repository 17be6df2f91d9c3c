// A0 in the mixed form: T_i = (B_i B_i^T) / (e_a + e_b - 2 f_ii) (Eq. mp2_tkk,
// positive denominator) on the tcgen05 tensor cores.  B_i is cut into
// fixed-point TF32 slices along the aux index (tf32_split.cuh) and contracted
// with itself by the split-precision kernel of tc_tf32x3.cuh, so T_i carries
// ~35 bits of its FP64 inputs; its eigen-decomposition stays FP64.
//
// Only the tiles that touch the lower triangle are computed.  Each element
// with a >= b is divided by its denominator and written to both T[a][b] and
// T[b][a], so T_i is exactly symmetric.
#include "internal.h"
#include "tc_tf32x3.cuh"

namespace osv {

// Slices of B_i with K = aux: slot u (orbital i0 + u), slice s, row a at
// Bt + ((u * NSL + s) * n_vir + a) * ldx.  One warp per (a, 32-aux chunk).
__global__ void __launch_bounds__(256) k_rslices(BSrc src, int i0, float* __restrict__ Bt, int ldx) {
  const int u = blockIdx.y, i = i0 + u;
  const int nch = (src.n_aux + tc::CHUNK - 1) / tc::CHUNK;
  const long long w = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (w >= (long long)src.n_vir * nch) return;   // warp-uniform
  const int a = (int)(w / nch), P = (int)(w % nch) * tc::CHUNK + (threadIdx.x & 31);
  float v[tc::NSL];
  tc::warp_fixed_slices(P < src.n_aux ? src.get(i, a, P) : 0.0, v);
  if (P < src.n_aux) {
    const size_t sl = (size_t)src.n_vir * ldx;
    float* o = Bt + ((size_t)u * tc::NSL * src.n_vir + a) * ldx + P;
#pragma unroll
    for (int s = 0; s < tc::NSL; s++) o[s * sl] = v[s];
  }
}

void launch_rslices(const BSrc& src, int i0, int nb, float* Bt, int ldx, cudaStream_t st) {
  if (!nb) return;
  const long long warps = (long long)src.n_vir * ((src.n_aux + tc::CHUNK - 1) / tc::CHUNK);
  dim3 grid((unsigned)((warps + 7) / 8), nb);
  k_rslices<<<grid, 256, 0, st>>>(src, i0, Bt, ldx);
  note_launch(1);
}

// T[a][b] = T[b][a] = (hi + lo) / (e_a + e_b - s) for a >= b; out = T_i, s = 2 f_ii.
struct EpiT {
  static constexpr bool kWarp = false;
  const double* e_vir;
  __device__ __forceinline__ void operator()(const tc::Job& jb, int r, int c, float h, float l) const {
    const int a = jb.m0 + r, b = jb.n0 + c;
    if (a < b) return;
    const double v = ((double)h + (double)l) / (e_vir[a] + e_vir[b] - jb.s);
    double* T = static_cast<double*>(jb.out);
    T[(size_t)a * jb.ld_out + b] = v;
    T[(size_t)b * jb.ld_out + a] = v;
  }
};

int launch_tii_tc(const float* Bt, long long rows, int n_aux, int ldx, const tc::Job* jobs, int n_jobs,
                  const double* e_vir, int* err, cudaStream_t st) {
  if (!n_jobs) return 0;
  if (cudaFuncSetAttribute(tc::k_tf32x3<EpiT>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM) != cudaSuccess)
    return -1;
  CUtensorMap ma, mb;
  if (!make_slice_map(&ma, Bt, n_aux, ldx, rows, tc::BM) || !make_slice_map(&mb, Bt, n_aux, ldx, rows, tc::BROWS))
    return -1;
  tc::k_tf32x3<EpiT><<<tc::persistent_grid(n_jobs), tc::NTHREADS, tc::SMEM, st>>>(ma, mb, jobs, n_jobs, n_aux, err, EpiT{e_vir});
  note_launch(1);
  return 0;
}

}  // namespace osv
