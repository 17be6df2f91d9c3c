// Mixed form, A1 in the orthonormal pair basis: G_p,x = U_p^T B_x on the
// tcgen05 tensor cores (Eq. osv_imua with the preconditioner basis of
// Eq. prec_eig).  Both operands enter as four fixed-point TF32 slices per
// 32-virtual chunk (tf32_split.cuh); the leading slice products are summed
// exactly by the tensor core (tc_tf32x3.cuh), so G carries ~35 bits of the
// FP64 inputs before its final rounding to FP32.
//
// Layout (row-major, K = n_vir innermost, rows padded to ldv floats):
//   Bs  [slot][slice][n_aux][ldv]   B_x^T slices of the orbitals of one batch
//   Us  [pair][slice][r][ldv]       U_p^T slices (written by k_ubasis)
// The tile M dimension is the aux index (128 per tile), N the pair-basis
// index mu (<= 64 per tile), so the output G[mu][P] is stored with the TMEM
// lane (aux) as the contiguous index.
//
// The epilogue keeps G as a normalised FP32 pair (G, lo), and k_gslices cuts it
// into the fixed-point slices of G^T along the aux index, the k-chunks of the
// next contraction K~_p = G_p,i G_p,j^T (Eq. osv_close_k in the orthonormal
// pair basis), which then runs on the tensor cores with the same split-precision
// kernel: exact slice products and ~35 bits in K~, where FP32 products of the
// rounded G would leave a relative error of ~1e-8 in every pair energy.
//   Gs  [G job][slice][r][ldg]      G_p,x slices, K = n_aux innermost
#include "internal.h"
#include "tc_tf32x3.cuh"

#include <cudaTypedefs.h>

namespace osv {

// B_x^T slices: one CTA per (32 virtuals x 32 aux functions) tile of one orbital
// (the 32 virtuals are one k-chunk), transposed through shared memory so that
// both the read of B (aux innermost) and the write of Bs (virtuals innermost)
// are coalesced.
__global__ void __launch_bounds__(256) k_bslices(BSrc src, const int* __restrict__ xs, float* __restrict__ Bs,
                                                 int ldv) {
  __shared__ double tile[32][33];
  const int u = blockIdx.z, x = xs[u];
  const int a0 = blockIdx.y * tc::CHUNK, P0 = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int da = ty; da < 32; da += 8) {
    const int a = a0 + da, P = P0 + tx;
    tile[tx][da] = (a < src.n_vir && P < src.n_aux) ? src.get(x, a, P) : 0.0;
  }
  __syncthreads();
  const size_t slice = (size_t)src.n_aux * ldv;
  float* base = Bs + (size_t)u * tc::NSL * slice;
  for (int dP = ty; dP < 32; dP += 8) {       // warp-uniform: one aux row per warp step
    const int P = P0 + dP, a = a0 + tx;
    float v[tc::NSL];
    tc::warp_fixed_slices(tile[dP][tx], v);
    if (P < src.n_aux && a < src.n_vir) {
      float* o = base + (size_t)P * ldv + a;
#pragma unroll
      for (int s = 0; s < tc::NSL; s++) o[s * slice] = v[s];
    }
  }
}

void launch_bslices(const BSrc& src, const int* xs, int n_x, float* Bs, int ldv, cudaStream_t st) {
  if (!n_x) return;
  dim3 grid((src.n_aux + 31) / 32, (src.n_vir + 31) / 32, n_x);
  k_bslices<<<grid, 256, 0, st>>>(src, xs, Bs, ldv);
  note_launch(1);
}

// G[mu][P] = hi + lo (TMEM lane = aux row P, column = mu), normalised by a
// two-sum: the leading FP32 part to G (the FP32 G of the gradient) and the
// remainder to the same position of a second array lo_shift floats further on;
// k_gslices cuts the pair into the slices of G^T.
struct EpiG2 {
  static constexpr bool kWarp = false;
  long long lo_shift;
  __device__ __forceinline__ void operator()(const tc::Job& jb, int r, int c, float h, float l) const {
    float s, e;
    tc::two_sum(h, l, s, e);
    float* g = static_cast<float*>(jb.out) + (size_t)c * jb.ld_out + r;
    g[0] = s;
    g[lo_shift] = e;
  }
};

// The slices of G_p,x^T from (G, lo): one warp per (mu, 32-aux chunk), lanes along
// the aux index; slice s of row mu at Gs[(x_row + s r + mu) ldg + P].
__global__ void __launch_bounds__(256) k_gslices(const GSJob* __restrict__ jobs, int n_aux, long long lo_shift,
                                                 float* __restrict__ Gs, int ldg) {
  const GSJob jb = jobs[blockIdx.y];
  const int nch = (n_aux + tc::CHUNK - 1) / tc::CHUNK;
  const long long w = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (w >= (long long)jb.r * nch) return;   // warp-uniform
  const int mu = (int)(w / nch), P = (int)(w % nch) * tc::CHUNK + (threadIdx.x & 31);
  const float* g = jb.G + (size_t)mu * n_aux + P;
  float v[tc::NSL];
  tc::warp_fixed_slices(P < n_aux ? (double)g[0] + (double)g[lo_shift] : 0.0, v);
  if (P < n_aux)
#pragma unroll
    for (int s2 = 0; s2 < tc::NSL; s2++) Gs[(size_t)(jb.x_row + s2 * jb.r + mu) * ldg + P] = v[s2];
}

void launch_gslices(const GSJob* jobs, int n_jobs, int max_r, int n_aux, long long lo_shift, float* Gs, int ldg,
                    cudaStream_t st) {
  if (!n_jobs) return;
  const long long warps = (long long)max_r * ((n_aux + tc::CHUNK - 1) / tc::CHUNK);
  k_gslices<<<dim3((unsigned)((warps + 7) / 8), n_jobs), 256, 0, st>>>(jobs, n_aux, lo_shift, Gs, ldg);
  note_launch(1);
}

// out[row][col] = hi + lo (row-major)
struct EpiRow {
  static constexpr bool kWarp = false;
  __device__ __forceinline__ void operator()(const tc::Job& jb, int r, int c, float h, float l) const {
    static_cast<float*>(jb.out)[(size_t)r * jb.ld_out + c] = h + l;
  }
};

// out[row][col] = hi + lo in FP64 (row-major): K~ from the slices of G
struct EpiRow64 {
  static constexpr bool kWarp = false;
  __device__ __forceinline__ void operator()(const tc::Job& jb, int r, int c, float h, float l) const {
    static_cast<double*>(jb.out)[(size_t)r * jb.ld_out + c] = (double)h + (double)l;
  }
};

namespace {
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}
}  // namespace

// 2-D FP32 map over rows x n_k (row stride ldk floats), 128-byte swizzle, box 32 x box_rows.
bool make_slice_map(CUtensorMap* m, const float* base, int n_k, int ldk, long long rows, int box_rows) {
  auto enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)n_k, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ldk * 4};
  cuuint32_t box[2] = {(cuuint32_t)tc::BK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int launch_gproj_tc(const float* Bs, long long a_rows, const float* Us, long long b_rows, int n_vir, int ldv,
                    const tc::Job* jobs, int n_jobs, long long lo_shift, int* err, cudaStream_t st) {
  if (!n_jobs) return 0;
  if (cudaFuncSetAttribute(tc::k_tf32x3<EpiG2>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM) !=
      cudaSuccess)
    return -1;
  CUtensorMap ma, mb;
  if (!make_slice_map(&ma, Bs, n_vir, ldv, a_rows, tc::BM) || !make_slice_map(&mb, Us, n_vir, ldv, b_rows, tc::BROWS))
    return -1;
  tc::k_tf32x3<EpiG2><<<tc::persistent_grid(n_jobs), tc::NTHREADS, tc::SMEM, st>>>(ma, mb, jobs, n_jobs, n_vir, err, EpiG2{lo_shift});
  note_launch(1);
  return 0;
}

int launch_kt_tc(const float* Gs, long long rows, int n_aux, int ldg, const tc::Job* jobs, int n_jobs, int* err,
                 cudaStream_t st) {
  if (!n_jobs) return 0;
  if (cudaFuncSetAttribute(tc::k_tf32x3<EpiRow64>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM) !=
      cudaSuccess)
    return -1;
  CUtensorMap ma, mb;
  if (!make_slice_map(&ma, Gs, n_aux, ldg, rows, tc::BM) || !make_slice_map(&mb, Gs, n_aux, ldg, rows, tc::BROWS))
    return -1;
  tc::k_tf32x3<EpiRow64><<<tc::persistent_grid(n_jobs), tc::NTHREADS, tc::SMEM, st>>>(ma, mb, jobs, n_jobs, n_aux, err, EpiRow64{});
  note_launch(1);
  return 0;
}

int launch_rows_tc(const float* A, long long a_rows, const float* B, long long b_rows, int n_vir, int ldv,
                   const tc::Job* jobs, int n_jobs, int* err, cudaStream_t st) {
  if (!n_jobs) return 0;
  if (cudaFuncSetAttribute(tc::k_tf32x3<EpiRow>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM) !=
      cudaSuccess)
    return -1;
  CUtensorMap ma, mb;
  if (!make_slice_map(&ma, A, n_vir, ldv, a_rows, tc::BM) || !make_slice_map(&mb, B, n_vir, ldv, b_rows, tc::BROWS))
    return -1;
  tc::k_tf32x3<EpiRow><<<tc::persistent_grid(n_jobs), tc::NTHREADS, tc::SMEM, st>>>(ma, mb, jobs, n_jobs, n_vir, err, EpiRow{});
  note_launch(1);
  return 0;
}

}  // namespace osv
