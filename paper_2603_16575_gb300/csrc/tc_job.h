// One output tile of the split-TF32 tensor-core contraction (tc_tf32x3.cuh).
#pragma once

namespace osv {
namespace tc {

constexpr int BM = 128;    // tile rows = TMEM lanes = MMA M
constexpr int BN = 64;     // max tile columns (MMA N <= 64)
constexpr int NSL = 4;     // fixed-point slices per operand (tf32_split.cuh)
constexpr int CHUNK = 32;  // k-extent that shares one power-of-two scale per row

struct Job {
  int a_row, a_sstride;    // A slice s: rows a_row + s * a_sstride + [0, 128) of the A tensor map
  int b_row, b_sstride;    // B slice s: rows b_row + s * b_sstride + [0, n) of the B tensor map
  int m_valid, n_valid;    // output rows (<= 128) and columns (<= 64) to store
  void* out;               // output of the epilogue (its layout is the epilogue's)
  int ld_out;
  int m0, n0;              // global row / column of the tile's first element
  double s;                // epilogue scalar
  int x_row, x_sstride;    // slice-writing epilogues: row of slice 0 of the output, rows per slice
};

}  // namespace tc
}  // namespace osv
