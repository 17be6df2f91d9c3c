// Views of the 4-block OSV pair matrices A_(ij,kl) = [Q_i Q_j]^T A [Q_k Q_l]
// (Eq. 4block_osv) over the stored blocks A_(x,y), x <= y; A_(y,x) = A_(x,y)^T.
#pragma once
#include "internal.h"

namespace osv {

__device__ __forceinline__ Blk sf_blk(const Tables& t, const double* const* tab, int x, int y) {
  if (x <= y) return Blk{tab[t.sf_id[x * t.n_occ + y]], t.n_osv[y], 0};
  return Blk{tab[t.sf_id[y * t.n_occ + x]], t.n_osv[x], 1};
}

// A_(ij,kl) for stored pairs i <= j, k <= l (a diagonal pair is one block).
__device__ __forceinline__ View pair_view(const Tables& t, const double* const* tab, int i, int j, int k, int l) {
  View v;
  const int ni = t.n_osv[i], nk = t.n_osv[k];
  v.rows = ni + (i != j ? t.n_osv[j] : 0);
  v.cols = nk + (k != l ? t.n_osv[l] : 0);
  v.rs = ni;
  v.cs = nk;
  v.b[0][0] = sf_blk(t, tab, i, k);
  v.b[0][1] = (k != l) ? sf_blk(t, tab, i, l) : v.b[0][0];
  v.b[1][0] = (i != j) ? sf_blk(t, tab, j, k) : v.b[0][0];
  v.b[1][1] = (i != j && k != l) ? sf_blk(t, tab, j, l) : ((i != j) ? v.b[1][0] : v.b[0][1]);
  return v;
}

__device__ __forceinline__ int pair_dim(const Tables& t, int i, int j) {
  return t.n_osv[i] + (i != j ? t.n_osv[j] : 0);
}

}  // namespace osv
