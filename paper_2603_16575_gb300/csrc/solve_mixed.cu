// A4 in the mixed form.  Algorithm 7 updates T_p += X_p (R~_p / D_p) X_p^T with
// R~_p = X_p^T R_p X_p.  Writing T_p = X_p Y_p X_p^T (T starts at 0 and every
// update lies in the span of X_p), Eq. (res_close) becomes, in the
// preconditioner basis,
//     R~_p = K~_p - D_p o Y_p + C_p,   C_p = sum_terms c_t Sigma_pq op(Y_q) Sigma_pq^T,
// with K~_p = X_p^T K_p X_p, Sigma_pq = X_p^T S_(p,q) X_q = U_p^T U_q (entries
// bounded by 1, since U_p = P_p X_p has orthonormal columns) and D_p the update denominators; the
// pair-diagonal F/S terms collapse to -D o Y exactly (X^T S X = 1,
// X^T F X = diag(e~)).  The update is Y_p <- (K~_p + C_p) / D_p.
//
// When the preconditioner basis is only approximate (X^T S X = 1 + Sh,
// X^T F X = diag(e~) + Fh, see precond_mixed.cu) the pair-diagonal terms give
// -D o Y_p + P_p(Y_p) with P = Gh (Y S~) + (S~ Y) Gh + G0 (Y Sh) + (Sh Y) G0,
// Gh = Fh - (f_ii+f_jj)/2 Sh, G0 = diag(e~) - (f_ii+f_jj)/2; P is added to C_p,
// so the fixed point is the exact one.  Sh and Gh are ~1e-7, their products FP32;
// P is linear in Y and that small, so it is re-formed only after the
// amplitudes have moved by more than P_LAG of their scale (in practice the
// first two or three sweeps), and the fixed point is exact up to P applied to
// that lag.
//
// Precision: the coupling C_p carries the off-diagonal occupied Fock elements
// (|c_t| ~ 1e-2 against |D| ~ 1), so the rounding of its FP32 products perturbs
// Y by ~ eps_32 |c| / |D| ~ 1e-9 relative.  The coupling products are FP32 (K =
// a pair order), Sigma_pq comes from the split-precision table, and C_p is
// accumulated over its terms in a compensated FP32 pair (two-sum: no FP64
// arithmetic, whose throughput is 1/64 of FP32 here).  K~_p, 1/D_p and Y_p (master
// copy) are double-float pairs (~48 bits), and so are the update and the energy
// <K~_p, 2Y_p - Y_p^T>.  The energy sum over the pairs and fragments is FP64.
#include "pairview.cuh"

namespace osv {

// K~_p = X_p^T K_p X_p (FP64), one CTA per pair (grid-stride).
__global__ void __launch_bounds__(NT) k_ktilde(Tables t, const KtJob* __restrict__ jobs, int n_jobs, double* scratch,
                                               int max_m) {
  __shared__ double sm[GEMM_SMEM_DOUBLES];
  double* W = scratch + (size_t)blockIdx.x * max_m * max_m;
  for (int jid = blockIdx.x; jid < n_jobs; jid += gridDim.x) {
    const KtJob jb = jobs[jid];
    const int m = pair_dim(t, jb.i, jb.j);
    const int pid = t.pair_id[jb.i * t.n_occ + jb.j];
    const int r = t.r[pid];
    const View Xv = dense_view(t.X[pid], m, r, m);
    cta_gemm(m, r, m, 1.0, dense_view(t.K[pid], m, m, m), Xv, 0.0, W, r, sm);
    cta_gemm(r, r, m, 1.0, transpose(Xv), dense_view(W, m, r, r), 0.0, jb.Kt, r, sm);
  }
}

void launch_ktilde(const Tables& t, const KtJob* jobs, int n_jobs, double* scratch, int n_cta, int max_m,
                   cudaStream_t st) {
  if (!n_jobs) return;
  k_ktilde<<<n_cta, NT, 0, st>>>(t, jobs, n_jobs, scratch, max_m);
  note_launch(1);
}

struct MTerm {     // coupling of local pair p to stored pair q: Sigma[sig] (cn Y_q + ct Y_q^T) Sigma[sig]^T
  int q;           // local stored pair
  int sig;         // index of Sigma_(p,q) in the fragment's list
  double cn, ct;   // coefficients of Y_q and of Y_q^T (terms with the same q share one Sigma)
};

// cn Y + ct Y^T of a square FP32 block, read element by element by the GEMM tiles.
struct ViewFmix {
  const float* p;
  int ld;
  float cn, ct;
  __device__ __forceinline__ float get(int r, int c) const {
    return cn * p[(size_t)r * ld + c] + ct * p[(size_t)c * ld + r];
  }
  __device__ __forceinline__ bool row_major() const { return true; }
};

// P(Y) is refreshed once the amplitudes have moved by more than this fraction of
// their scale (max |Y| after the first sweep) since it was last formed: P is
// ~1e-7 of the pair-diagonal terms, so a lag of 1e-2 of Y leaves ~1e-9 of P's
// own contribution.
constexpr double P_LAG = 1e-2;

constexpr int MAX_TERMS = 24;   // 6 pairs x 4 coupling terms (three-orbital fragments)

// Sigma_(lo,hi) = U_lo^T U_hi of pair ids lo < hi, stored [r_lo][r_hi]: entry
// id of (lo, hi) is found in hi_id[off[lo] .. off[lo+1]) (ascending), its data
// at base + pos[id].
__device__ __forceinline__ const float* sigma_lookup(const SigmaTable& st, int lo, int hi) {
  int a = st.off[lo], b = st.off[lo + 1];
  while (a < b) {
    const int mid = (a + b) >> 1;
    if (st.hi[mid] < hi) a = mid + 1;
    else b = mid;
  }
  return (a < st.off[lo + 1] && st.hi[a] == hi) ? st.base + st.pos[a] : nullptr;
}

// MINB: resident CTAs per SM the registers are budgeted for (2: 128 registers; 3: 80, with spills)
template <int MINB>
__global__ void __launch_bounds__(NT, MINB) k_frag_solve_mixed(Tables t, const int* __restrict__ frag_orbs,
                                                         const int* __restrict__ order, int n_frag, int max_m,
                                                         SolveOpts o, SigmaTable sgt, double* scratch, int* counter,
                                                         FragOut* out, double* Tstore,
                                                         const long long* __restrict__ Toff, int* err) {
  __shared__ float fsm[GEMM_SMEM_F32];
  __shared__ double red[40];
  __shared__ int s_f;
  __shared__ MTerm terms[6][8];
  __shared__ int nterm[6];
  __shared__ int sig_p[MAX_TERMS], sig_q[MAX_TERMS];
  __shared__ int s_nsig;
  __shared__ const float* sig_ptr[MAX_TERMS];   // Sigma_pq = sig_ptr (ld sig_ld), transposed when sig_tr
  __shared__ int sig_ld[MAX_TERMS], sig_tr[MAX_TERMS];
  const size_t M2 = (size_t)max_m * max_m;
  double* base = scratch + (size_t)blockIdx.x * frag_mixed_scratch_doubles(max_m);
  // the amplitudes, 1/D and K~ as double-float pairs: the update and the energy
  // run on the FP32 pipes at ~48 bits
  dfl* Yd[6];
  float* Chi[6];            // C_p as a compensated FP32 pair (Chi + Clo)
  float* Clo[6];
  dfl* invD[6];
  dfl* Ktd[6];
  float* Y32[6];
  for (int u = 0; u < 6; u++) {
    Yd[u] = reinterpret_cast<dfl*>(base + u * M2);
    Chi[u] = reinterpret_cast<float*>(base + 6 * M2) + (size_t)u * M2;
    Clo[u] = reinterpret_cast<float*>(base + 6 * M2) + (size_t)(6 + u) * M2;
    invD[u] = reinterpret_cast<dfl*>(base + (12 + u) * M2);
    Ktd[u] = reinterpret_cast<dfl*>(base + (18 + u) * M2);
  }
  float* fb = reinterpret_cast<float*>(base + 24 * M2);
  for (int u = 0; u < 6; u++) Y32[u] = fb + u * M2;
  float* W32 = fb + 6 * M2;
  float* A1 = fb + 7 * M2;
  float* A2 = fb + 8 * M2;
  float* Pp[6];              // P_p(Y_p), refreshed when the amplitudes have drifted (FP32)
  for (int u = 0; u < 6; u++) Pp[u] = fb + (9 + u) * M2;
  float* G0[6];              // e~_a - (f_ii + f_jj)/2 per pair (FP32)
  for (int u = 0; u < 6; u++) G0[u] = fb + 15 * M2 + (size_t)u * max_m;
  const double* f = t.f_occ;
  const int n = t.n_occ;
  while (true) {
    if (threadIdx.x == 0) s_f = atomicAdd(counter, 1);
    __syncthreads();
    const int fi = s_f;
    __syncthreads();
    if (fi >= n_frag) break;
    const int fid = order[fi];
    int orbs[3];
    int nc = 0;
    for (int u = 0; u < 3; u++) {
      const int v = frag_orbs[3 * fid + u];
      if (v >= 0) orbs[nc++] = v;
    }
    const int np = nc * (nc + 1) / 2;
    int pa[6], pb[6], pm[6], pr[6], pid[6];
    for (int a = 0, lp = 0; a < nc; a++)
      for (int b = a; b < nc; b++, lp++) {
        pa[lp] = a;
        pb[lp] = b;
        pm[lp] = pair_dim(t, orbs[a], orbs[b]);
        pid[lp] = t.pair_id[orbs[a] * n + orbs[b]];
        pr[lp] = t.r[pid[lp]];
      }
    // coupling terms of every pair and the distinct (p, q) overlaps they use
    if (threadIdx.x == 0) {
      int ns = 0;
      for (int p = 0; p < np; p++) {
        const int a = pa[p], b = pb[p], i = orbs[a], j = orbs[b];
        int nt = 0;
        for (int c = 0; c < nc; c++) {
          const int k = orbs[c];
          for (int s2 = 0; s2 < 2; s2++) {
            int x, y;
            double coef;
            if (s2 == 0) {
              if (c == b) continue;
              x = a; y = c; coef = -f[k * n + j];
            } else {
              if (c == a) continue;
              x = c; y = b; coef = -f[i * n + k];
            }
            if (coef == 0.0) continue;
            const int qa = min(x, y), qb = max(x, y);
            const int q = qa * nc - qa * (qa - 1) / 2 + (qb - qa);
            int sg = -1;
            for (int u = 0; u < ns; u++)
              if (sig_p[u] == p && sig_q[u] == q) sg = u;
            if (sg < 0) { sg = ns; sig_p[ns] = p; sig_q[ns] = q; ns++; }
            int tu = -1;   // terms on the same q (Y_q and Y_q^T, diagonal pairs) share one product
            for (int u = 0; u < nt; u++)
              if (terms[p][u].q == q) tu = u;
            if (tu < 0) { tu = nt++; terms[p][tu] = MTerm{q, sg, 0.0, 0.0}; }
            if (x > y) terms[p][tu].ct += coef;
            else terms[p][tu].cn += coef;
          }
        }
        nterm[p] = nt;
      }
      s_nsig = ns;
    }
    __syncthreads();
    // Sigma_pq = X_p^T S_(p,q) X_q = U_p^T U_q from the table built before the
    // launch (split-precision tensor-core products, one per pair couple)
    for (int u = threadIdx.x; u < s_nsig; u += NT) {
      const int P = pid[sig_p[u]], Q = pid[sig_q[u]];
      const int lo = min(P, Q), hi = max(P, Q);
      const float* sp = sigma_lookup(sgt, lo, hi);
      if (!sp) atomicOr(err, ERR_SIZE);
      sig_ptr[u] = sp;
      sig_ld[u] = t.r[hi];
      sig_tr[u] = (P != lo);
    }
    __syncthreads();
    bool sig_ok = true;
    for (int u = 0; u < s_nsig; u++) sig_ok &= sig_ptr[u] != nullptr;
    for (int p = 0; p < np; p++) {
      const int rp = pr[p];
      const double fij = f[orbs[pa[p]] * n + orbs[pa[p]]] + f[orbs[pb[p]] * n + orbs[pb[p]]];
      const double* et = t.et[pid[p]];
      const double* Kt = t.Kt[pid[p]];
      for (int idx = threadIdx.x; idx < rp * rp; idx += NT) {
        Yd[p][idx] = dfl{0.f, 0.f};
        Y32[p][idx] = 0.f;
        Pp[p][idx] = 0.f;
        invD[p][idx] = df_from(1.0 / (fij - et[idx / rp] - et[idx % rp]));   // update denominators, once per fragment
        Ktd[p][idx] = df_from(Kt[idx]);
      }
      for (int a = threadIdx.x; a < rp; a += NT) G0[p][a] = (float)(et[a] - 0.5 * fij);
    }
    __syncthreads();
    double e_prev = 0.0, e = 0.0, um = 0.0;
    double y_scale = 0.0, drift = 0.0;   // max |Y| after the first sweep; max-norm moves since P was formed
    int status = ERR_NOCONV, iters = o.max_iter;
    for (int it = 1; it <= o.max_iter; it++) {
      // the first sweep starts from Y = 0: C = P = 0
      const bool refresh_P = it > 1 && drift > P_LAG * y_scale;
      if (refresh_P) drift = 0.0;
      // C_p from the previous sweep's amplitudes (Jacobi)
      for (int p = 0; p < np; p++) {
        const int rp = pr[p];
        for (int idx = threadIdx.x; idx < rp * rp; idx += NT) Chi[p][idx] = Clo[p][idx] = 0.f;
        __syncthreads();
        for (int u = 0; u < nterm[p] && sig_ok && it > 1; u++) {
          const MTerm tm = terms[p][u];
          const int rq = pr[tm.q];
          const ViewF S{sig_ptr[tm.sig], sig_ld[tm.sig], sig_tr[tm.sig]};        // Sigma_pq   (r_p x r_q)
          const ViewF St{sig_ptr[tm.sig], sig_ld[tm.sig], !sig_tr[tm.sig]};      // Sigma_pq^T (r_q x r_p)
          // W = (cn Y_q + ct Y_q^T) Sigma_pq^T, C_p += Sigma_pq W
          if (tm.ct == 0.0)
            cta_gemm_f32s<float>(rq, rp, rq, tm.cn, ViewF{Y32[tm.q], rq, 0}, St, 0.0, W32, rp, fsm, o.tiles);
          else if (tm.cn == 0.0)
            cta_gemm_f32s<float>(rq, rp, rq, tm.ct, ViewF{Y32[tm.q], rq, 1}, St, 0.0, W32, rp, fsm, o.tiles);
          else
            cta_gemm_f32s<float>(rq, rp, rq, 1.0, ViewFmix{Y32[tm.q], rq, (float)tm.cn, (float)tm.ct}, St, 0.0,
                                 W32, rp, fsm, o.tiles);
          cta_gemm_f32s_acc2(rp, rp, rq, 1.f, S, ViewF{W32, rp, 0}, Chi[p], Clo[p], rp, fsm, o.tiles);
        }
        // leftovers of an inexact preconditioner basis (S~ = 1 + Sh, G0 = diag(e~) - (f_ii+f_jj)/2):
        // P = Gh (Y S~) + (S~ Y) Gh + G0 (Y Sh) + (Sh Y) G0, from the amplitudes of the last refresh
        const float* Sh = t.Sh ? t.Sh[pid[p]] : nullptr;
        if (Sh && refresh_P) {
          const float* Gh = t.Gh[pid[p]];
          const float* g0 = G0[p];
          cta_gemm_f32s<float>(rp, rp, rp, 1.0, ViewF{Y32[p], rp, 0}, ViewF{Sh, rp, 0}, 0.0, A1, rp, fsm, o.tiles);
          cta_gemm_f32s<float>(rp, rp, rp, 1.0, ViewF{Sh, rp, 0}, ViewF{Y32[p], rp, 0}, 0.0, A2, rp, fsm, o.tiles);
          for (int idx = threadIdx.x; idx < rp * rp; idx += NT) {
            const int a = idx / rp, b = idx % rp;
            Pp[p][idx] = g0[a] * A1[idx] + g0[b] * A2[idx];
            A1[idx] += Y32[p][idx];
            A2[idx] += Y32[p][idx];
          }
          __syncthreads();
          cta_gemm_f32s<float>(rp, rp, rp, 1.0, ViewF{Gh, rp, 0}, ViewF{A1, rp, 0}, 1.0, Pp[p], rp, fsm, o.tiles);
          cta_gemm_f32s<float>(rp, rp, rp, 1.0, ViewF{A2, rp, 0}, ViewF{Gh, rp, 0}, 1.0, Pp[p], rp, fsm, o.tiles);
        }
      }
      // Y_p <- (K~_p + C_p) / D_p and the energy <K~_p, 2Y_p - Y_p^T>, double-float
      um = 0.0;
      e = 0.0;
      for (int p = 0; p < np; p++) {
        const int rp = pr[p];
        const dfl* Kd = Ktd[p];
        dfl* Y = Yd[p];
        float du = 0.f;
        for (int idx = threadIdx.x; idx < rp * rp; idx += NT) {
          float ch, cl;
          two_sum_f(Chi[p][idx], Clo[p][idx] + Pp[p][idx], ch, cl);
          const dfl y = df_mul(df_add(Kd[idx], dfl{ch, cl}), invD[p][idx]);
          const dfl yo = Y[idx];
          du = fmaxf(du, fabsf((y.h - yo.h) + (y.l - yo.l)));
          Y[idx] = y;
        }
        um = fmax(um, cta_max((double)du, red));
        float sh = 0.f, sl = 0.f;
        for (int idx = threadIdx.x; idx < rp * rp; idx += NT) {
          const int r = idx / rp, c = idx % rp;
          const dfl y = Y[idx];
          df_acc(sh, sl, Kd[idx], df_add(df_add(y, y), df_neg(Y[(size_t)c * rp + r])));
          Y32[p][idx] = y.h;
        }
        const double s = cta_sum((double)sh + (double)sl, red);
        e += (pa[p] == pb[p]) ? s : 2.0 * s;
      }
      if (!isfinite(e) || !isfinite(um)) { status = ERR_NONFINITE; iters = it; break; }
      if (it == 1) y_scale = um;
      drift += um;
      if (um < o.tol_update && fabs(e - e_prev) < fmax(o.tol_energy, 1e-11 * fabs(e))) {
        status = 0;
        iters = it;
        break;
      }
      e_prev = e;
    }
    if (threadIdx.x == 0) out[fid] = FragOut{e, um, iters, status};
    if (Tstore) {   // Y_p (r x r) for the gradient, in slots of m_p x m_p
      double* dst = Tstore + Toff[fid];
      for (int p = 0; p < np; p++) {
        const int rp = pr[p];
        for (int idx = threadIdx.x; idx < rp * rp; idx += NT) dst[idx] = df_to(Yd[p][idx]);
        dst += (size_t)pm[p] * pm[p];
      }
    }
    __syncthreads();
  }
}

void launch_frag_solve_mixed(const Tables& t, const int* frag_orbs, const int* order, int n_frag, int max_m,
                             SolveOpts o, const SigmaTable& sgt, double* scratch, int n_cta, int* counter,
                             FragOut* out, double* Tstore, const long long* Toff, int* err, int ctas_per_sm,
                             cudaStream_t st) {
  if (n_frag == 0) return;
  cudaMemsetAsync(counter, 0, sizeof(int), st);
  if (ctas_per_sm >= 3)
    k_frag_solve_mixed<3><<<n_cta, NT, 0, st>>>(t, frag_orbs, order, n_frag, max_m, o, sgt, scratch, counter, out,
                                                Tstore, Toff, err);
  else
    k_frag_solve_mixed<2><<<n_cta, NT, 0, st>>>(t, frag_orbs, order, n_frag, max_m, o, sgt, scratch, counter, out,
                                                Tstore, Toff, err);
  note_launch(1);
}

}  // namespace osv
