// Internal interfaces between the host runtime (api.cu) and the kernel
// translation units of libosvmp2.  Not part of the C ABI.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include "common.cuh"
#include "tc_job.h"

namespace osv {

// Device-resident lookup tables of the pair store (all pointers are device).
struct Tables {
  int n_occ;
  int n_vir;
  const int* n_osv;             // [n_occ]
  const double* const* Q;       // [n_occ] -> Q_i [n_vir][n_osv_i]
  const int* sf_id;             // [n_occ*n_occ]: (x<=y) -> S/F block id, -1 if absent
  const double* const* S;       // [n_blocks] S_(x,y) [n_x][n_y]
  const double* const* F;       // [n_blocks] F_(x,y)
  const int* pair_id;           // [n_occ*n_occ]: (i<=j) -> pair id, -1 if absent
  const double* const* K;       // [n_pairs] K_(ij,ij) [m][m]
  const double* const* X;       // [n_pairs] X [m][m] (first r columns valid)
  const double* const* et;      // [n_pairs] e~ [m] (first r valid)
  const int* r;                 // [n_pairs]
  const double* const* Kt;      // [n_pairs] K~ = X^T K X  [r][r]
  const float* const* U;        // [n_pairs] mixed form: U = P X  [n_vir][r] (FP32)
  const float* const* Sh;       // [n_pairs] mixed form: X^T S X - 1 [r][r] (FP32), NULL if X is exact
  const float* const* Gh;       // [n_pairs] mixed form: X^T F X - diag(e~) - (f_ii+f_jj)/2 Sh [r][r]
  const double* f_occ;          // [n_occ][n_occ]
};

// Process-wide count of kernel launches issued by the library.
void note_launch(int n);

struct SolveOpts {
  double tol_update, tol_energy;
  int max_iter;
  int tiles;      // mixed solver: tile set of its FP32 contractions (cta_gemm_f32s)
};

// Per-fragment result record written by the solvers.
struct FragOut {
  double energy;
  double umax;
  int iters;
  int status;   // 0 ok, ERR_* bits otherwise
};

// ---- A0 (osv_build.cu)
// T_ii of orbitals [i0, i0+nb) into T [nb][nv][nv].
void launch_tii(const BSrc& src, const double* e_vir, const double* f_occ, int n_occ, int i0, int nb,
                double* T, cudaStream_t st);
// Mixed form (tii_tc.cu): slices of B_i along the aux index for orbitals
// [i0, i0+nb): slot u, slice s, row a at Bt + ((u * tc::NSL + s) * n_vir + a) * ldx;
// then the tensor-core tiles of T (jobs built by the host, out = T_i, s = 2 f_ii).
void launch_rslices(const BSrc& src, int i0, int nb, float* Bt, int ldx, cudaStream_t st);
int launch_tii_tc(const float* Bt, long long rows, int n_aux, int ldx, const tc::Job* jobs, int n_jobs,
                  const double* e_vir, int* err, cudaStream_t st);
// Eigen-decomposition of each T[b] and selection omega >= thr (all if thr <= 0),
// at most kmax per orbital: V [nb][kmax][nv] (eigenvector-major), w [nb][kmax], k [nb], err |= ERR_*.
// d, e, tau (3 nv) + Z (nv*nv, full path) or the tridiagonalisation's partial sums,
// then 4 groups x 176 nv of lane-batched inverse iteration (top-k path)
// Per-orbital scratch of k_eig_osv: d, e, tau; the work room (Z, partial sums,
// inverse-iteration factors); the kept vectors as double-float pairs (mixed form).
__host__ __device__ inline size_t eig_osv_work_doubles(int nv) {
  return (size_t)nv * nv > (size_t)4 * 176 * nv ? (size_t)nv * nv : (size_t)4 * 176 * nv;
}
__host__ __device__ inline size_t eig_osv_scratch_doubles(int nv, int kmax) {
  return (size_t)3 * nv + eig_osv_work_doubles(nv) + (size_t)kmax * nv + 64;
}
// dfl_tridiag: the top-k path tridiagonalises in double-float arithmetic (the
// mixed-form OSV build, whose T_ii is a split-precision product).
void launch_eig_osv(double* T, int nb, int nv, double thr, int kmax, double* V, double* w, int* k,
                    double* scratch, int* err, bool dfl_tridiag, cudaStream_t st);
// Back-transformation of the kept eigenvectors of the top-k path (n_vir above
// the shared-memory limit, thr > 0) after launch_eig_osv; a no-op otherwise.
void launch_eig_back(double* T, int nb, int nv, double thr, int kmax, double* V, const int* k, double* scratch,
                     bool dfl_tridiag, cudaStream_t st);
// Randomized OSVs (rosv.cu; Algorithm 3) for a batch of nb orbitals with T_ii in
// T [nb][nv][nv].  Scratch layout (offsets in doubles) from rosv_layout; the
// Gaussian draw k of orbital i, entry a, is the Irwin-Hall normal of counter
// (i * ROSV_ROWS_PER_ORBITAL + k) * nv + a on the key of stream 7 of the seed.
constexpr uint64_t ROSV_ROWS_PER_ORBITAL = 1ull << 16;
constexpr int ROSV_WINDOW = 10;   // look-ahead rows r of the range finder
struct RosvLayout {
  int rows;                 // r + n_max Gaussian rows per orbital
  size_t y, z, tt, svd, svd_per, wmax, nrows, total;
  int ldk;                  // row stride of the TF32 slice store (mixed form)
  long long store_rows;     // rows of the slice store: nb * NSL * (nv + rows)
};
RosvLayout rosv_layout(int nb, int nv, int r, int n_max, int kmax);
// FP64 form: out[u] = A_u T_u with A_u the Gaussian rows (mode 0, rows rows) or
// Z_u (mode 1, nrows[u] of n_max = rows rows).
void launch_rosv_gemm64(int mode, const double* T, int nb, int nv, int i0, uint64_t key, const double* Z,
                        const int* nrows, int rows, double* out, cudaStream_t st);
// Mixed form: TF32 slices (K = nv) of T rows (part 0), Gaussian rows (1) or Z rows (2).
void launch_rosv_slices(int part, const double* T, int nb, int nv, int i0, uint64_t key, const double* Z,
                        int z_rows, const int* nrows, int rows, float* slices, int ldk, cudaStream_t st);
void launch_rosv_finder(double* Y, int nb, int nv, int r, int n_max, double l_osv, double* Z, int* nrows,
                        double* wmax, int* err, cudaStream_t st);
// FP64 form: M[u] = T~ T~^T ([nb][ldm][ldm], zero outside nrows[u]).
void launch_rosv_gram64(const double* Tt, const int* nrows, int nb, int nv, int n_max, int ldm, double* M,
                        cudaStream_t st);
// Q = Q~^T Z and omega = sqrt(eigenvalues of M) for the ks[u] kept eigenvectors Vs ([nb][ldm][ldm]).
void launch_rosv_backq(const double* Vs, const double* ws, const int* ks, const double* Z, const int* nrows, int nb,
                       int nv, int n_max, int ldm, int kmax, double* V, double* w, int* k, cudaStream_t st);
// Copy V[b][:, :k_b] into the packed Q store (Q[i0+b] as [nv][k]).
void launch_pack_q(const double* V, const double* w, int nb, int nv, int kmax, const int* k,
                   double* const* Qdst, double* const* wdst, cudaStream_t st);

// ---- A1-A2 (pair_integrals.cu)
struct ProjJob {         // B~_{i}^{(x)} = B[i]^T Q_x  -> out [n_aux][n_x]
  int i, x;
  double* out;
};
void launch_project(const BSrc& src, const Tables& t, const ProjJob* jobs, int n_jobs, int max_nx, int fp32,
                    cudaStream_t st);
struct KJob {            // K_(ij,ij) from the projections
  int i, j;
  const double* Bii;     // B~_i^(i)  [n_aux][n_i]
  const double* Bij;     // B~_i^(j)  [n_aux][n_j]   (NULL if i == j)
  const double* Bji;     // B~_j^(i)
  const double* Bjj;     // B~_j^(j)
  double* out;           // [m][m]
};
void launch_exchange(const Tables& t, int n_aux, const KJob* jobs, int n_jobs, int max_m, int fp32, cudaStream_t st);
struct SFJob {           // S_(x,y), F_(x,y)
  int x, y;
  double* S;
  double* F;
};
void launch_sf(const Tables& t, const double* e_vir, const SFJob* jobs, int n_jobs, int max_n,
               cudaStream_t st);

// ---- A3 (precond.cu)
struct PJob {            // preconditioner of pair (i,j): X, e~, r (+ the mixed form's leftovers)
  int i, j;
  double* X;
  double* et;
  int* r;
  float* Sh;             // mixed form only: X^T S X - 1          [r][r]
  float* Gh;             // mixed form only: X^T F X - diag(e~) - (f_ii+f_jj)/2 Sh
};
__host__ __device__ inline size_t precond_scratch_doubles(int max_m) {
  return 6 * (size_t)max_m * max_m + 4 * (size_t)max_m + 64;
}
void launch_precond(const Tables& t, double tau_s, const PJob* jobs, int n_jobs, int max_m, double* scratch,
                    int n_cta, int* err, cudaStream_t st);
// One warp per pair (pair order <= 192); returns -1 if max_m is too large.
size_t precond_w_scratch_doubles(int max_m, int n_warps);
int launch_precond_w(const Tables& t, double tau_s, const PJob* jobs, int n_jobs, int max_m, double* scratch,
                     int n_warps, int* err, cudaStream_t st);
// Mixed form (precond_mixed.cu): block-structured canonical orthogonalisation in
// FP64, F' diagonalised in FP32, exact leftovers Sh/Gh; -1 if max_m is too large.
// Per-pair intermediates: one slot of precond_mixed_slot_doubles(m) at slots + off[job];
// mdim[job] = pair order m; order: the jobs in the order the CTAs take them
// (grid-stride; descending m balances the launch).
size_t precond_mixed_slot_doubles(int m);
size_t precond_mixed_scratch_doubles(int max_m, int n_cta);
int launch_precond_mixed(const Tables& t, double tau_s, const PJob* jobs, const int* order, int n_jobs, int max_m,
                         double* slots, const long long* off, const int* mdim, double* scratch, int n_cta, int* err,
                         cudaStream_t st);

// ---- A4-A5 (solve.cu)
// Fragments: orbs [n][3] (-1 padded, ascending), order[] = processing order.
// per CTA: T, R, G1, G2 for six pairs + two work matrices
__host__ __device__ inline size_t frag_scratch_doubles(int max_m) { return 26 * (size_t)max_m * max_m + 64; }
// Tstore (may be NULL): converged amplitudes of fragment f are written at
// Tstore + Toff[f], local pairs (a<=b) in order, each m_p x m_p.
void launch_frag_solve(const Tables& t, const int* frag_orbs, const int* order, int n_frag, int max_m,
                       SolveOpts o, double* scratch, int n_cta, int* counter, FragOut* out,
                       double* Tstore, const long long* Toff, cudaStream_t st);
// Mixed-form pair build (ubasis.cu) in the orthonormal pair basis U = P X.
struct UJob {
  int i, j;
  float* U;            // [n_vir][r]
  float* Us;           // TF32 slices of U^T (tf32_split.cuh): slice s row mu at Us + (s * r + mu) * ldv
  int ldv;
};
struct GJob {          // G = U^T B_x  [r][n_aux]
  int x, r;
  const float* U;
  float* G;
};
void launch_ubasis(const Tables& t, const UJob* jobs, int n_jobs, int n_cta, double* scratch, int max_r,
                   cudaStream_t st);
// B_x for the orbitals xs[0..n_x) as TF32 slices (tf32_split.cuh), transposed:
// slot u, slice s, row P at Bs + ((u * tc::NSL + s) * n_aux + P) * ldv
void launch_bslices(const BSrc& src, const int* xs, int n_x, float* Bs, int ldv, cudaStream_t st);
// G tiles with the split-TF32 tensor-core kernel: A = Bs (rows a_rows), B = Us (rows b_rows), K = n_vir;
// G is written as a normalised FP32 pair: the leading part at job.out, the remainder
// lo_shift floats further on.  Returns 0, or -1 if a tensor map could not be encoded.
int launch_gproj_tc(const float* Bs, long long a_rows, const float* Us, long long b_rows, int n_vir, int ldv,
                    const tc::Job* jobs, int n_jobs, long long lo_shift, int* err, cudaStream_t st);
// The slices of G^T from the pair (G, lo): slice s of row mu at Gs[(x_row + s r + mu) ldg + P].
struct GSJob {
  const float* G;      // [r][n_aux], remainder at G + lo_shift
  int r, x_row;
};
void launch_gslices(const GSJob* jobs, int n_jobs, int max_r, int n_aux, long long lo_shift, float* Gs, int ldg,
                    cudaStream_t st);
// K~ = G_i G_j^T tiles from the slices in Gs (rows in total, K = n_aux), FP64 row-major output.
int launch_kt_tc(const float* Gs, long long rows, int n_aux, int ldg, const tc::Job* jobs, int n_jobs, int* err,
                 cudaStream_t st);
// 2-D FP32 tensor map over rows x n_k (row stride ldk floats, a multiple of 4),
// 128-byte swizzle, box tc::BK x box_rows; false if the driver rejects it.
bool make_slice_map(CUtensorMap* m, const float* base, int n_k, int ldk, long long rows, int box_rows);

// Mixed form (solve_mixed.cu): per pair K~ = X^T K X, then the fragment solve in
// the preconditioner basis with FP32 coupling products.
struct KtJob {
  int i, j;
  double* Kt;
};
void launch_ktilde(const Tables& t, const KtJob* jobs, int n_jobs, double* scratch, int n_cta, int max_m,
                   cudaStream_t st);
// per CTA: Y, 1/D (6 + 6 FP64), C as (hi, lo) (12 FP32) + Y32 (6 FP32) + 3 work (FP32) + G0 (6 max_m FP32)
__host__ __device__ inline size_t frag_mixed_scratch_doubles(int max_m) {
  const size_t M2 = (size_t)max_m * max_m;
  return 24 * M2 + (15 * M2 + 6 * (size_t)max_m + 1) / 2 + 64;
}
// Pair-couple overlaps Sigma_(lo,hi) = U_lo^T U_hi (pair ids lo < hi) of one MBE
// call, stored [r_lo][r_hi] at base + pos[id]; the ids of couples (lo, *) are
// off[lo] .. off[lo+1]-1 with partner hi[id] ascending.
struct SigmaTable {
  const int* off;
  const int* hi;
  const long long* pos;
  const float* base;
};
void launch_frag_solve_mixed(const Tables& t, const int* frag_orbs, const int* order, int n_frag, int max_m,
                             SolveOpts o, const SigmaTable& sgt, double* scratch, int n_cta, int* counter,
                             FragOut* out, double* Tstore, const long long* Toff, int* err, int ctas_per_sm,
                             cudaStream_t st);
// Row-major tiles of U-slice products (gproj_tc.cu): out[row * ld_out + col] = A_row . B_col,
// A and B tensor maps over (possibly different) U slice stores with K = n_vir.
int launch_rows_tc(const float* A, long long a_rows, const float* B, long long b_rows, int n_vir, int ldv,
                   const tc::Job* jobs, int n_jobs, int* err, cudaStream_t st);

// E = sum_f w_f * E_f in a fixed order -> e_out (device scalar)
void launch_weighted_sum(const FragOut* out, const int* weights, int n, double* e_out, cudaStream_t st);

// General subsystem solve: one kernel per Jacobi sweep over pairs.
struct SubDev {
  int nc;
  const int* orbs;          // [nc]
  double* const* T;         // [np] amplitude per local pair
  double* const* R;         // [np]
  double* const* G1;        // [np] F_p - f_ii S_p
  double* const* G2;        // [np] F_p - f_jj S_p
  double* const* W;         // [n_cta] work matrices (2 per CTA: W, Rt)
  double* pe;               // [np] pair energies
  double* pu;               // [np] pair max|update|
};
void launch_sub_prepare(const Tables& t, const SubDev& s, int np, int n_cta, cudaStream_t st);
void launch_sub_residual(const Tables& t, const SubDev& s, int np, int n_cta, cudaStream_t st);
void launch_sub_update(const Tables& t, const SubDev& s, int np, int n_cta, cudaStream_t st);

// ---- A6 (grad.cu)
struct GradContrib {       // one fragment's amplitude of a pair and the fragment weight
  const double* T;
  int weight;
};

// ---- occupied-orbital localization (localize.cu; Algorithm 2)
// P: scratch [n][n][n_atom]; U out [n][n]; out[0] = L, out[1] = last dL; status[0] = sweeps,
// status[1] = 1 if converged (device).
void launch_pm_localize(const double* C, int n_ao, int n, const int* atom_ao, int n_atom, double l_loc, int max_sweeps,
                        double* P, double* U, double* out, int* status, int num_sms, cudaStream_t st);
// The same sweeps over a cooperative grid (atoms spread over the CTAs, one bounded grid
// barrier per rotation); false when the grid cannot be co-resident (nothing launched
// then).  part: 4 * min(n_atom, num_sms) doubles; bar: 2 unsigned; err |= ERR_TIMEOUT
// if a barrier wait gave up.
bool launch_pm_localize_grid(const double* C, int n, const int* atom_ao, int n_atom, double l_loc, int max_sweeps,
                             double* P, double* U, double* out, int* status, double* part, unsigned* bar, int* err,
                             int num_sms, cudaStream_t st);

// ---- pair screening and weak pairs (screen.cu), FP64 in both forms
// s2b[p] of the pairs (i, j) = pairs[p] (Eq. s2b), grid-stride over n_cta CTAs.
void launch_s2b(const Tables& t, const int2* pairs, int n_pairs, double* s2b, int n_cta, cudaStream_t st);
struct DiagJob {           // T_ii (raw basis, [n_i][n_i]) = sum of contributions [c0, c1)
  int i, pid;              // orbital, id of the pair (i, i)
  int c0, c1;
  double* T;
};
// mixed != 0: contributions are Y (r x r) of the pair (i,i)'s preconditioner basis.
// scratch: 2 max_n^2 doubles per CTA.
void launch_diag_amp(const Tables& t, const DiagJob* jobs, int n_jobs, const GradContrib* contrib, int mixed,
                     double* scratch, int max_n, int n_cta, cudaStream_t st);
struct WeakJob {           // weak pair (i, j), i < j
  int i, j;
  const double* Bii;       // B~_i^(i) [n_aux][n_i]
  const double* Bjj;       // B~_j^(j) [n_aux][n_j]
  const double* S;         // S_(i,j) [n_i][n_j]
  const double* Ti;        // MBE(3) diagonal amplitude T_(i,i) [n_i][n_i]
  const double* Tj;
  const double* Xi;        // eigenbasis of F_(i,i) (columns; exact in the FP64 form, the mixed
  const double* Xj;        //   preconditioner basis of the pair (i,i) otherwise), row stride ldxi
  const double* ei;        // their eigenvalues
  const double* ej;
  int ldxi, ldxj;
  const double* Fi;        // F_(i,i) [n_i][n_i], F_(j,j) (mixed form's residual updates)
  const double* Fj;
};
// Weak-pair energies (both orders) into e_out[job]; scratch: 6 max_n^2 doubles per CTA.
void launch_weak(const Tables& t, int n_aux, const WeakJob* jobs, int n_jobs, double* scratch, int max_n, int n_cta,
                 double* e_out, int mixed, cudaStream_t st);
// Mixed form: B~_i^(i) = B_i^T Q_i in double-float for the jobs (i, x = i, out [n_aux][n_i]).
void launch_project_df(const BSrc& src, const Tables& t, const ProjJob* jobs, int n_jobs, cudaStream_t st);
struct GradPairJob {       // W_p = sum c T~, H_p = sum c (T~ S T^T + [i!=j] T~^T S T)
  int i, j;
  int c0, c1;              // contributions [c0, c1)
  double* W;
  double* H;
};
struct GradYTerm {         // rows [row0, row0+n_x) of W'_p (W or W^T) times P_p^T B_partner
  int pi, pj;
  int trans;
  int row0;
  const double* W;
  const double* Bt_i;      // B~_partner^(pi)  [n_aux][n_pi]
  const double* Bt_j;      // B~_partner^(pj)  [n_aux][n_pj]  (unused when pi == pj)
};
struct GradYJob {          // Y_o^(x) [n_x][n_aux] = sum of terms [t0, t1)
  int o, x;
  int t0, t1;
  double* Y;
};
struct GradBTerm {
  int x;
  const double* Y;
};
struct GradBJob {          // dB_i = 4 sum_x Q_x Y_i^(x) over terms [t0, t1)
  int i;
  int t0, t1;
};
void launch_grad_pair(const Tables& t, const GradPairJob* jobs, int n_jobs, const GradContrib* contrib,
                      double* scratch, int n_cta, int max_m, cudaStream_t st);
void launch_grad_de(const Tables& t, const GradPairJob* jobs, int n_jobs, double* scratch, int n_cta, int max_m,
                    double* dpair, double* de, cudaStream_t st);
void launch_grad_df(const Tables& t, const int* frag_orbs, const int* weights, const double* Tstore,
                    const long long* Toff, int n_frag, int max_m, double* scratch, int n_cta, double* gfrag,
                    const int* fptr, const int* flist, double* df, cudaStream_t st);
void launch_grad_Y(const Tables& t, int n_aux, const GradYJob* jobs, int n_jobs, const GradYTerm* terms, int max_n,
                   cudaStream_t st);
void launch_grad_dB(const Tables& t, int n_aux, const GradBJob* jobs, int n_jobs, const GradBTerm* terms, double* dB,
                    cudaStream_t st);

// ---- A6, OSV-relaxed part (grad_relax.cu)
struct RelaxKJob {          // exchange part of dP_(i,j): alpha [B_i (A_j W~^T) + B_j (A_i W~)]
  int i, j;
  const double* W;          // W~ = sum_C c_C T~ [m][m]
  const double* bt_ii;      // B_i^T Q_i [n_aux][n_i]
  const double* bt_ij;      // B_i^T Q_j (unused for i = j)
  const double* bt_ji;      // B_j^T Q_i
  const double* bt_jj;      // B_j^T Q_j
  double* out;              // [n_vir][m]
};
struct RelaxFragJob {       // the rest of dP for every pair of one fragment
  int orbs[3];
  int no;
  double c;                 // fragment weight
  const double* T;          // the fragment's amplitudes, pairs (a <= b) in order
  double* slot[3];          // [n_vir][n_x] per orbital of the fragment
};
struct RelaxGTerm {         // a block of columns added into G_x
  const double* p;
  int ld, col0;
};
struct RelaxGJob {          // G_x = dE/dQ_x [n_vir][n_x] = sum of terms [t0, t1)
  int x;
  int t0, t1;
  double* G;
};
struct RelaxRJob {          // eigenvector response of orbital x
  int x;
  const double* V;          // all eigenvectors of T_xx, eigenvector-major, descending eigenvalues
  const double* w;          // [n_vir] eigenvalues, descending
  const double* T;          // T_xx [n_vir][n_vir]
  const double* G;          // dE/dQ_x [n_vir][n_x]
  double* Z;                // [n_vir][n_vir]: the adjoint of T_xx, then Z / D
  double* Y;                // [n_vir - n_x][n_x]
  double* Xr;               // [n_vir][n_x]
  double* de;               // [n_vir]
  double* df;               // [1]
};
void launch_relax_kpart(const Tables& t, const BSrc& bs, const RelaxKJob* jobs, int n_jobs, double* scratch,
                        int n_cta, int max_m, cudaStream_t st);
void launch_relax_frag(const Tables& t, const double* e_vir, const RelaxFragJob* jobs, int n_jobs, double* scratch,
                       size_t scr_per, int n_cta, int max_m, cudaStream_t st);
void launch_relax_gather(int n_vir, const int* n_osv, const RelaxGJob* jobs, int n_jobs, const RelaxGTerm* terms,
                         cudaStream_t st);
void launch_relax_resp(const Tables& t, const BSrc& bs, const double* e_vir, const RelaxRJob* jobs, int nb,
                       double* dB, double* de, double* df, cudaStream_t st);
void launch_grad_de_reduce(const double* dpair, int n_pairs, int nv, double* de, cudaStream_t st);
void launch_grad_df_reduce(const Tables& t, const int* frag_orbs, const double* gfrag, int n_frag, const int* fptr,
                           const int* flist, double* df, cudaStream_t st);

// ---- A6, mixed form (grad_mixed.cu): Tstore holds Y_p (T_p = X_p Y_p X_p^T)
struct GradZJob {          // Z = op(W~) G  [r][n_aux]
  int r;
  int trans;
  const double* W;
  const float* G;
  float* Z;
};
struct GradMBTerm {        // U_p [n_vir][r] times Z [r][n_aux]
  int r;
  const float* U;
  const float* Z;
};
void launch_gradm_pair(const Tables& t, const GradPairJob* jobs, int n_jobs, const GradContrib* contrib,
                       double* scratch, int n_cta, int max_m, cudaStream_t st);
void launch_gradm_de(const Tables& t, const GradPairJob* jobs, int n_jobs, double* scratch, int n_cta, int max_m,
                     double* dpair, double* de, cudaStream_t st);
void launch_gradm_df(const Tables& t, const int* frag_orbs, const int* weights, const double* Tstore,
                     const long long* Toff, int n_frag, int max_m, double* scratch, int n_cta, double* gfrag,
                     const int* fptr, const int* flist, double* df, cudaStream_t st);
void launch_gradm_Z(int n_aux, const GradZJob* jobs, int n_jobs, int max_r, cudaStream_t st);
void launch_gradm_dB(int n_vir, int n_aux, const GradBJob* jobs, int n_jobs, const GradMBTerm* terms, double* dB,
                     cudaStream_t st);

}  // namespace osv
