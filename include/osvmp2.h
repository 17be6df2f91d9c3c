/*
 * osvmp2.h -- C ABI of the GB300 MBE(3)-OSV-MP2 pair-solve library (libosvmp2.so).
 *
 * Method: Liang & Yang, "Multi-GPU MBE(3)-OSV-MP2 for Performant Large-Scale
 * ab initio Calculations" (arXiv 2603.16575).  The library computes, on one
 * GPU, the data-parallel path of that method:
 *   A0  OSVs of every occupied LMO (Eq. osv_gen from the semi-canonical T_ii of
 *       Eq. mp2_tkk), kept where omega >= l_osv                 -> osvmp2_build_osv
 *   A1  OSV projection of the RI integrals (Eq. osv_imua)
 *   A2  pair blocks K (Eq. osv_close_k), S and F (Eq. 4block_osv, Algorithm 5)
 *                                                              -> osvmp2_pair_integrals
 *   A3  preconditioner F X = S X E~ per pair (Eq. prec_eig)
 *   A4  residual iterations per fragment (Eq. res_close, Algorithm 7)
 *                                                              -> osvmp2_solve
 *   A5  MBE(3) energy (Eqs. tmbediag-deltaoff as fragment weights)
 *                                                              -> osvmp2_mbe3_energy
 *   A6  frozen-OSV adjoint dE/dB, dE/de_vir, dE/df             -> osvmp2_energy_grad
 *       the same with the OSV response (relaxed OSVs)           -> osvmp2_energy_grad_relaxed
 *
 * Conventions (all entry points):
 *   - Every function returns an osvmp2_status; nothing throws across the ABI.
 *     On failure osvmp2_last_error(ctx) gives a one-line reason.
 *   - Arrays are row-major, innermost index last, FP64 unless stated.
 *     "device" = memory of the ctx's GPU (cudaMalloc / torch CUDA tensors);
 *     "host" = ordinary CPU memory.  The caller owns every pointer it passes;
 *     the library never frees them and keeps no reference after the call
 *     returns, except the osvmp2_system arrays, which must stay valid and
 *     unchanged until the next osvmp2_build_osv or osvmp2_destroy.
 *   - Work is queued on the ctx's stream.  Calls that return host scalars
 *     (energies, counts) synchronise that stream before returning.
 *   - Memory the method needs between calls (OSVs, projected integrals, pair
 *     blocks, preconditioners, amplitudes, workspace) is owned by the ctx and
 *     allocated with cudaMalloc on the ctx's device; OSVMP2_E_NOMEM if that fails.
 *   - A ctx is not thread-safe; use one ctx per host thread.
 *   - Energies are in Hartree, distances in Angstrom.
 */
#ifndef OSVMP2_H
#define OSVMP2_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct osvmp2_ctx osvmp2_ctx;

typedef enum {
  OSVMP2_OK = 0,
  OSVMP2_E_ARG = 1,      /* invalid argument (null pointer, size, index, order) */
  OSVMP2_E_CUDA = 2,     /* a CUDA runtime call or kernel launch failed */
  OSVMP2_E_NOMEM = 3,    /* device allocation failed */
  OSVMP2_E_NOCONV = 4,   /* amplitude iterations hit max_iter (see osvmp2_mbe_stats) */
  OSVMP2_E_NUMERIC = 5,  /* eigen-solver did not converge or produced non-finite values */
  OSVMP2_E_STATE = 6,    /* call order violated (e.g. pair_integrals before build_osv) */
  OSVMP2_E_TIMEOUT = 7   /* a bounded device-side wait (a tensor-core pipeline barrier) gave up:
                            the kernel left its loops early, waited (bounded) for its copies and
                            tensor-core operations in flight, released its tensor memory and
                            flagged the call; the call's results are invalid */
} osvmp2_status;

/* Arithmetic of the projection/exchange contractions (A1-A2) and of the residual
 * products (A4).  OSV eigen-decomposition, preconditioner, update denominators
 * and every energy accumulation are FP64 in all forms. */
typedef enum {
  OSVMP2_FP64 = 0,   /* all FP64 on the CUDA cores */
  OSVMP2_MIXED = 1   /* split-precision products with FP32 accumulation, FP64 elsewhere */
} osvmp2_prec;

typedef struct {
  double tau_s;       /* drop S_(ij,ij) eigenvalues below tau_s * max eigenvalue (default 1e-10) */
  double tol_update;  /* stop when max |R~ / D| below this ...                (default 1e-7)  */
  double tol_energy;  /* ... and |E_C(it) - E_C(it-1)| below this, Eh         (default 1e-13;
                          fragment solves use at least 16 ulps of |E_C|, the FP64 rounding floor
                          of the fragment energy, and the mixed form 1e-11 |E_C|) */
                      /* (the energy test does the fine convergence: the update
                          has a rounding floor of ~eps*cond(S_(ij,ij)))       */
  int32_t max_iter;   /* amplitude iterations per fragment                    (default 100) */
  int32_t osv_prec;   /* arithmetic of the T_ii contraction B_i B_i^T in osvmp2_build_osv
                         (an osvmp2_prec; default OSVMP2_FP64).  OSVMP2_MIXED runs it on
                         the tensor cores with split-precision operands (~35 significant
                         bits); the eigen-decomposition stays FP64 in both.  Library
                         extension: the paper forms T_ii in one precision only. */
  int32_t no_autotune; /* 0 (default): the first osvmp2_mbe3_energy for a given fragment count and
                          largest pair order times the candidate launch shapes of the mixed
                          fragment solve and keeps the fastest (osvmp2_get_solve_plan); 1: fixed
                          default shape (2 CTAs per SM); 2: fixed shape of 3 CTAs per SM.  The
                          energies are identical either way. */
  int32_t mem_cap_mib; /* 0 (default): no limit.  Otherwise the device memory this ctx may hold at
                          once (its cache, pair store and temporaries), in MiB; a request beyond it
                          fails with OSVMP2_E_NOMEM as a failed cudaMalloc would.  Library extension
                          for callers that run under a memory budget. */
  int32_t osv_method;  /* OSV generation in osvmp2_build_osv: 0 (default) full eigen-decomposition
                          of T_ii; 1 randomized (Algorithm 3): adaptive range finder on Gaussian rows
                          (look-ahead r = 10, stop when every look-ahead row has norm
                          <= l_osv / (10 sqrt(2/pi))), then the SVD of T~ = Z T_ii through the
                          eigen-decomposition of T~ T~^T.  The Gaussian draws are the Irwin-Hall(12)
                          normals of the system's seed, stream 7, counter (i 2^16 + k) n_vir + a. */
  int32_t rosv_max_rows; /* randomized OSVs: rows the range finder may take per orbital (0: min(n_vir,
                          256)); running out is OSVMP2_E_NUMERIC. */
  int32_t reserved[2];
} osvmp2_opts;

/* Synthetic or caller-supplied system.  All arrays are read by the kernels. */
typedef struct {
  int32_t n_occ, n_vir, n_aux;
  const double *B;      /* device [n_occ][n_vir][n_aux] RI integrals (ia|P), or NULL:
                           regenerate on the device as B = env[i][a] * z(seed,i,a,P) */
  uint64_t seed;        /* generator seed when B == NULL (counter-based, SplitMix64) */
  const double *env;    /* device [n_occ][n_vir] envelope, required when B == NULL */
  const double *f_occ;  /* device [n_occ][n_occ] symmetric occupied (LMO) Fock block */
  const double *e_vir;  /* device [n_vir] canonical virtual orbital energies */
  const double *r_occ;  /* host [n_occ][3] LMO centres (fragment lists); may be NULL
                           if osvmp2_mbe3_energy / osvmp2_energy_grad are not used */
} osvmp2_system;

typedef struct {
  int64_t n_single, n_pair, n_triple;  /* kept clusters */
  int64_t n_pair_blocks;               /* unique pairs (i<=j) whose blocks were built */
  int32_t max_iter_used;               /* largest iteration count over fragments */
  int32_t n_unconverged;               /* fragments that hit max_iter */
  int64_t worst_fragment;              /* index of the first unconverged fragment, or -1 */
  double max_update;                   /* largest final max|R~/D| over fragments */
  double flops;                        /* algorithmic FP operations of A1-A5 in this call */
  int64_t n_weak;                      /* weak pairs (osvmp2_mbe3_energy_screened; 0 otherwise) */
} osvmp2_mbe_stats;

/* Pair-class cuts of the paper's cluster selection (Section 3.4), applied to
 * s2b_ij = sum_{mu nu} <mu_i|nu_j>^2 / sqrt(n_i n_j) (Eq. s2b). */
typedef struct {
  double s2b_distant;  /* pairs with s2b below this are distant and dropped      (paper: 1e-7) */
  double s2b_close;    /* pairs with s2b >= this are close (MBE clusters); the
                          rest are weak (single-block, non-iterative)            (paper: 1e-2) */
  double s3b_min;      /* a triple of three close pairs is kept when
                          s3b = (s2b_ij + s2b_ik + s2b_jk) / 3 >= this (Eq. s3b) (paper: 0.2)  */
} osvmp2_screen;

/* ---- context ------------------------------------------------------------ */

/* Create a ctx on CUDA device `device` queueing work on `cuda_stream`
 * (a cudaStream_t; NULL = legacy default stream).  opts may be NULL (defaults). */
int osvmp2_create(osvmp2_ctx **ctx, int device, void *cuda_stream, const osvmp2_opts *opts);
/* Release all ctx-owned device memory.  Safe on NULL. */
void osvmp2_destroy(osvmp2_ctx *ctx);
/* Last error message of this ctx ("" if none).  Valid until the next call on ctx. */
const char *osvmp2_last_error(const osvmp2_ctx *ctx);
/* Fill opts with the defaults listed in osvmp2_opts. */
void osvmp2_default_opts(osvmp2_opts *opts);
/* Replace the options of ctx (validated as in osvmp2_create; E_ARG leaves them
 * unchanged).  Takes effect for the next call; built OSVs and pair blocks are
 * kept. */
int osvmp2_set_opts(osvmp2_ctx *ctx, const osvmp2_opts *opts);
/* Launch shape of the last mixed MBE(3) fragment solve: out[0] CTAs per SM (1-3; 3 runs the
 * solver built for 80 registers per thread), out[1] tile set
 * of its FP32 contractions (0: 64/96-wide tiles, 1: also 80-wide), out[2] 1 if chosen by the
 * autotuner, out[3] number of tuned (fragment count, largest pair order) keys.  out: 4 ints
 * (host).  The solve and the MBE(3) sum run as one CUDA graph, replayed with updated
 * arguments on later calls.  Library extension (the paper does not batch this way). */
int osvmp2_get_solve_plan(const osvmp2_ctx *ctx, int32_t *out);
/* Number of CUDA kernels this library has launched in this process (all ctxs). */
int64_t osvmp2_kernel_launches(void);

/* ---- A0: OSV generation (Eq. mp2_tkk, Eq. osv_gen, Algorithm 3's output) --
 * For every occupied i: T_ii[a][b] = sum_P B[i,a,P] B[i,b,P] / (e_a + e_b - 2 f_ii),
 * full FP64 symmetric eigen-decomposition on the GPU, keep eigenvectors with
 * omega >= l_osv (all when l_osv <= 0), descending omega, each eigenvector signed
 * so that its largest-magnitude entry is positive.
 * n_osv_host: host [n_occ] out, OSV count per orbital.  Discards pair data of a
 * previous system. */
int osvmp2_build_osv(osvmp2_ctx *ctx, const osvmp2_system *sys, double l_osv, int32_t *n_osv_host);

/* Copy Q_i (device [n_vir][n_osv_i], row-major) and omega_i (device [n_osv_i]) out. */
int osvmp2_get_osv(osvmp2_ctx *ctx, int32_t i, double *Q_dev, double *omega_dev);

/* ---- A1-A2: pair integrals (Eq. osv_imua, Eq. osv_close_k, Algorithm 5) -----
 * pairs: host [n_pairs][2], 0-based, i <= j.  For every listed pair and every
 * diagonal pair (i,i) of its orbitals, build on the device:
 *   B~_i^(x) = B[i]^T Q_x (aux x OSV), K_(ij,ij) = (P^T B_i)(P^T B_j)^T,
 *   S_(x,y) = Q_x^T Q_y and F_(x,y) = Q_x^T diag(e_vir) Q_y with P = [Q_i Q_j]
 *   (P_ii = Q_i), then the preconditioner X, e~ of Eq. prec_eig.
 * Pairs already built are skipped.  prec selects the contraction arithmetic. */
int osvmp2_pair_integrals(osvmp2_ctx *ctx, const int32_t *pairs, int64_t n_pairs, osvmp2_prec prec);

/* Copy the blocks of built pair (i,j), i<=j, to device buffers of m*m doubles,
 * m = n_i + n_j (n_i if i == j); any output may be NULL. */
int osvmp2_get_pair_blocks(osvmp2_ctx *ctx, int32_t i, int32_t j, double *K_dev, double *S_dev,
                           double *F_dev);

/* Preconditioner of built pair (i,j) (Eq. prec_eig): X (device [m][m], row-major;
 * columns 0..r-1 valid) with X^T S X = 1 and X^T F X = diag(e~), e~ (device [m],
 * first r valid), r (host scalar) = number of S_(ij,ij) eigenvalues above
 * tau_s * max.  Any output may be NULL. */
int osvmp2_get_precond(osvmp2_ctx *ctx, int32_t i, int32_t j, double *X_dev, double *et_dev, int32_t *r_out);

/* ---- A3-A4: OSV-MP2 solve of one subsystem (Eq. res_close, Algorithm 7) ----
 * orbs: host [n_orbs] distinct occupied indices (e.g. all of them).  Solves the
 * coupled residual equations of every pair in the subsystem (k summed over the
 * subsystem only), Jacobi sweeps preconditioned by Eq. prec_eig.
 * e_out: host scalar, E = sum_{i,j in orbs} <K_(ij), 2T_(ij) - T_(ij)^T>.
 * pair_e_out: host [n_orbs*(n_orbs+1)/2] or NULL: pair energies for i<=j in the
 * order (orbs[0],orbs[0]), (orbs[0],orbs[1]), ...; i != j counted twice.
 * iters_out: host scalar or NULL. */
int osvmp2_solve(osvmp2_ctx *ctx, const int32_t *orbs, int32_t n_orbs, osvmp2_prec prec,
                 double *e_out, double *pair_e_out, int32_t *iters_out);

/* ---- A5: MBE(3) energy ------------------------------------------------------
 * Fragments: every single; every pair with |r_i - r_j|^2 <= r2_cut^2; every
 * triple whose three pairs satisfy d^2 <= r3_cut^2 and are kept pairs.
 * E = sum_C c_C E_C with c_ijk = 1, c_ij = 1 - #kept triples containing ij,
 * c_i = 1 - #kept pairs containing i + #kept triples containing i.
 * Builds the needed pair integrals, solves all fragments in one persistent
 * launch, and accumulates E in FP64 in fragment order.  stats may be NULL. */
int osvmp2_mbe3_energy(osvmp2_ctx *ctx, double r2_cut, double r3_cut, osvmp2_prec prec,
                       double *e_out, osvmp2_mbe_stats *stats);

/* Fragment list of the last osvmp2_mbe3_energy / osvmp2_energy_grad call:
 * host outputs, each may be NULL: orbs [n][3] (-1 padded), weights [n],
 * energies [n] (E_C).  *n_frag_out receives the count (also when arrays are NULL). */
int osvmp2_fragment_results(osvmp2_ctx *ctx, int64_t *n_frag_out, int32_t *orbs, int32_t *weights,
                            double *energies);

/* Host-only fragment enumeration with the rule of osvmp2_mbe3_energy.
 * r_occ host [n_occ][3].  If orbs_out (host [cap][3]) is non-NULL and cap is
 * large enough, writes the list (singles, pairs, triples, each lexicographic)
 * and weights_out (host [cap]).  *n_out = number of fragments. */
int osvmp2_mbe3_fragments(const double *r_occ, int32_t n_occ, double r2_cut, double r3_cut,
                          int64_t cap, int32_t *orbs_out, int32_t *weights_out, int64_t *n_out);

/* ---- A5 with the paper's cluster selection (Section 3.4; Eqs. s2b, s3b) ----
 * s2b of every pair i < j, computed on the GPU in FP64 from the OSVs of the
 * last osvmp2_build_osv.  Host outputs, each may be NULL: s2b_out [n_occ][n_occ]
 * (symmetric, diagonal 1), class_out [n_occ][n_occ] (2 close, 1 weak, 0 distant;
 * diagonal 2), counts [3] (close, weak, distant pairs i < j). */
int osvmp2_pair_screening(osvmp2_ctx *ctx, const osvmp2_screen *scr, double *s2b_out, int32_t *class_out,
                          int64_t *counts);

/* MBE(3) energy over the clusters the screening selects -- every single, every
 * close pair, every triple of close pairs with s3b >= s3b_min, weights as in
 * osvmp2_mbe3_energy -- plus the weak pairs (Algorithm 7, weak branch): for
 * each weak pair the single-block residual (Eq. res_weak, read as
 * K_(i,j) + F_(i,i) T + T F_(j,j) - (f_ii + f_jj) T - f_ij [T_(i,i) S_(i,j) + S_(i,j) T_(j,j)]
 * with K_(i,j) from Eq. osv_weak_k and T_(i,i) the MBE(3) diagonal amplitude of
 * Eq. tmbediag) solved in one update in the eigenbases of F_(i,i), F_(j,j); its
 * energy 2 <K_(i,j), T_(i,j)> per ordered pair, both orders counted.  The
 * weak-pair arithmetic is FP64 in both forms; prec selects the clusters' form.
 * e_out (host) = cluster sum + weak sum; e_weak_out (host, nullable) = weak sum.
 * Distances (r_occ) are not used. */
int osvmp2_mbe3_energy_screened(osvmp2_ctx *ctx, const osvmp2_screen *scr, osvmp2_prec prec, double *e_out,
                                double *e_weak_out, osvmp2_mbe_stats *stats);

/* Weak pairs of the last osvmp2_mbe3_energy_screened (empty after other calls):
 * *n_out = count; pairs (host [n][2], i < j, lexicographic) and energies
 * (host [n], both orders) may be NULL. */
int osvmp2_weak_results(osvmp2_ctx *ctx, int64_t *n_out, int32_t *pairs, double *energies);

/* ---- occupied-orbital localization (Section 3.2, Algorithm 2, Eq. loc_theta) ----
 * Jacobi-sweep Pipek-Mezey localization with Loewdin charges.  C: device
 * [n_ao][n_occ], orthonormal columns in an orthonormal (Loewdin) AO basis;
 * atom_ao: host [n_atom + 1] AO offsets of the atoms (0 ... n_ao, ascending).
 * P^A_ij = sum_{alpha in A} C_alpha,i C_alpha,j; sweeps over the pairs i < j in
 * order with a_ij = sum_A (P^A_ij)^2 - (P^A_ii - P^A_jj)^2 / 4,
 * b_ij = sum_A P^A_ij (P^A_ii - P^A_jj), theta = atan2(b_ij, -a_ij) / 4 (the
 * branch that maximises the functional), rotation skipped when
 * |sin theta| < 1e-10; a sweep adds sqrt(a^2 + b^2)(1 - cos 4 theta) to dL, and
 * the sweeps stop when dL <= l_loc (paper: 1e-3).
 * U: device [n_occ][n_occ] out, the localized orbitals are C U; L_out (host,
 * nullable): sum_{i,A} (P^A_ii)^2 at the end; sweeps_out (host, nullable).
 * OSVMP2_E_NOCONV after max_sweeps sweeps (U and L then hold the last state).
 * Uses the ctx's stream and memory cache only; needs no system. */
int osvmp2_localize_pm(osvmp2_ctx *ctx, const double *C_dev, int32_t n_ao, int32_t n_occ, const int32_t *atom_ao,
                       int32_t n_atom, double l_loc, int32_t max_sweeps, double *U_dev, double *L_out,
                       int32_t *sweeps_out);

/* ---- A6: frozen-OSV gradient --------------------------------------------
 * MBE(3) energy as osvmp2_mbe3_energy, plus (device outputs, each may be NULL):
 *   dE_dB [n_occ][n_vir][n_aux]: dE/dB[i,a,P] = 4 sum_C c_C sum_j (T~_ij^C B_j)[a,P]
 *   dE_de [n_vir]              : 2 sum_C c_C sum_ij sum_b T~_ij^ab T_ij^ab
 *   dE_df [n_occ][n_occ]       : symmetrised derivative w.r.t. the occupied Fock block
 * with T~ = 2T - T^T in the full virtual space and the OSVs held fixed.  Outputs
 * are overwritten. */
int osvmp2_energy_grad(osvmp2_ctx *ctx, double r2_cut, double r3_cut, osvmp2_prec prec,
                       double *e_out, double *dE_dB, double *dE_df, double *dE_de,
                       osvmp2_mbe_stats *stats);

/* ---- A6 with relaxed OSVs --------------------------------------------------
 * The gradient of osvmp2_energy_grad plus the response of the kept OSVs of every
 * orbital to T_ii (Eq. osv_gen on the T_ii of Eq. mp2_tkk), i.e. the derivative of
 * the MBE(3) energy with the OSVs rebuilt from B, e_vir and f_occ.  The OSV count of
 * every orbital is held fixed: the truncated energy jumps where an eigenvalue of T_ii
 * crosses l_osv, and the response scales with 1 / (eigenvalue gap at the cut), whose
 * smallest value over the orbitals is written to *min_gap_out (may be NULL).
 *   dE/dQ_x: the Q_x columns of alpha [R~ P T^T + R~^T P T] over the stored pairs of
 *            every fragment (weights c_C), R the full-space residual of Eq. res_close,
 *            R~ = 2R - R^T, alpha = 4 (i < j) or 2 (i = j);
 *   Z_x    = sym(Z_d Y Q_x^T), Y_lk = z_l^T (dE/dq_k) / (omega_k - omega_l) over the
 *            discarded eigenpairs (omega_l, z_l) of T_xx;
 *   dE/dB_x += 2 (Z_x / D) B_x, dE/de_a -= 2 sum_(x,b) (Z_x T_xx / D)_ab,
 *   dE/df_xx += 2 sum (Z_x T_xx / D),  D_ab = e_a + e_b - 2 f_xx.
 * FP64 form only (the pair store of an FP64 osvmp2_mbe3_energy), exact OSVs only
 * (opts.osv_method 0): OSVMP2_E_ARG otherwise.  T_ii and its eigenpairs are formed again
 * in FP64 inside the call; after a mixed OSV build (opts.osv_prec) they agree with the
 * built OSVs to that build's accuracy.  OSVMP2_E_NUMERIC when the FP64
 * eigenvalues of T_xx give another count above l_osv than the built OSVs, or no
 * positive gap at the cut.  Outputs as osvmp2_energy_grad (overwritten). */
int osvmp2_energy_grad_relaxed(osvmp2_ctx *ctx, double r2_cut, double r3_cut, double *e_out,
                               double *dE_dB, double *dE_df, double *dE_de,
                               osvmp2_mbe_stats *stats, double *min_gap_out);

/* ---- profiling -----------------------------------------------------------
 * Phases timed with CUDA events on the ctx stream around their kernels. */
enum {
  OSVMP2_PH_TII = 0,       /* A0: T_ii from B (Eq. mp2_tkk) */
  OSVMP2_PH_EIG = 1,       /* A0: eigen-decomposition and selection (Eq. osv_gen) */
  OSVMP2_PH_SF = 2,        /* A2: S_(x,y), F_(x,y) */
  OSVMP2_PH_PROJECT = 3,   /* A1: B~ = B^T Q (Eq. osv_imua) */
  OSVMP2_PH_EXCHANGE = 4,  /* A2: K_(ij,ij) (Eq. osv_close_k) */
  OSVMP2_PH_PRECOND = 5,   /* A3: Eq. prec_eig */
  OSVMP2_PH_SOLVE = 6,     /* A4: persistent fragment solve (Algorithm 7) */
  OSVMP2_PH_MBE_SUM = 7,   /* A5: weighted fragment-energy sum */
  OSVMP2_PH_SUBSOLVE = 8,  /* A4: pair-parallel subsystem solve (osvmp2_solve) */
  OSVMP2_PH_GRAD = 9,      /* A6: adjoint kernels */
  /* single kernels, timed inside the phases above */
  OSVMP2_PH_K_GPROJ = 10,  /* mixed A1: the tensor-core G = U^T B launches (inside PROJECT) */
  OSVMP2_PH_K_EIG = 11,    /* A0: the OSV eigen-decomposition launches, without the
                              back-transformation (inside EIG) */
  OSVMP2_PH_K_FRAGSOLVE = 12, /* A4: the persistent fragment solve and its energy sum (inside SOLVE) */
  OSVMP2_PH_SIGMA = 13,    /* mixed A4 set-up: pair-couple overlaps on the tensor cores (inside SOLVE) */
  OSVMP2_PH_WEAK = 14,     /* weak pairs: diagonal amplitudes, S blocks, K_(i,j), solve */
  OSVMP2_PH_SCREEN = 15,   /* s2b of every pair */
  OSVMP2_PH_LOCALIZE = 16, /* Pipek-Mezey localization (osvmp2_localize_pm) */
  OSVMP2_PH_RELAX = 17,    /* A6 relaxed: OSV response (osvmp2_energy_grad_relaxed) */
  OSVMP2_NPHASE = 20
};
/* Accumulated since the last reset, per phase (host arrays of OSVMP2_NPHASE, any
 * may be NULL): device milliseconds, algorithmic FP operations (GEMM-shaped
 * phases; 0 where not counted), DRAM bytes the phase must read at least
 * (0 where not counted) and number of timed launches.  Synchronises the ctx stream. */
int osvmp2_profile(osvmp2_ctx *ctx, double *ms, double *flops, double *bytes, int64_t *calls, int reset);

/* ---- generator ---------------------------------------------------------
 * Materialise B[i0:i0+n_i][n_vir][n_aux] = env[i][a] * z(seed,i,a,P) on the
 * device (out: device [n_i][n_vir][n_aux]); z is the Irwin-Hall(12) normal from
 * three SplitMix64 draws defined in the synthetic-input module. */
int osvmp2_generate_B(int32_t n_occ, int32_t n_vir, int32_t n_aux, uint64_t seed, const double *env,
                      int32_t i0, int32_t n_i, double *out, void *cuda_stream);

/* ---- allocation-free preconditioner ------------------------------------------
 * The paper has no counterpart to this entry point: it exists for callers that
 * cannot call cudaMalloc -- a process that hands all GPU memory to its own pool
 * allocator at start-up and forbids further driver allocations, a plug-in that
 * runs inside another application's CUDA context under that application's
 * memory budget, or a latency-critical loop in which an allocation (which may
 * synchronise the device) is unacceptable.
 *
 * It computes the same preconditioner as osvmp2_pair_integrals does for one pair
 * (canonical orthogonalisation of S with eigenvalues below tau_s * max dropped,
 * then the eigen-decomposition of Y^T F Y; X^T S X = 1, X^T F X = diag(e~)) from
 * caller-supplied dense matrices, and allocates nothing: its scratch is a
 * file-scope device array sized for m <= OSVMP2_NOALLOC_MAX_M (about 3.2 MB),
 * which every GPU that loads the library holds until the process exits.
 *   S_dev, F_dev : device [m][m] row-major S_(ij,ij), F_(ij,ij)     (read)
 *   X_dev        : device [m][m] row-major, columns 0..r-1 written  (out)
 *   et_dev       : device [m], entries 0..r-1 written               (out)
 *   r_dev        : device int32, r (out): the number of kept directions; 0 if S has no
 *                  eigenvalue above tau_s * max (e.g. S = 0: X and e~ are then not
 *                  written); -1 if S or F holds a NaN or Inf, or an eigen-solve
 *                  failed or gave a non-finite eigenvalue
 *   cuda_stream  : cudaStream_t to queue the single kernel on (NULL = legacy default)
 *   err, err_len : optional host buffer for a one-line error message
 * Returns OSVMP2_E_ARG (with a message) for null pointers, tau_s < 0, or m outside
 * 1..OSVMP2_NOALLOC_MAX_M, OSVMP2_E_CUDA if the launch fails.  The call is
 * asynchronous; outputs are ready when the stream reaches the kernel's end.
 * Every call looks up the device address of the static scratch in the
 * caller's current context with cudaGetSymbolAddress (host code cannot use the
 * array's name as a device address), so a reset or replaced context never sees
 * a stale address.  The first call in a context may load the library's device
 * code into it (lazy module loading); make that first call before any stream
 * capture.  Every call shares the one scratch
 * array and the kernel writes each scratch element before reading it, so
 * nothing from an earlier call needs clearing -- but calls whose kernels
 * overlap on the GPU (different streams without ordering) race on that array:
 * order them on one stream or with events. */
#define OSVMP2_NOALLOC_MAX_M 256
int osvmp2_precond_noalloc(const double *S_dev, const double *F_dev, int32_t m, double tau_s, double *X_dev,
                           double *et_dev, int32_t *r_dev, void *cuda_stream, char *err, int32_t err_len);

#ifdef __cplusplus
}
#endif
#endif /* OSVMP2_H */
