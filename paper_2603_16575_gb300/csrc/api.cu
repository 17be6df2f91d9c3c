// Host runtime of libosvmp2: the C ABI entry points, the ctx that owns the
// device-resident OSV / pair store, job lists for the kernels, and the MBE(3)
// fragment enumeration.  All arithmetic of the method runs in the kernels.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cstdint>
#include <map>
#include <unordered_map>
#include <string>
#include <vector>

#include "osvmp2.h"
#include "internal.h"

namespace {
constexpr int PW_MAX_ORDER = 192;   // largest pair order of the one-warp preconditioners
}

using namespace osv;

namespace osv {
static std::atomic<long long> g_launches{0};
void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace osv

namespace {

constexpr uint64_t STREAM_MUL = 0xD1B54A32D192ED03ull;
constexpr uint64_t STREAM_B = 5;   // stream id of B in the generator definition

struct Frag {
  int orbs[3];
  int weight;
};

}  // namespace

// Device-memory cache of a ctx.  Blocks released by the temporaries of a call
// and by the pair store go to a free list and are handed out again to later
// requests of similar size, so a repeated call (one energy step after another)
// allocates nothing from the driver and never waits in cudaFree.  All work of
// a ctx runs on its one stream, so a reused block is only touched by work
// enqueued after the last use by its previous owner.  Sizes are rounded up
// (256-byte granules below 1 MiB, 1 MiB granules above); a free block serves a
// request when it is at most an eighth (plus one granule) larger; a failed
// cudaMalloc first returns every cached block to the driver.
struct DevPool {
  std::multimap<size_t, void*> free_blocks;   // size -> block
  std::unordered_map<void*, size_t> size_of;  // every block the pool handed out
};

// Launch shape of the mixed fragment solve, chosen per (fragment count, largest
// pair order) by the autotuner of mbe3_core: CTAs per SM and the tile set of
// the solver's FP32 contractions.  Every candidate computes the same numbers
// (one CTA per fragment, the same FMA order), so the choice changes time only.
struct SolvePlan {
  int ctas_per_sm = 2;
  int tiles = 0;
  bool tuned = false;
  float ms = 0.f;      // measured time of the chosen plan (autotuned plans)
};

struct osvmp2_ctx {
  DevPool pool;
  size_t held = 0;                                  // device bytes this ctx holds from the driver
  std::unordered_map<void*, size_t> raw_size;       // every driver block it holds, with its size
  std::map<std::pair<int, int>, SolvePlan> plans;   // mixed solve plans by (n_frag, max_m)
  SolvePlan last_plan;
  cudaStream_t cap_st = nullptr;      // private stream used only to record the solve graph
  cudaGraphExec_t solve_exec = nullptr;
  int device = 0;
  cudaStream_t st = nullptr;
  osvmp2_opts opts{};
  std::string err;
  int num_sms = 148;
  std::vector<void*> sys_allocs;     // freed when a new system is set
  std::vector<void*> pair_allocs;    // pair store; freed with the system or on a precision change
  int pair_prec = -1;                // precision the pair store was built with
  // system
  bool have_sys = false;
  osvmp2_system sys{};
  uint64_t key = 0;
  std::vector<double> r_occ;
  // OSVs
  bool have_osv = false;
  std::vector<int> n_osv;
  std::vector<double*> Qp, Wp;
  double l_osv = 0.0;        // cut of the last OSV build
  int cap_pairs = 0;
  // device tables
  int* n_osv_d = nullptr;
  double** Q_d = nullptr;
  int* sf_id_d = nullptr;
  double** S_d = nullptr;
  double** F_d = nullptr;
  int* pair_id_d = nullptr;
  double** K_d = nullptr;
  double** X_d = nullptr;
  double** et_d = nullptr;
  double** Kt_d = nullptr;
  float** U_d = nullptr;
  float** Sh_d = nullptr;
  float** Gh_d = nullptr;
  int* r_d = nullptr;
  int* err_d = nullptr;
  double* scal_d = nullptr;          // device scalars (energies)
  // host mirrors
  std::vector<int> sf_id, pair_id, bt_id;
  std::vector<double*> S_h, F_h, K_h, X_h, et_h, bt_h, Kt_h;
  std::vector<float*> U_h, Gi_h, Gj_h;   // mixed form: per pair U = P X and G = U^T B
  std::vector<float*> Sh_h, Gh_h;        // mixed form: preconditioner leftovers (NULL: exact X)
  // mixed form: where the TF32 slices of U_p^T live (allocation base, its rows, first row)
  std::vector<float*> us_base_h;
  std::vector<long long> us_alloc_rows_h, us_row_h;
  int us_ldv = 0;
  std::vector<int> m_h;
  std::vector<int> pi_h, pj_h;       // pair id -> (i, j)
  // last MBE call
  std::vector<Frag> frags;
  std::vector<FragOut> frag_out;
  std::vector<std::pair<int, int>> weak;   // weak pairs of the last screened call
  std::vector<double> weak_e;              // and their energies (both orders)
  // per-phase device time (CUDA events on st) and algorithmic flops, accumulated
  // a phase may be entered several times between collections (batched
  // launches): each entry takes the next (begin, end) pair of its event pool
  std::vector<cudaEvent_t> ph_ev[OSVMP2_NPHASE];
  size_t ph_used[OSVMP2_NPHASE] = {};
  double ms[OSVMP2_NPHASE] = {};
  double flops[OSVMP2_NPHASE] = {};
  double bytes[OSVMP2_NPHASE] = {};
  long long calls[OSVMP2_NPHASE] = {};
  std::vector<int> r_h;               // preconditioner ranks (host copy)
  std::vector<double> f_h;            // occupied Fock block (host copy, flop counts)
};

namespace {

int fail(osvmp2_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return code;
}

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(c, e_ == cudaErrorMemoryAllocation ? OSVMP2_E_NOMEM : OSVMP2_E_CUDA,        \
                  "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

#define TRY(expr)          \
  do {                     \
    int s_ = (expr);       \
    if (s_) return s_;     \
  } while (0)

// Every driver allocation of a ctx goes through raw_malloc / raw_free, which
// keep the byte count that the optional cap (opts.mem_cap_mib) is checked
// against; a request beyond the cap fails as a failed cudaMalloc would.
cudaError_t raw_malloc(osvmp2_ctx* c, void** p, size_t bytes) {
  *p = nullptr;
  if (c->opts.mem_cap_mib > 0 && c->held + bytes > ((size_t)c->opts.mem_cap_mib << 20))
    return cudaErrorMemoryAllocation;
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) {
    c->held += bytes;
    c->raw_size[*p] = bytes;
  }
  return e;
}
void raw_free(osvmp2_ctx* c, void* p) {
  auto it = c->raw_size.find(p);
  if (it != c->raw_size.end()) {
    c->held -= it->second;
    c->raw_size.erase(it);
  }
  cudaFree(p);
}

int dalloc(osvmp2_ctx* c, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = raw_malloc(c, p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, OSVMP2_E_NOMEM, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
  }
  c->sys_allocs.push_back(*p);
  return 0;
}
template <class T>
int dalloc_t(osvmp2_ctx* c, T** p, size_t n) {
  return dalloc(c, reinterpret_cast<void**>(p), n * sizeof(T));
}

size_t pool_round(size_t b) {
  constexpr size_t MiB = (size_t)1 << 20;
  if (b < MiB) return (std::max<size_t>(b, 16) + 255) & ~(size_t)255;
  return (b + MiB - 1) & ~(MiB - 1);
}
// Return every cached block to the driver.
void pool_trim(osvmp2_ctx* c) {
  if (c->pool.free_blocks.empty()) return;
  if (c->st) cudaStreamSynchronize(c->st);
  for (auto& kv : c->pool.free_blocks) {
    c->pool.size_of.erase(kv.second);
    raw_free(c, kv.second);
  }
  c->pool.free_blocks.clear();
}
cudaError_t pool_get(osvmp2_ctx* c, void** p, size_t bytes) {
  const size_t r = pool_round(bytes);
  const size_t slack = r / 8 + (r < ((size_t)1 << 20) ? 256 : ((size_t)1 << 20));
  auto it = c->pool.free_blocks.lower_bound(r);
  if (it != c->pool.free_blocks.end() && it->first <= r + slack) {
    *p = it->second;
    c->pool.free_blocks.erase(it);
    return cudaSuccess;
  }
  cudaError_t e = raw_malloc(c, p, r);
  if (e != cudaSuccess) {
    cudaGetLastError();
    pool_trim(c);
    e = raw_malloc(c, p, r);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return e;
  }
  c->pool.size_of[*p] = r;
  return cudaSuccess;
}
void pool_put(osvmp2_ctx* c, void* p) {
  if (!p) return;
  auto s = c->pool.size_of.find(p);
  if (s == c->pool.size_of.end()) {
    raw_free(c, p);
    return;
  }
  c->pool.free_blocks.emplace(s->second, p);
}

// Temporary device buffer returned to the ctx's cache at scope exit.
struct Tmp {
  void* p = nullptr;
  osvmp2_ctx* c = nullptr;
  ~Tmp() {
    if (p) pool_put(c, p);
  }
};
int tmp_alloc(osvmp2_ctx* c, Tmp& t, size_t bytes) {
  if (t.p) pool_put(t.c, t.p);
  t.c = c;
  cudaError_t e = pool_get(c, &t.p, bytes);
  if (e != cudaSuccess) {
    t.p = nullptr;
    return fail(c, OSVMP2_E_NOMEM, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
  }
  return 0;
}

void free_system(osvmp2_ctx* c) {
  if (c->st) cudaStreamSynchronize(c->st);
  for (void* p : c->sys_allocs) raw_free(c, p);
  c->sys_allocs.clear();
  for (void* p : c->pair_allocs) pool_put(c, p);
  c->pair_allocs.clear();
  c->pair_prec = -1;
  c->have_sys = c->have_osv = false;
  c->n_osv.clear(); c->Qp.clear(); c->Wp.clear();
  c->sf_id.clear(); c->pair_id.clear(); c->bt_id.clear();
  c->S_h.clear(); c->F_h.clear(); c->K_h.clear(); c->X_h.clear(); c->et_h.clear(); c->bt_h.clear(); c->Kt_h.clear();
  c->U_h.clear(); c->Gi_h.clear(); c->Gj_h.clear(); c->Sh_h.clear(); c->Gh_h.clear();
  c->us_base_h.clear(); c->us_alloc_rows_h.clear(); c->us_row_h.clear();
  c->m_h.clear(); c->pi_h.clear(); c->pj_h.clear();
  c->frags.clear(); c->frag_out.clear(); c->weak.clear(); c->weak_e.clear();
  c->n_osv_d = nullptr; c->Q_d = nullptr; c->sf_id_d = nullptr; c->S_d = c->F_d = nullptr;
  c->pair_id_d = nullptr; c->K_d = c->X_d = c->et_d = c->Kt_d = nullptr; c->r_d = nullptr; c->U_d = nullptr;
  c->Sh_d = c->Gh_d = nullptr;
}

Tables tables(const osvmp2_ctx* c) {
  Tables t;
  t.n_occ = c->sys.n_occ;
  t.n_vir = c->sys.n_vir;
  t.n_osv = c->n_osv_d;
  t.Q = c->Q_d;
  t.sf_id = c->sf_id_d;
  t.S = c->S_d;
  t.F = c->F_d;
  t.pair_id = c->pair_id_d;
  t.K = c->K_d;
  t.X = c->X_d;
  t.et = c->et_d;
  t.r = c->r_d;
  t.Kt = c->Kt_d;
  t.U = c->U_d;
  t.Sh = c->Sh_d;
  t.Gh = c->Gh_d;
  t.f_occ = c->sys.f_occ;
  return t;
}

BSrc bsrc(const osvmp2_ctx* c) {
  return BSrc{c->sys.B, c->sys.env, c->key, c->sys.n_vir, c->sys.n_aux};
}

void ph_collect(osvmp2_ctx* c);

int check_err_flag(osvmp2_ctx* c, const char* where) {
  int h = 0;
  CK(cudaMemcpyAsync(&h, c->err_d, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  CK(cudaGetLastError());
  ph_collect(c);
  if (h & ERR_EIG) return fail(c, OSVMP2_E_NUMERIC, "%s: eigen-solver did not converge", where);
  if (h & ERR_NONFINITE) return fail(c, OSVMP2_E_NUMERIC, "%s: non-finite values", where);
  if (h & ERR_SIZE) return fail(c, OSVMP2_E_NUMERIC, "%s: size limit exceeded", where);
  if (h & ERR_TIMEOUT) return fail(c, OSVMP2_E_TIMEOUT, "%s: a tensor-core pipeline wait timed out", where);
  return 0;
}

void ph_begin(osvmp2_ctx* c, int ph) {
  auto& ev = c->ph_ev[ph];
  while (ev.size() < c->ph_used[ph] + 2) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return;   // timing is best effort: this entry goes untimed
    }
    ev.push_back(e);
  }
  cudaEventRecord(ev[c->ph_used[ph]], c->st);
}
void ph_end(osvmp2_ctx* c, int ph, double flops, double bytes = 0.0) {
  auto& ev = c->ph_ev[ph];
  if (ev.size() >= c->ph_used[ph] + 2) {
    cudaEventRecord(ev[c->ph_used[ph] + 1], c->st);
    c->ph_used[ph] += 2;
  }
  c->flops[ph] += flops;
  c->bytes[ph] += bytes;
  c->calls[ph]++;
}
// Call after a stream synchronisation: fold finished phase timings in.
void ph_collect(osvmp2_ctx* c) {
  for (int ph = 0; ph < OSVMP2_NPHASE; ph++) {
    for (size_t k = 0; k + 1 < c->ph_used[ph]; k += 2) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, c->ph_ev[ph][k], c->ph_ev[ph][k + 1]) == cudaSuccess) c->ms[ph] += t;
      else cudaGetLastError();
    }
    c->ph_used[ph] = 0;
  }
}

template <class T>
int upload(osvmp2_ctx* c, T* dst, const std::vector<T>& src) {
  if (src.empty()) return 0;
  CK(cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, c->st));
  return 0;
}

double dist2(const double* r, int i, int j) {
  const double dx = r[3 * i] - r[3 * j];
  const double dy = r[3 * i + 1] - r[3 * j + 1];
  const double dz = r[3 * i + 2] - r[3 * j + 2];
  return dx * dx + dy * dy + dz * dz;
}

// Kept clusters and inclusion-exclusion weights (singles, pairs, triples; each
// lexicographic).  Squared distances are compared with the squared cutoffs.
void enumerate_fragments(const double* r, int n, double r2, double r3, std::vector<Frag>& out) {
  out.clear();
  const double c2 = r2 * r2, c3 = r3 * r3;
  std::vector<unsigned char> ok2((size_t)n * n, 0), ok3((size_t)n * n, 0);
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) {
      if (i == j) continue;
      const double d = dist2(r, i, j);
      ok2[(size_t)i * n + j] = d <= c2;
      ok3[(size_t)i * n + j] = (d <= c3) && (d <= c2);
    }
  std::vector<int> pair_cnt(n, 0), tri_cnt(n, 0), tri_pair((size_t)n * n, 0);
  std::vector<Frag> pairs, triples;
  for (int i = 0; i < n; i++)
    for (int j = i + 1; j < n; j++)
      if (ok2[(size_t)i * n + j]) {
        pairs.push_back(Frag{{i, j, -1}, 0});
        pair_cnt[i]++;
        pair_cnt[j]++;
      }
  for (int i = 0; i < n; i++)
    for (int j = i + 1; j < n; j++) {
      if (!ok3[(size_t)i * n + j]) continue;
      for (int k = j + 1; k < n; k++) {
        if (!ok3[(size_t)i * n + k] || !ok3[(size_t)j * n + k]) continue;
        triples.push_back(Frag{{i, j, k}, 1});
        tri_cnt[i]++; tri_cnt[j]++; tri_cnt[k]++;
        tri_pair[(size_t)i * n + j]++;
        tri_pair[(size_t)i * n + k]++;
        tri_pair[(size_t)j * n + k]++;
      }
    }
  for (int i = 0; i < n; i++) out.push_back(Frag{{i, -1, -1}, 1 - pair_cnt[i] + tri_cnt[i]});
  for (auto& p : pairs) {
    p.weight = 1 - tri_pair[(size_t)p.orbs[0] * n + p.orbs[1]];
    out.push_back(p);
  }
  for (auto& t : triples) out.push_back(t);
}

// Clusters selected by s2b / s3b (Section 3.4): close pairs s2b >= close, weak
// pairs distant <= s2b < close, triples of three close pairs with
// (s2b_ij + s2b_ik + s2b_jk) / 3 >= s3b_min; weights as in enumerate_fragments.
// s2b: host [n][n], symmetric.
void screened_fragments(const double* s2b, int n, const osvmp2_screen& sc, std::vector<Frag>& out,
                        std::vector<std::pair<int, int>>& weak) {
  out.clear();
  weak.clear();
  std::vector<unsigned char> close((size_t)n * n, 0);
  std::vector<int> pair_cnt(n, 0), tri_cnt(n, 0), tri_pair((size_t)n * n, 0);
  std::vector<Frag> pairs, triples;
  for (int i = 0; i < n; i++)
    for (int j = i + 1; j < n; j++) {
      const double v = s2b[(size_t)i * n + j];
      if (v >= sc.s2b_close) {
        close[(size_t)i * n + j] = close[(size_t)j * n + i] = 1;
        pairs.push_back(Frag{{i, j, -1}, 0});
        pair_cnt[i]++;
        pair_cnt[j]++;
      } else if (v >= sc.s2b_distant) {
        weak.push_back({i, j});
      }
    }
  for (int i = 0; i < n; i++)
    for (int j = i + 1; j < n; j++) {
      if (!close[(size_t)i * n + j]) continue;
      for (int k = j + 1; k < n; k++) {
        if (!close[(size_t)i * n + k] || !close[(size_t)j * n + k]) continue;
        const double s3 = (s2b[(size_t)i * n + j] + s2b[(size_t)i * n + k] + s2b[(size_t)j * n + k]) / 3.0;
        if (!(s3 >= sc.s3b_min)) continue;
        triples.push_back(Frag{{i, j, k}, 1});
        tri_cnt[i]++; tri_cnt[j]++; tri_cnt[k]++;
        tri_pair[(size_t)i * n + j]++;
        tri_pair[(size_t)i * n + k]++;
        tri_pair[(size_t)j * n + k]++;
      }
    }
  for (int i = 0; i < n; i++) out.push_back(Frag{{i, -1, -1}, 1 - pair_cnt[i] + tri_cnt[i]});
  for (auto& p : pairs) {
    p.weight = 1 - tri_pair[(size_t)p.orbs[0] * n + p.orbs[1]];
    out.push_back(p);
  }
  for (auto& t : triples) out.push_back(t);
}

int pair_dim_h(const osvmp2_ctx* c, int i, int j) { return c->n_osv[i] + (i != j ? c->n_osv[j] : 0); }

int palloc(osvmp2_ctx* c, double** p, size_t n) {
  *p = nullptr;
  const size_t bytes = std::max<size_t>(16, n * sizeof(double));
  cudaError_t e = pool_get(c, reinterpret_cast<void**>(p), bytes);
  if (e != cudaSuccess)
    return fail(c, OSVMP2_E_NOMEM, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
  c->pair_allocs.push_back(*p);
  return 0;
}

// Drop every built pair (blocks, projections, K, preconditioners).
int reset_pairs(osvmp2_ctx* c) {
  CK(cudaStreamSynchronize(c->st));
  for (void* p : c->pair_allocs) pool_put(c, p);
  c->pair_allocs.clear();
  const size_t nn = (size_t)c->sys.n_occ * c->sys.n_occ;
  c->sf_id.assign(nn, -1);
  c->pair_id.assign(nn, -1);
  c->bt_id.assign(nn, -1);
  c->S_h.clear(); c->F_h.clear(); c->K_h.clear(); c->X_h.clear(); c->et_h.clear(); c->bt_h.clear(); c->Kt_h.clear();
  c->U_h.clear(); c->Gi_h.clear(); c->Gj_h.clear(); c->Sh_h.clear(); c->Gh_h.clear();
  c->us_base_h.clear(); c->us_alloc_rows_h.clear(); c->us_row_h.clear();
  c->m_h.clear(); c->pi_h.clear(); c->pj_h.clear(); c->r_h.clear();
  TRY(upload(c, c->sf_id_d, c->sf_id));
  TRY(upload(c, c->pair_id_d, c->pair_id));
  c->pair_prec = -1;
  return 0;
}

// FP operations of one Jacobi sweep of a fragment as the solver performs it:
// per pair p (m x m, rank r) 4 GEMMs m^3 for G1 T S + S T G2, two GEMMs per
// coupling term (q != p, coefficient != 0), the four GEMMs of the
// preconditioned update and the energy contraction.
double fragment_iter_flops(const osvmp2_ctx* c, const Frag& f) {
  const int n = c->sys.n_occ;
  int orbs[3], nc = 0;
  for (int u = 0; u < 3; u++)
    if (f.orbs[u] >= 0) orbs[nc++] = f.orbs[u];
  double fl = 0.0;
  for (int a = 0; a < nc; a++)
    for (int b = a; b < nc; b++) {
      const int i = orbs[a], j = orbs[b];
      const double m = pair_dim_h(c, i, j);
      const int pid = c->pair_id[(size_t)i * n + j];
      const double r = (pid >= 0 && pid < (int)c->r_h.size()) ? c->r_h[pid] : m;
      fl += 8.0 * m * m * m + 4.0 * m * m * r + 4.0 * m * r * r + 3.0 * m * m;
      for (int cc = 0; cc < nc; cc++)
        for (int s2 = 0; s2 < 2; s2++) {
          if (s2 == 0 && cc == b) continue;
          if (s2 == 1 && cc == a) continue;
          const int x = (s2 == 0) ? a : cc, y = (s2 == 0) ? cc : b;
          const int k = orbs[cc];
          const double coef = (s2 == 0) ? c->f_h[(size_t)k * n + j] : c->f_h[(size_t)i * n + k];
          if (coef == 0.0) continue;
          const double mq = pair_dim_h(c, orbs[std::min(x, y)], orbs[std::max(x, y)]);
          fl += 2.0 * mq * mq * m + 2.0 * m * m * mq;
        }
    }
  return fl;
}

// FP operations of the preconditioner-basis solve of a fragment: the Sigma_pq
// set-up (S X_q, then X_p^T (S X_q)) once, then per sweep two GEMMs per
// coupling term (op(Y_q) Sigma^T, Sigma (...)), plus the element-wise update.
double fragment_mixed_flops(const osvmp2_ctx* c, const Frag& f, int iters) {
  const int n = c->sys.n_occ;
  int orbs[3], nc = 0;
  for (int u = 0; u < 3; u++)
    if (f.orbs[u] >= 0) orbs[nc++] = f.orbs[u];
  auto rr = [&](int i, int j) {
    const int pid = c->pair_id[(size_t)i * n + j];
    return (double)((pid >= 0 && pid < (int)c->r_h.size()) ? c->r_h[pid] : pair_dim_h(c, i, j));
  };
  double setup = 0.0, sweep = 0.0;
  std::vector<std::pair<int, int>> seen;
  for (int a = 0; a < nc; a++)
    for (int b = a; b < nc; b++) {
      const int i = orbs[a], j = orbs[b];
      const double mp = pair_dim_h(c, i, j), rp = rr(i, j);
      sweep += 6.0 * rp * rp;
      for (int cc = 0; cc < nc; cc++)
        for (int s2 = 0; s2 < 2; s2++) {
          if (s2 == 0 && cc == b) continue;
          if (s2 == 1 && cc == a) continue;
          const int x = (s2 == 0) ? a : cc, y = (s2 == 0) ? cc : b;
          const int k = orbs[cc];
          const double coef = (s2 == 0) ? c->f_h[(size_t)k * n + j] : c->f_h[(size_t)i * n + k];
          if (coef == 0.0) continue;
          const int qi = orbs[std::min(x, y)], qj = orbs[std::max(x, y)];
          const double mq = pair_dim_h(c, qi, qj), rq = rr(qi, qj);
          sweep += 2.0 * rq * rq * rp + 2.0 * rp * rq * rp;
          const std::pair<int, int> key{a * 3 + b, qi * n + qj};
          if (std::find(seen.begin(), seen.end(), key) == seen.end()) {
            seen.push_back(key);
            setup += 2.0 * mp * mq * rq + 2.0 * rp * mp * rq;
          }
        }
    }
  return setup + iters * sweep;
}

// Build S/F blocks, projections, K and preconditioners for every listed pair
// (and the diagonal pairs of its orbitals) that is not built yet.
// Mixed form: G_p,x = U_p^T B_x for every G job on the tensor cores.  The
// orbitals x are processed in batches whose B_x^T slices fit a fixed budget;
// within a batch the tiles are ordered by (x, aux tile, pair) so that the
// pairs sharing an aux tile of B_x read it while it is resident in L2.
int gproj_tensor(osvmp2_ctx* c, const std::vector<GJob>& gj, const std::vector<long long>& usrow, const float* Us,
                 long long us_rows, int ldv, long long lo_shift) {
  const int nv = c->sys.n_vir, nx = c->sys.n_aux, n = c->sys.n_occ;
  if (us_rows + tc::BN >= (long long)INT32_MAX)
    return fail(c, OSVMP2_E_ARG, "U slice store exceeds the tensor-map row range");
  std::vector<std::vector<int>> by_x(n);
  for (size_t q = 0; q < gj.size(); q++) by_x[gj[q].x].push_back((int)q);
  std::vector<int> xs;
  for (int x = 0; x < n; x++)
    if (!by_x[x].empty()) xs.push_back(x);
  if (xs.empty()) return 0;
  const size_t slot_bytes = (size_t)tc::NSL * nx * ldv * sizeof(float);
  const size_t budget = (size_t)4 << 30;
  const size_t per_batch = std::max<size_t>(1, std::min<size_t>(xs.size(), budget / slot_bytes));
  if ((long long)per_batch * tc::NSL * nx + tc::BM >= (long long)INT32_MAX)
    return fail(c, OSVMP2_E_ARG, "B slice batch exceeds the tensor-map row range");
  Tmp bs, xd;
  TRY(tmp_alloc(c, bs, per_batch * slot_bytes));
  TRY(tmp_alloc(c, xd, xs.size() * sizeof(int)));
  CK(cudaMemcpyAsync(xd.p, xs.data(), xs.size() * sizeof(int), cudaMemcpyHostToDevice, c->st));
  const int n_mt = (nx + tc::BM - 1) / tc::BM;
  for (size_t b0 = 0; b0 < xs.size(); b0 += per_batch) {
    const int nb = (int)std::min(per_batch, xs.size() - b0);
    launch_bslices(bsrc(c), (const int*)xd.p + b0, nb, (float*)bs.p, ldv, c->st);
    CK(cudaGetLastError());
    // Tile order: per orbital x, blocks of PB (pair, column tile) jobs, each with all
    // its aux tiles; a wave of the persistent grid then holds every aux tile of B_x
    // and only PB tiles of the U slices, so the B_x tiles stay in L2 across the
    // waves of x and every U tile is read once.
    const int PB = std::max(1, c->num_sms / std::max(1, n_mt));
    std::vector<tc::Job> jobs;
    for (int u = 0; u < nb; u++) {
      std::vector<std::pair<int, int>> pn;   // (G job, first column)
      for (int q : by_x[xs[b0 + u]])
        for (int n0 = 0; n0 < gj[q].r; n0 += tc::BN) pn.push_back({q, n0});
      for (size_t p0 = 0; p0 < pn.size(); p0 += PB)
        for (int mt = 0; mt < n_mt; mt++)
          for (size_t pp = p0; pp < std::min(pn.size(), p0 + (size_t)PB); pp++) {
            const int q = pn[pp].first, n0 = pn[pp].second;
            const GJob& g = gj[q];
            tc::Job jb;
            jb.a_row = u * tc::NSL * nx + mt * tc::BM;
            jb.a_sstride = nx;
            jb.b_row = (int)(usrow[q] + n0);
            jb.b_sstride = g.r;
            jb.m_valid = std::min(tc::BM, nx - mt * tc::BM);
            jb.n_valid = std::min(tc::BN, g.r - n0);
            jb.out = g.G + (size_t)n0 * nx + mt * tc::BM;
            jb.ld_out = nx;
            jb.m0 = mt * tc::BM;
            jb.n0 = n0;
            jb.s = 0.0;
            jobs.push_back(jb);
          }
    }
    Tmp jd;
    TRY(tmp_alloc(c, jd, jobs.size() * sizeof(tc::Job)));
    CK(cudaMemcpyAsync(jd.p, jobs.data(), jobs.size() * sizeof(tc::Job), cudaMemcpyHostToDevice, c->st));
    double fl = 0.0;
    for (const tc::Job& jb : jobs) fl += 2.0 * (double)jb.m_valid * jb.n_valid * nv;
    ph_begin(c, OSVMP2_PH_K_GPROJ);
    if (launch_gproj_tc((const float*)bs.p, (long long)nb * tc::NSL * nx, Us, us_rows, nv, ldv, (const tc::Job*)jd.p,
                        (int)jobs.size(), lo_shift, c->err_d, c->st))
      return fail(c, OSVMP2_E_CUDA, "tensor-map encoding for the G projection failed");
    ph_end(c, OSVMP2_PH_K_GPROJ, fl);
    CK(cudaGetLastError());
  }
  return 0;
}

int ensure_pairs_impl(osvmp2_ctx* c, const std::vector<std::pair<int, int>>& req, osvmp2_prec prec);

// A failure part-way through leaves pairs marked as pending and blocks only
// partly written; the whole pair store is dropped then (the OSVs are kept), so
// the next call on the ctx rebuilds what it needs instead of using them.
int ensure_pairs(osvmp2_ctx* c, const std::vector<std::pair<int, int>>& req, osvmp2_prec prec) {
  if (!c->have_osv) return fail(c, OSVMP2_E_STATE, "osvmp2_build_osv has not been called");
  if (prec != OSVMP2_FP64 && prec != OSVMP2_MIXED) return fail(c, OSVMP2_E_ARG, "unknown precision %d", (int)prec);
  for (auto& p : req)
    if (p.first < 0 || p.second < 0 || p.first >= c->sys.n_occ || p.second >= c->sys.n_occ || p.first > p.second)
      return fail(c, OSVMP2_E_ARG, "pair (%d,%d) invalid: need 0 <= i <= j < n_occ", p.first, p.second);
  const int rc = ensure_pairs_impl(c, req, prec);
  if (rc != 0 && rc != OSVMP2_E_STATE && c->have_osv) {
    const std::string msg = c->err;
    cudaGetLastError();
    reset_pairs(c);
    c->err = msg;
  }
  return rc;
}

int ensure_pairs_impl(osvmp2_ctx* c, const std::vector<std::pair<int, int>>& req, osvmp2_prec prec) {
  if (!c->have_osv) return fail(c, OSVMP2_E_STATE, "osvmp2_build_osv has not been called");
  if (prec != OSVMP2_FP64 && prec != OSVMP2_MIXED) return fail(c, OSVMP2_E_ARG, "unknown precision %d", (int)prec);
  if (c->pair_prec >= 0 && c->pair_prec != (int)prec) TRY(reset_pairs(c));
  c->pair_prec = (int)prec;
  const int n = c->sys.n_occ;
  std::vector<std::pair<int, int>> newp;
  auto want = [&](int i, int j) {
    if (c->pair_id[(size_t)i * n + j] == -1) {
      c->pair_id[(size_t)i * n + j] = -2;   // mark as pending
      newp.push_back({i, j});
    }
  };
  for (auto& p : req) {
    int i = p.first, j = p.second;
    if (i < 0 || j < 0 || i >= n || j >= n || i > j)
      return fail(c, OSVMP2_E_ARG, "pair (%d,%d) invalid: need 0 <= i <= j < n_occ", i, j);
    want(i, i);
    want(j, j);
    want(i, j);
  }
  if (newp.empty()) return 0;
  std::sort(newp.begin(), newp.end());
  const int nv = c->sys.n_vir, nx = c->sys.n_aux;
  // S/F blocks
  std::vector<SFJob> sfj;
  size_t sf_doubles = 0;
  for (auto& p : newp) {
    const size_t id = (size_t)p.first * n + p.second;
    if (c->sf_id[id] == -1) {
      c->sf_id[id] = -2;
      sfj.push_back(SFJob{p.first, p.second, nullptr, nullptr});
      sf_doubles += 2 * (size_t)c->n_osv[p.first] * c->n_osv[p.second];
    }
  }
  // projections B~_i^(x)
  std::vector<ProjJob> pj;
  size_t bt_doubles = 0;
  auto want_bt = [&](int i, int x) {
    const size_t id = (size_t)i * n + x;
    if (c->bt_id[id] == -1) {
      c->bt_id[id] = -2;
      pj.push_back(ProjJob{i, x, nullptr});
      bt_doubles += (size_t)nx * c->n_osv[x];
    }
  };
  const bool mixed = prec == OSVMP2_MIXED;
  for (auto& p : newp) {
    if (mixed) break;    // the mixed form projects onto U = P X instead (ubasis.cu)
    want_bt(p.first, p.first);
    if (p.first != p.second) {
      want_bt(p.first, p.second);
      want_bt(p.second, p.first);
      want_bt(p.second, p.second);
    }
  }
  size_t k_doubles = 0;
  int max_m = 0, max_n = 0, max_nx = 0;
  for (auto& p : newp) {
    const int m = pair_dim_h(c, p.first, p.second);
    k_doubles += 3 * (size_t)m * m + m;
    max_m = std::max(max_m, m);
  }
  for (int i = 0; i < n; i++) max_n = std::max(max_n, c->n_osv[i]);
  max_nx = max_n;
  double *sf_mem = nullptr, *bt_mem = nullptr, *k_mem = nullptr;
  TRY(palloc(c, &sf_mem, sf_doubles));
  TRY(palloc(c, &bt_mem, bt_doubles));
  TRY(palloc(c, &k_mem, k_doubles));
  {
    size_t off = 0;
    for (auto& j : sfj) {
      const size_t sz = (size_t)c->n_osv[j.x] * c->n_osv[j.y];
      j.S = sf_mem + off;
      j.F = sf_mem + off + sz;
      off += 2 * sz;
      c->sf_id[(size_t)j.x * n + j.y] = (int)c->S_h.size();
      c->S_h.push_back(j.S);
      c->F_h.push_back(j.F);
    }
  }
  {
    size_t off = 0;
    for (auto& j : pj) {
      j.out = bt_mem + off;
      off += (size_t)nx * c->n_osv[j.x];
      c->bt_id[(size_t)j.i * n + j.x] = (int)c->bt_h.size();
      c->bt_h.push_back(j.out);
    }
  }
  std::vector<KJob> kj;
  std::vector<PJob> pjb;
  std::vector<int> new_ids;
  // mixed form: leftovers Sh, Gh of the preconditioner basis (m^2 floats each per pair)
  const bool mixed_pc = mixed;
  float* shmem = nullptr;
  if (mixed_pc) {
    size_t shf = 0;
    for (auto& p : newp) {
      const size_t m = pair_dim_h(c, p.first, p.second);
      shf += 2 * m * m;
    }
    TRY(palloc(c, reinterpret_cast<double**>(&shmem), (shf + 1) / 2 + 1));
  }
  c->Sh_h.resize(c->K_h.size(), nullptr);
  c->Gh_h.resize(c->K_h.size(), nullptr);
  {
    size_t off = 0, shoff = 0;
    for (auto& p : newp) {
      const int i = p.first, j = p.second, m = pair_dim_h(c, i, j);
      const int pid = (int)c->K_h.size();
      if (pid >= c->cap_pairs) return fail(c, OSVMP2_E_ARG, "pair capacity exceeded");
      double* K = k_mem + off;
      double* X = K + (size_t)m * m;
      double* et = X + (size_t)m * m;
      double* Kt = et + m;
      off += 3 * (size_t)m * m + m;
      c->Kt_h.push_back(Kt);
      c->pair_id[(size_t)i * n + j] = pid;
      c->K_h.push_back(K);
      c->X_h.push_back(X);
      c->et_h.push_back(et);
      c->m_h.push_back(m);
      c->pi_h.push_back(i);
      c->pj_h.push_back(j);
      auto bt = [&](int a, int x) { return c->bt_h[c->bt_id[(size_t)a * n + x]]; };
      if (mixed) {
        // no raw-basis exchange block in the mixed form
      } else if (i == j) kj.push_back(KJob{i, j, bt(i, i), nullptr, nullptr, nullptr, K});
      else kj.push_back(KJob{i, j, bt(i, i), bt(i, j), bt(j, i), bt(j, j), K});
      float* Sh = nullptr;
      float* Gh = nullptr;
      if (mixed_pc) {
        Sh = shmem + shoff;
        Gh = Sh + (size_t)m * m;
        shoff += 2 * (size_t)m * m;
      }
      c->Sh_h.push_back(Sh);
      c->Gh_h.push_back(Gh);
      pjb.push_back(PJob{i, j, X, et, c->r_d + pid, Sh, Gh});
    }
  }
  // device tables
  TRY(upload(c, c->sf_id_d, c->sf_id));
  TRY(upload(c, c->pair_id_d, c->pair_id));
  TRY(upload(c, c->S_d, c->S_h));
  TRY(upload(c, c->F_d, c->F_h));
  TRY(upload(c, c->K_d, c->K_h));
  TRY(upload(c, c->X_d, c->X_h));
  TRY(upload(c, c->et_d, c->et_h));
  TRY(upload(c, c->Kt_d, c->Kt_h));
  TRY(upload(c, c->Sh_d, c->Sh_h));
  TRY(upload(c, c->Gh_d, c->Gh_h));
  // job arrays
  Tmp jsf, jpj, jk, jp, scr;
  TRY(tmp_alloc(c, jsf, sfj.size() * sizeof(SFJob)));
  TRY(tmp_alloc(c, jpj, pj.size() * sizeof(ProjJob)));
  TRY(tmp_alloc(c, jk, kj.size() * sizeof(KJob)));
  TRY(tmp_alloc(c, jp, pjb.size() * sizeof(PJob)));
  if (!sfj.empty()) CK(cudaMemcpyAsync(jsf.p, sfj.data(), sfj.size() * sizeof(SFJob), cudaMemcpyHostToDevice, c->st));
  if (!pj.empty()) CK(cudaMemcpyAsync(jpj.p, pj.data(), pj.size() * sizeof(ProjJob), cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(jk.p, kj.data(), kj.size() * sizeof(KJob), cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(jp.p, pjb.data(), pjb.size() * sizeof(PJob), cudaMemcpyHostToDevice, c->st));
  CK(cudaMemsetAsync(c->err_d, 0, sizeof(int), c->st));
  const Tables t = tables(c);
  double f_sf = 0, f_pj = 0, f_k = 0;
  for (auto& j : sfj) f_sf += 4.0 * nv * (double)c->n_osv[j.x] * c->n_osv[j.y];
  for (auto& j : pj) f_pj += 2.0 * nx * (double)nv * c->n_osv[j.x];
  for (auto& j : kj) { const double m = pair_dim_h(c, j.i, j.j); f_k += 2.0 * nx * m * m; }
  ph_begin(c, OSVMP2_PH_SF);
  launch_sf(t, c->sys.e_vir, (const SFJob*)jsf.p, (int)sfj.size(), max_n, c->st);
  ph_end(c, OSVMP2_PH_SF, f_sf);
  CK(cudaGetLastError());
  if (!mixed) {   // raw-basis projection and exchange blocks (FP64 form only)
    ph_begin(c, OSVMP2_PH_PROJECT);
    launch_project(bsrc(c), t, (const ProjJob*)jpj.p, (int)pj.size(), max_nx, 0, c->st);
    ph_end(c, OSVMP2_PH_PROJECT, f_pj, c->sys.B ? 8.0 * (double)pj.size() * nx * nv : 0.0);
    CK(cudaGetLastError());
    ph_begin(c, OSVMP2_PH_EXCHANGE);
    launch_exchange(t, nx, (const KJob*)jk.p, (int)kj.size(), max_m, 0, c->st);
    ph_end(c, OSVMP2_PH_EXCHANGE, f_k);
    CK(cudaGetLastError());
  }
  const int n_cta = std::min<int>((int)pjb.size(), 2 * c->num_sms);
  const int n_warps = std::min<int>((int)pjb.size(), 16 * c->num_sms);
  const int n_cta_pm = std::min<int>((int)pjb.size(), 3 * c->num_sms);
  const bool warp_pc = max_m <= PW_MAX_ORDER;
  TRY(tmp_alloc(c, scr, std::max({(size_t)n_cta * precond_scratch_doubles(max_m),
                                  warp_pc ? precond_w_scratch_doubles(max_m, n_warps) : (size_t)0,
                                  mixed_pc ? precond_mixed_scratch_doubles(max_m, n_cta_pm) : (size_t)0}) *
                                     sizeof(double)));
  Tmp pm_slots, pm_off, pm_m, pm_order;
  if (mixed_pc) {
    std::vector<long long> off(pjb.size());
    std::vector<int> md(pjb.size()), ord(pjb.size());
    long long tot = 0;
    for (size_t q = 0; q < pjb.size(); q++) {
      md[q] = pair_dim_h(c, pjb[q].i, pjb[q].j);
      off[q] = tot;
      tot += (long long)precond_mixed_slot_doubles(md[q]);
      ord[q] = (int)q;
    }
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return md[a] > md[b]; });
    TRY(tmp_alloc(c, pm_slots, (size_t)tot * sizeof(double)));
    TRY(tmp_alloc(c, pm_off, off.size() * sizeof(long long)));
    TRY(tmp_alloc(c, pm_m, md.size() * sizeof(int)));
    TRY(tmp_alloc(c, pm_order, ord.size() * sizeof(int)));
    CK(cudaMemcpyAsync(pm_off.p, off.data(), off.size() * sizeof(long long), cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(pm_m.p, md.data(), md.size() * sizeof(int), cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(pm_order.p, ord.data(), ord.size() * sizeof(int), cudaMemcpyHostToDevice, c->st));
  }
  double f_pc = 0.0;
  for (auto& j : pjb) {
    const double m = pair_dim_h(c, j.i, j.j);
    if (mixed_pc) {   // FP64: 1 - M^T M, its eigen-decomposition, Y^T F Y, X = Y W, W^T S W, W^T F W
      const double ni = c->n_osv[j.i], nj = (j.i == j.j) ? 0.0 : c->n_osv[j.j];
      f_pc += 2.0 * ni * nj * nj + 9.0 * nj * nj * nj + 2.0 * (m * m * nj + m * m * m) + 2.0 * m * m * m +
              8.0 * m * m * m;
    } else {
      f_pc += 9.0 * m * m * m + 2.0 * m * m * m + 2.0 * m * m * m + 9.0 * m * m * m + 2.0 * m * m * m;
    }
  }
  ph_begin(c, OSVMP2_PH_PRECOND);
  if (mixed_pc) {
    if (launch_precond_mixed(t, c->opts.tau_s, (const PJob*)jp.p, (const int*)pm_order.p, (int)pjb.size(), max_m,
                             (double*)pm_slots.p, (const long long*)pm_off.p, (const int*)pm_m.p, (double*)scr.p,
                             n_cta_pm, c->err_d, c->st))
      return fail(c, OSVMP2_E_ARG, "pair order %d exceeds the mixed preconditioner's shared scratch", max_m);
  } else if (warp_pc)
    launch_precond_w(t, c->opts.tau_s, (const PJob*)jp.p, (int)pjb.size(), max_m, (double*)scr.p, n_warps, c->err_d,
                     c->st);
  else
    launch_precond(t, c->opts.tau_s, (const PJob*)jp.p, (int)pjb.size(), max_m, (double*)scr.p, n_cta, c->err_d,
                   c->st);
  ph_end(c, OSVMP2_PH_PRECOND, f_pc);
  CK(cudaGetLastError());
  TRY(check_err_flag(c, "pair integrals"));
  c->r_h.resize(c->K_h.size());
  CK(cudaMemcpyAsync(c->r_h.data(), c->r_d, c->r_h.size() * sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (mixed) {   // U = P X, G = U^T B, K~ = G_i G_j^T (orthonormal pair basis)
    size_t ufl = 0, gfl = 0, us_rows = 0;
    int max_r = 0;
    const int ldv = (nv + 3) & ~3;     // TMA row stride: a multiple of 16 bytes
    std::vector<UJob> uj;
    std::vector<GJob> gj;
    std::vector<long long> g_usrow;    // row of slice 0 of U_p^T in Us, per G job
    std::vector<int> g_gsrow;          // row of slice 0 of G_p,x^T in Gs, per G job
    std::vector<tc::Job> ktj;          // K~ tiles from the slices of G
    const int ldg = (nx + 3) & ~3;
    long long gs_rows = 0;
    for (auto& p : newp) {
      const int pid = c->pair_id[(size_t)p.first * n + p.second];
      const int r = c->r_h[pid];
      max_r = std::max(max_r, r);
      ufl += (size_t)nv * r;
      gfl += (size_t)r * nx * (p.first == p.second ? 1 : 2);
      us_rows += tc::NSL * (size_t)r;
    }
    float *umem = nullptr, *gmem = nullptr, *usmem = nullptr;
    TRY(palloc(c, reinterpret_cast<double**>(&umem), (ufl + 1) / 2 + 1));
    TRY(palloc(c, reinterpret_cast<double**>(&gmem), (gfl + 1) / 2 + 1));
    TRY(palloc(c, reinterpret_cast<double**>(&usmem), (us_rows * ldv + 1) / 2 + 1));
    // rows past a pair's r (read by the fixed-height TMA boxes) must hold finite values
    CK(cudaMemsetAsync(usmem, 0, us_rows * ldv * sizeof(float), c->st));
    c->U_h.resize(c->K_h.size(), nullptr);
    c->Gi_h.resize(c->K_h.size(), nullptr);
    c->Gj_h.resize(c->K_h.size(), nullptr);
    c->us_base_h.resize(c->K_h.size(), nullptr);
    c->us_alloc_rows_h.resize(c->K_h.size(), 0);
    c->us_row_h.resize(c->K_h.size(), 0);
    c->us_ldv = ldv;
    size_t uo = 0, go = 0, urow = 0;
    double f_u = 0.0, f_g = 0.0, f_kg = 0.0;
    for (auto& p : newp) {
      const int i = p.first, j = p.second, pid = c->pair_id[(size_t)i * n + j];
      const int r = c->r_h[pid], m = pair_dim_h(c, i, j);
      float* U = umem + uo;
      uo += (size_t)nv * r;
      c->U_h[pid] = U;
      uj.push_back(UJob{i, j, U, usmem + urow * ldv, ldv});
      c->us_base_h[pid] = usmem;
      c->us_alloc_rows_h[pid] = (long long)us_rows;
      c->us_row_h[pid] = (long long)urow;
      f_u += 2.0 * nv * (double)m * r;
      float* Gi = gmem + go;
      go += (size_t)r * nx;
      gj.push_back(GJob{i, r, U, Gi});
      g_usrow.push_back((long long)urow);
      const long long gi_row = gs_rows;
      g_gsrow.push_back((int)gs_rows);
      gs_rows += tc::NSL * (long long)r;
      float* Gj = Gi;
      long long gj_row = gi_row;
      if (i != j) {
        Gj = gmem + go;
        go += (size_t)r * nx;
        gj.push_back(GJob{j, r, U, Gj});
        g_usrow.push_back((long long)urow);
        gj_row = gs_rows;
        g_gsrow.push_back((int)gs_rows);
        gs_rows += tc::NSL * (long long)r;
      }
      urow += tc::NSL * (size_t)r;
      f_g += (i != j ? 2.0 : 1.0) * 2.0 * r * (double)nv * nx;
      c->Gi_h[pid] = Gi;
      c->Gj_h[pid] = Gj;
      for (int m0 = 0; m0 < r; m0 += tc::BM)
        for (int n0 = 0; n0 < r; n0 += tc::BN) {
          tc::Job jb;
          jb.a_row = (int)(gi_row + m0);
          jb.a_sstride = r;
          jb.b_row = (int)(gj_row + n0);
          jb.b_sstride = r;
          jb.m_valid = std::min(tc::BM, r - m0);
          jb.n_valid = std::min(tc::BN, r - n0);
          jb.out = c->Kt_h[pid] + (size_t)m0 * r + n0;
          jb.ld_out = r;
          jb.m0 = m0;
          jb.n0 = n0;
          jb.s = 0.0;
          jb.x_row = jb.x_sstride = 0;
          ktj.push_back(jb);
        }
      f_kg += 2.0 * (double)r * r * nx;
    }
    std::vector<float*> uall(c->K_h.size(), nullptr);
    for (size_t q = 0; q < c->U_h.size(); q++) uall[q] = c->U_h[q];
    CK(cudaMemcpyAsync(c->U_d, uall.data(), uall.size() * sizeof(float*), cudaMemcpyHostToDevice, c->st));
    if (gs_rows + tc::BM >= (long long)INT32_MAX)
      return fail(c, OSVMP2_E_ARG, "G slice store exceeds the tensor-map row range");
    Tmp ju, jkt, gsl, glo, jgs;
    TRY(tmp_alloc(c, ju, uj.size() * sizeof(UJob)));
    TRY(tmp_alloc(c, glo, (gfl + 1) * sizeof(float)));   // remainders of the G pairs
    std::vector<GSJob> gsj;
    for (size_t q = 0; q < gj.size(); q++) gsj.push_back(GSJob{gj[q].G, gj[q].r, g_gsrow[q]});
    TRY(tmp_alloc(c, jgs, gsj.size() * sizeof(GSJob)));
    CK(cudaMemcpyAsync(jgs.p, gsj.data(), gsj.size() * sizeof(GSJob), cudaMemcpyHostToDevice, c->st));
    const long long lo_shift = (long long)((float*)glo.p - gmem);
    TRY(tmp_alloc(c, jkt, ktj.size() * sizeof(tc::Job)));
    TRY(tmp_alloc(c, gsl, (size_t)gs_rows * ldg * sizeof(float)));
    CK(cudaMemcpyAsync(ju.p, uj.data(), uj.size() * sizeof(UJob), cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(jkt.p, ktj.data(), ktj.size() * sizeof(tc::Job), cudaMemcpyHostToDevice, c->st));
    Tmp uscr;
    TRY(tmp_alloc(c, uscr, (size_t)n_cta * nv * std::max(max_r, 1) * sizeof(double)));
    ph_begin(c, OSVMP2_PH_PROJECT);
    launch_ubasis(t, (const UJob*)ju.p, (int)uj.size(), n_cta, (double*)uscr.p, max_r, c->st);
    CK(cudaGetLastError());
    TRY(gproj_tensor(c, gj, g_usrow, usmem, (long long)us_rows, ldv, lo_shift));
    launch_gslices((const GSJob*)jgs.p, (int)gsj.size(), max_r, nx, lo_shift, (float*)gsl.p, ldg, c->st);
    ph_end(c, OSVMP2_PH_PROJECT, f_u + f_g, c->sys.B ? 8.0 * (double)gj.size() * nx * nv : 0.0);
    CK(cudaGetLastError());
    ph_begin(c, OSVMP2_PH_EXCHANGE);
    if (launch_kt_tc((const float*)gsl.p, gs_rows, nx, ldg, (const tc::Job*)jkt.p, (int)ktj.size(), c->err_d, c->st))
      return fail(c, OSVMP2_E_CUDA, "tensor-map encoding for K~ failed");
    ph_end(c, OSVMP2_PH_EXCHANGE, f_kg);
    CK(cudaGetLastError());
    TRY(check_err_flag(c, "mixed pair build"));
  } else {   // K~ = X^T K X (used by the preconditioner-basis solver)
    std::vector<KtJob> ktj;
    for (size_t q = 0; q < kj.size(); q++) ktj.push_back(KtJob{kj[q].i, kj[q].j, c->Kt_h[c->pair_id[(size_t)kj[q].i * n + kj[q].j]]});
    Tmp jkt;
    TRY(tmp_alloc(c, jkt, ktj.size() * sizeof(KtJob)));
    CK(cudaMemcpyAsync(jkt.p, ktj.data(), ktj.size() * sizeof(KtJob), cudaMemcpyHostToDevice, c->st));
    launch_ktilde(t, (const KtJob*)jkt.p, (int)ktj.size(), (double*)scr.p, n_cta, max_m, c->st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->st));
  }
  (void)prec;
  CK(cudaStreamSynchronize(c->st));
  TRY(check_err_flag(c, "pair integrals"));
  return 0;
}

// S/F blocks (x < y) that are not built yet, without the pair data around them
// (the weak pairs need S_(i,j) only).
int ensure_sf_blocks_impl(osvmp2_ctx* c, const std::vector<std::pair<int, int>>& blocks) {
  const int n = c->sys.n_occ;
  std::vector<SFJob> sfj;
  size_t dbl = 0;
  for (auto& b : blocks) {
    const size_t id = (size_t)b.first * n + b.second;
    if (c->sf_id[id] == -1) {
      c->sf_id[id] = -2;
      sfj.push_back(SFJob{b.first, b.second, nullptr, nullptr});
      dbl += 2 * (size_t)c->n_osv[b.first] * c->n_osv[b.second];
    }
  }
  if (sfj.empty()) return 0;
  double* mem = nullptr;
  TRY(palloc(c, &mem, dbl));
  size_t off = 0;
  double fl = 0.0;
  for (auto& j : sfj) {
    const size_t sz = (size_t)c->n_osv[j.x] * c->n_osv[j.y];
    j.S = mem + off;
    j.F = mem + off + sz;
    off += 2 * sz;
    c->sf_id[(size_t)j.x * n + j.y] = (int)c->S_h.size();
    c->S_h.push_back(j.S);
    c->F_h.push_back(j.F);
    fl += 4.0 * c->sys.n_vir * (double)c->n_osv[j.x] * c->n_osv[j.y];
  }
  TRY(upload(c, c->sf_id_d, c->sf_id));
  TRY(upload(c, c->S_d, c->S_h));
  TRY(upload(c, c->F_d, c->F_h));
  Tmp jd;
  TRY(tmp_alloc(c, jd, sfj.size() * sizeof(SFJob)));
  CK(cudaMemcpyAsync(jd.p, sfj.data(), sfj.size() * sizeof(SFJob), cudaMemcpyHostToDevice, c->st));
  ph_begin(c, OSVMP2_PH_SF);
  launch_sf(tables(c), c->sys.e_vir, (const SFJob*)jd.p, (int)sfj.size(), 0, c->st);
  ph_end(c, OSVMP2_PH_SF, fl);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->st));
  return 0;
}
int ensure_sf_blocks(osvmp2_ctx* c, const std::vector<std::pair<int, int>>& blocks) {
  const int rc = ensure_sf_blocks_impl(c, blocks);
  if (rc != 0) {
    const std::string msg = c->err;
    cudaGetLastError();
    reset_pairs(c);
    c->err = msg;
  }
  return rc;
}

// s2b of every pair (Eq. s2b) on the device, into a host [n][n] matrix (diagonal 1).
int compute_s2b(osvmp2_ctx* c, std::vector<double>& s2b) {
  const int n = c->sys.n_occ;
  s2b.assign((size_t)n * n, 1.0);
  std::vector<int2> pl;
  pl.reserve((size_t)n * (n - 1) / 2);
  double fl = 0.0;
  for (int i = 0; i < n; i++)
    for (int j = i + 1; j < n; j++) {
      pl.push_back(make_int2(i, j));
      fl += 2.0 * c->sys.n_vir * (double)c->n_osv[i] * c->n_osv[j];
    }
  if (pl.empty()) return 0;
  Tmp pd, vd;
  TRY(tmp_alloc(c, pd, pl.size() * sizeof(int2)));
  TRY(tmp_alloc(c, vd, pl.size() * sizeof(double)));
  CK(cudaMemcpyAsync(pd.p, pl.data(), pl.size() * sizeof(int2), cudaMemcpyHostToDevice, c->st));
  ph_begin(c, OSVMP2_PH_SCREEN);
  launch_s2b(tables(c), (const int2*)pd.p, (int)pl.size(), (double*)vd.p,
             (int)std::min<size_t>(pl.size(), 4 * (size_t)c->num_sms), c->st);
  ph_end(c, OSVMP2_PH_SCREEN, fl);
  CK(cudaGetLastError());
  std::vector<double> v(pl.size());
  CK(cudaMemcpyAsync(v.data(), vd.p, v.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  for (size_t q = 0; q < pl.size(); q++) {
    s2b[(size_t)pl[q].x * n + pl[q].y] = v[q];
    s2b[(size_t)pl[q].y * n + pl[q].x] = v[q];
  }
  return 0;
}

bool screen_valid(const osvmp2_screen* sc) {
  return sc && sc->s2b_distant >= 0.0 && sc->s2b_close >= sc->s2b_distant && sc->s3b_min >= 0.0 &&
         std::isfinite(sc->s2b_close) && std::isfinite(sc->s3b_min);
}

}  // namespace

// ============================================================== C ABI
extern "C" {

int64_t osvmp2_kernel_launches(void) { return (int64_t)osv::g_launches.load(); }

void osvmp2_default_opts(osvmp2_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->tau_s = 1e-10;
  o->tol_update = 1e-7;
  o->tol_energy = 1e-13;
  o->max_iter = 100;
}

static bool opts_valid(const osvmp2_opts& o) {
  return o.max_iter > 0 && o.tau_s >= 0 && o.tol_update > 0 && o.tol_energy > 0 && o.mem_cap_mib >= 0 &&
         (o.osv_method == 0 || o.osv_method == 1) && o.rosv_max_rows >= 0 &&
         (o.osv_prec == OSVMP2_FP64 || o.osv_prec == OSVMP2_MIXED) && (o.no_autotune >= 0 && o.no_autotune <= 2);
}

int osvmp2_get_solve_plan(const osvmp2_ctx* c, int32_t* out) {
  if (!c || !out) return OSVMP2_E_ARG;
  out[0] = c->last_plan.ctas_per_sm;
  out[1] = c->last_plan.tiles;
  out[2] = c->last_plan.tuned ? 1 : 0;
  out[3] = (int32_t)c->plans.size();
  return OSVMP2_OK;
}

int osvmp2_set_opts(osvmp2_ctx* c, const osvmp2_opts* opts) {
  if (!c || !opts) return OSVMP2_E_ARG;
  c->err.clear();
  if (!opts_valid(*opts)) return fail(c, OSVMP2_E_ARG, "invalid options");
  c->opts = *opts;
  return OSVMP2_OK;
}

int osvmp2_create(osvmp2_ctx** out, int device, void* cuda_stream, const osvmp2_opts* opts) {
  if (!out) return OSVMP2_E_ARG;
  *out = nullptr;
  osvmp2_ctx* c = new osvmp2_ctx();
  c->device = device;
  c->st = (cudaStream_t)cuda_stream;
  osvmp2_default_opts(&c->opts);
  if (opts) c->opts = *opts;
  if (!opts_valid(c->opts)) {
    delete c;
    return OSVMP2_E_ARG;
  }
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaMalloc(&c->err_d, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&c->scal_d, 16 * sizeof(double));
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return OSVMP2_E_CUDA;
  }
  *out = c;
  return OSVMP2_OK;
}

void osvmp2_destroy(osvmp2_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  free_system(c);
  pool_trim(c);
  if (c->solve_exec) cudaGraphExecDestroy(c->solve_exec);
  if (c->cap_st) cudaStreamDestroy(c->cap_st);
  if (c->err_d) cudaFree(c->err_d);
  if (c->scal_d) cudaFree(c->scal_d);
  for (int ph = 0; ph < OSVMP2_NPHASE; ph++)
    for (cudaEvent_t e : c->ph_ev[ph]) cudaEventDestroy(e);
  delete c;
}

const char* osvmp2_last_error(const osvmp2_ctx* c) { return c ? c->err.c_str() : "null ctx"; }

// Mixed-form T_i of orbitals [i0, i0+b) on the tensor cores: B_i slices for up
// to nsl orbitals at a time, then the lower-triangle tiles of each T_i.
int tii_tensor(osvmp2_ctx* c, int i0, int b, double* T, float* Bt, int nsl, int ldx) {
  const int nv = c->sys.n_vir, nx = c->sys.n_aux, n = c->sys.n_occ;
  const int n_mt = (nv + tc::BM - 1) / tc::BM, n_nt = (nv + tc::BN - 1) / tc::BN;
  for (int u0 = 0; u0 < b; u0 += nsl) {
    const int nu = std::min(nsl, b - u0);
    launch_rslices(bsrc(c), i0 + u0, nu, Bt, ldx, c->st);
    CK(cudaGetLastError());
    std::vector<tc::Job> jobs;
    for (int u = 0; u < nu; u++) {
      const int i = i0 + u0 + u;
      for (int mt = 0; mt < n_mt; mt++)
        for (int nt = 0; nt < n_nt && nt * tc::BN < (mt + 1) * tc::BM; nt++) {
          tc::Job jb;
          jb.a_row = u * tc::NSL * nv + mt * tc::BM;
          jb.a_sstride = nv;
          jb.b_row = u * tc::NSL * nv + nt * tc::BN;
          jb.b_sstride = nv;
          jb.m_valid = std::min(tc::BM, nv - mt * tc::BM);
          jb.n_valid = std::min(tc::BN, nv - nt * tc::BN);
          jb.out = T + (size_t)(u0 + u) * nv * nv;
          jb.ld_out = nv;
          jb.m0 = mt * tc::BM;
          jb.n0 = nt * tc::BN;
          jb.s = 2.0 * c->f_h[(size_t)i * n + i];
          jobs.push_back(jb);
        }
    }
    Tmp jd;
    TRY(tmp_alloc(c, jd, jobs.size() * sizeof(tc::Job)));
    CK(cudaMemcpyAsync(jd.p, jobs.data(), jobs.size() * sizeof(tc::Job), cudaMemcpyHostToDevice, c->st));
    if (launch_tii_tc(Bt, (long long)nu * tc::NSL * nv, nx, ldx, (const tc::Job*)jd.p, (int)jobs.size(),
                      c->sys.e_vir, c->err_d, c->st))
      return fail(c, OSVMP2_E_CUDA, "tensor-map encoding for T_ii failed");
    CK(cudaGetLastError());
  }
  return 0;
}

// Randomized OSVs of orbitals [i0, i0+b) from their T_ii in T (Algorithm 3):
// V [b][kmax][nv], w [b][kmax], k [b] as the exact path writes them.
static int rosv_batch(osvmp2_ctx* c, double* T, int b, int i0, double l_osv, int n_max, int kmax, bool tensor,
                      const RosvLayout& rl, double* scr, float* slices, uint64_t key, double* V, double* w, int* k,
                      std::vector<int>& nrows_h) {
  const int nv = c->sys.n_vir, rows = rl.rows;
  double* Y = scr + rl.y;
  double* Z = scr + rl.z;
  double* Tt = scr + rl.tt;
  int* nrows = reinterpret_cast<int*>(scr + rl.nrows);
  auto tc_jobs = [&](int u, int m_rows, double* out, int out_rows, std::vector<tc::Job>& jobs) {
    const long long base = (long long)u * tc::NSL * (nv + rows);
    for (int m0 = 0; m0 < m_rows; m0 += tc::BM)
      for (int n0 = 0; n0 < nv; n0 += tc::BN) {
        tc::Job jb{};
        jb.a_row = (int)(base + (long long)tc::NSL * nv + m0);
        jb.a_sstride = rows;
        jb.b_row = (int)(base + n0);
        jb.b_sstride = nv;
        jb.m_valid = std::min(tc::BM, m_rows - m0);
        jb.n_valid = std::min(tc::BN, nv - n0);
        jb.out = out + ((size_t)u * out_rows + m0) * nv + n0;
        jb.ld_out = nv;
        jb.m0 = m0;
        jb.n0 = n0;
        jobs.push_back(jb);
      }
  };
  auto run_tc = [&](std::vector<tc::Job>& jobs) -> int {
    if (jobs.empty()) return 0;
    Tmp jd;
    TRY(tmp_alloc(c, jd, jobs.size() * sizeof(tc::Job)));
    CK(cudaMemcpyAsync(jd.p, jobs.data(), jobs.size() * sizeof(tc::Job), cudaMemcpyHostToDevice, c->st));
    if (launch_kt_tc(slices, rl.store_rows, nv, rl.ldk, (const tc::Job*)jd.p, (int)jobs.size(), c->err_d, c->st))
      return fail(c, OSVMP2_E_CUDA, "tensor-map encoding for the randomized OSVs failed");
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->st));   // the job list is a temporary
    return 0;
  };
  double fl = 2.0 * rows * (double)nv * nv * b;
  if (tensor) {
    launch_rosv_slices(0, T, b, nv, i0, key, nullptr, 0, nullptr, rows, slices, rl.ldk, c->st);
    launch_rosv_slices(1, T, b, nv, i0, key, nullptr, 0, nullptr, rows, slices, rl.ldk, c->st);
    CK(cudaGetLastError());
    std::vector<tc::Job> jobs;
    for (int u = 0; u < b; u++) tc_jobs(u, rows, Y, rows, jobs);
    TRY(run_tc(jobs));
  } else {
    launch_rosv_gemm64(0, T, b, nv, i0, key, nullptr, nullptr, rows, Y, c->st);
    CK(cudaGetLastError());
  }
  launch_rosv_finder(Y, b, nv, ROSV_WINDOW, n_max, l_osv, Z, nrows, scr + rl.wmax, c->err_d, c->st);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(nrows_h.data(), nrows, b * sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  for (int u = 0; u < b; u++) fl += 2.0 * nrows_h[u] * (double)nv * nv + 2.0 * nrows_h[u] * (double)nrows_h[u] * nv;
  if (tensor) {
    launch_rosv_slices(2, T, b, nv, i0, key, Z, n_max, nrows, rows, slices, rl.ldk, c->st);
    CK(cudaGetLastError());
    std::vector<tc::Job> jobs;
    for (int u = 0; u < b; u++) tc_jobs(u, nrows_h[u], Tt, n_max, jobs);
    TRY(run_tc(jobs));
  } else {
    launch_rosv_gemm64(1, T, b, nv, i0, key, Z, nrows, n_max, Tt, c->st);
    CK(cudaGetLastError());
  }
  // SVD of T~ through T~ T~^T = Q~ omega^2 Q~^T: the Gram matrices (padded to the
  // batch's largest row count; the padding adds only zero eigenvalues, never kept)
  // go through the OSV eigen-kernel with the cut l_osv^2, then Q = Z^T Q~.
  int ldm = 1;
  for (int u = 0; u < b; u++) ldm = std::max(ldm, nrows_h[u]);
  double* M = scr + rl.svd;
  double* Vs = M + (size_t)b * ldm * ldm;
  double* ws = Vs + (size_t)b * ldm * ldm;
  int* ks = reinterpret_cast<int*>(ws + (size_t)b * ldm);
  double* es = ws + (size_t)b * ldm + b;
  if (tensor) {
    CK(cudaMemsetAsync(M, 0, (size_t)b * ldm * ldm * sizeof(double), c->st));
    launch_rosv_slices(3, T, b, nv, i0, key, Tt, n_max, nrows, rows, slices, rl.ldk, c->st);
    CK(cudaGetLastError());
    std::vector<tc::Job> jobs;
    for (int u = 0; u < b; u++) {
      const long long base = (long long)u * tc::NSL * (nv + rows);
      for (int m0 = 0; m0 < nrows_h[u]; m0 += tc::BM)
        for (int n0 = 0; n0 < nrows_h[u]; n0 += tc::BN) {
          tc::Job jb{};
          jb.a_row = (int)(base + m0);
          jb.a_sstride = nv;
          jb.b_row = (int)(base + n0);
          jb.b_sstride = nv;
          jb.m_valid = std::min(tc::BM, nrows_h[u] - m0);
          jb.n_valid = std::min(tc::BN, nrows_h[u] - n0);
          jb.out = M + (size_t)u * ldm * ldm + (size_t)m0 * ldm + n0;
          jb.ld_out = ldm;
          jb.m0 = m0;
          jb.n0 = n0;
          jobs.push_back(jb);
        }
    }
    TRY(run_tc(jobs));
  } else {
    launch_rosv_gram64(Tt, nrows, b, nv, n_max, ldm, M, c->st);
    CK(cudaGetLastError());
  }
  const double thr2 = l_osv * l_osv;
  launch_eig_osv(M, b, ldm, thr2, ldm, Vs, ws, ks, es, c->err_d, false, c->st);
  launch_eig_back(M, b, ldm, thr2, ldm, Vs, ks, es, false, c->st);
  launch_rosv_backq(Vs, ws, ks, Z, nrows, b, nv, n_max, ldm, kmax, V, w, k, c->st);
  CK(cudaGetLastError());
  c->flops[OSVMP2_PH_EIG] += fl;
  return 0;
}

int osvmp2_build_osv(osvmp2_ctx* c, const osvmp2_system* s, double l_osv, int32_t* n_osv_host) {
  if (!c || !s) return OSVMP2_E_ARG;
  c->err.clear();
  if (s->n_occ <= 0 || s->n_vir <= 0 || s->n_aux <= 0)
    return fail(c, OSVMP2_E_ARG, "sizes must be positive (n_occ=%d n_vir=%d n_aux=%d)", s->n_occ, s->n_vir, s->n_aux);
  if (!s->B && !s->env) return fail(c, OSVMP2_E_ARG, "either B or env must be given");
  if (!s->f_occ || !s->e_vir) return fail(c, OSVMP2_E_ARG, "f_occ and e_vir are required");
  if ((int64_t)s->n_occ * s->n_occ > (int64_t)1 << 30) return fail(c, OSVMP2_E_ARG, "n_occ too large");
  if (c->opts.osv_method == 1 && !(l_osv > 0.0))
    return fail(c, OSVMP2_E_ARG, "randomized OSVs need l_osv > 0 (the range finder stops on it)");
  CK(cudaSetDevice(c->device));
  free_system(c);
  c->sys = *s;
  c->have_sys = true;
  c->l_osv = l_osv;
  c->key = mix64((uint64_t)s->seed ^ (STREAM_B * STREAM_MUL));
  c->r_occ.clear();
  if (s->r_occ) c->r_occ.assign(s->r_occ, s->r_occ + 3 * (size_t)s->n_occ);
  c->f_h.resize((size_t)s->n_occ * s->n_occ);
  CK(cudaMemcpy(c->f_h.data(), s->f_occ, c->f_h.size() * sizeof(double), cudaMemcpyDeviceToHost));
  const int n = s->n_occ, nv = s->n_vir;
  c->cap_pairs = n * (n + 1) / 2;
  TRY(dalloc_t(c, &c->n_osv_d, n));
  TRY(dalloc_t(c, &c->Q_d, n));
  TRY(dalloc_t(c, &c->sf_id_d, (size_t)n * n));
  TRY(dalloc_t(c, &c->pair_id_d, (size_t)n * n));
  TRY(dalloc_t(c, &c->S_d, c->cap_pairs));
  TRY(dalloc_t(c, &c->F_d, c->cap_pairs));
  TRY(dalloc_t(c, &c->K_d, c->cap_pairs));
  TRY(dalloc_t(c, &c->X_d, c->cap_pairs));
  TRY(dalloc_t(c, &c->et_d, c->cap_pairs));
  TRY(dalloc_t(c, &c->r_d, c->cap_pairs));
  TRY(dalloc_t(c, &c->Kt_d, c->cap_pairs));
  TRY(dalloc_t(c, &c->U_d, c->cap_pairs));
  TRY(dalloc_t(c, &c->Sh_d, c->cap_pairs));
  TRY(dalloc_t(c, &c->Gh_d, c->cap_pairs));
  c->sf_id.assign((size_t)n * n, -1);
  c->pair_id.assign((size_t)n * n, -1);
  c->bt_id.assign((size_t)n * n, -1);
  TRY(upload(c, c->sf_id_d, c->sf_id));
  TRY(upload(c, c->pair_id_d, c->pair_id));
  // batch the orbitals so that T, V and the eigen scratch stay within the budget below, in
  // batches of equal size (one CTA per orbital in the eigen kernel)
  const bool rosv = c->opts.osv_method == 1;
  const int n_max = rosv ? std::min(nv, c->opts.rosv_max_rows > 0 ? c->opts.rosv_max_rows : 256) : 0;
  const int kmax = rosv ? n_max : nv;
  const RosvLayout rl1 = rosv_layout(1, nv, ROSV_WINDOW, std::max(n_max, 1), kmax);
  const size_t per = ((size_t)nv * nv + (size_t)nv * kmax + kmax +
                      (rosv ? rl1.total + (size_t)tc::NSL * (nv + rl1.rows) * rl1.ldk / 2 + 1
                            : (size_t)nv * nv + eig_osv_scratch_doubles(nv, kmax))) * sizeof(double);
  // batch budget: a quarter of the free device memory, at most 64 GB (at most half of
  // the ctx's cap when one is set), at least 4 GB
  size_t budget = (size_t)4 << 30;
  {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) budget = std::max(budget, std::min(fr / 4, (size_t)64 << 30));
    else cudaGetLastError();
    if (c->opts.mem_cap_mib > 0) budget = std::min(budget, ((size_t)c->opts.mem_cap_mib << 20) / 2);
  }
  int nb = (int)std::max<size_t>(1, std::min<size_t>((size_t)n, budget / per));
  nb = std::min(nb, 4 * c->num_sms);
  {
    const int nbatch = (n + nb - 1) / nb;
    nb = (n + nbatch - 1) / nbatch;
  }
  const bool tii_tc = c->opts.osv_prec == OSVMP2_MIXED;
  const int ldx = (s->n_aux + 3) & ~3;
  const size_t slot_bytes = (size_t)tc::NSL * nv * ldx * sizeof(float);
  const int nsl = tii_tc ? (int)std::max<size_t>(1, std::min<size_t>((size_t)nb, ((size_t)1 << 30) / slot_bytes)) : 0;
  Tmp Tm, Vm, wm, km, sm, Bt;
  if (tii_tc) TRY(tmp_alloc(c, Bt, (size_t)nsl * slot_bytes));
  TRY(tmp_alloc(c, Tm, (size_t)nb * nv * nv * sizeof(double)));
  TRY(tmp_alloc(c, Vm, (size_t)nb * nv * kmax * sizeof(double)));
  TRY(tmp_alloc(c, wm, (size_t)nb * kmax * sizeof(double)));
  TRY(tmp_alloc(c, km, (size_t)nb * sizeof(int)));
  const RosvLayout rl = rosv_layout(nb, nv, ROSV_WINDOW, std::max(n_max, 1), kmax);
  Tmp rsl;
  if (rosv) {
    TRY(tmp_alloc(c, sm, rl.total * sizeof(double)));
    if (tii_tc) TRY(tmp_alloc(c, rsl, (size_t)rl.store_rows * rl.ldk * sizeof(float)));
    if (tii_tc && rl.store_rows + tc::BM >= (long long)INT32_MAX)
      return fail(c, OSVMP2_E_ARG, "randomized OSV slice store exceeds the tensor-map row range");
  } else {
    TRY(tmp_alloc(c, sm, (size_t)nb * eig_osv_scratch_doubles(nv, kmax) * sizeof(double)));
  }
  std::vector<int> nrows_h(nb);
  const uint64_t rosv_key = mix64((uint64_t)s->seed ^ (7ull * STREAM_MUL));
  Tmp qtab;
  TRY(tmp_alloc(c, qtab, 2 * (size_t)nb * sizeof(double*)));
  c->n_osv.assign(n, 0);
  c->Qp.assign(n, nullptr);
  c->Wp.assign(n, nullptr);
  CK(cudaMemsetAsync(c->err_d, 0, sizeof(int), c->st));
  std::vector<int> kh(nb);
  for (int i0 = 0; i0 < n; i0 += nb) {
    const int b = std::min(nb, n - i0);
    ph_begin(c, OSVMP2_PH_TII);
    if (tii_tc)
      TRY(tii_tensor(c, i0, b, (double*)Tm.p, (float*)Bt.p, nsl, ldx));
    else
      launch_tii(bsrc(c), s->e_vir, s->f_occ, n, i0, b, (double*)Tm.p, c->st);
    ph_end(c, OSVMP2_PH_TII, (double)b * nv * (double)nv * s->n_aux, s->B ? 8.0 * b * (double)nv * s->n_aux : 0.0);
    CK(cudaGetLastError());
    ph_begin(c, OSVMP2_PH_EIG);
    if (rosv) {
      TRY(rosv_batch(c, (double*)Tm.p, b, i0, l_osv, n_max, kmax, tii_tc, rl, (double*)sm.p, (float*)rsl.p, rosv_key,
                     (double*)Vm.p, (double*)wm.p, (int*)km.p, nrows_h));
      ph_end(c, OSVMP2_PH_EIG, 0.0);
      int h = 0;
      CK(cudaMemcpyAsync(&h, c->err_d, sizeof(int), cudaMemcpyDeviceToHost, c->st));
      CK(cudaStreamSynchronize(c->st));
      if (h & ERR_SIZE)
        return fail(c, OSVMP2_E_NUMERIC,
                    "randomized OSVs: the range finder needs more than %d rows for an orbital of [%d, %d) "
                    "(raise opts.rosv_max_rows)", n_max, i0, i0 + b);
    } else {
      const double nd = nv;
      const bool full = (nv <= 160) || (l_osv <= 0.0);
      const double fl = (double)b * (full ? 9.0 * nd * nd * nd : (4.0 / 3.0) * nd * nd * nd);
      ph_begin(c, OSVMP2_PH_K_EIG);
      launch_eig_osv((double*)Tm.p, b, nv, l_osv, kmax, (double*)Vm.p, (double*)wm.p, (int*)km.p, (double*)sm.p,
                     c->err_d, tii_tc, c->st);
      ph_end(c, OSVMP2_PH_K_EIG, fl);
      launch_eig_back((double*)Tm.p, b, nv, l_osv, kmax, (double*)Vm.p, (const int*)km.p, (double*)sm.p, tii_tc,
                      c->st);
      ph_end(c, OSVMP2_PH_EIG, fl);
    }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(kh.data(), km.p, b * sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    ph_collect(c);
    size_t tot = 0;
    for (int u = 0; u < b; u++) tot += (size_t)kh[u] * (nv + 1);
    double* mem = nullptr;
    TRY(dalloc_t(c, &mem, tot));
    std::vector<double*> qd(2 * b);
    size_t off = 0;
    for (int u = 0; u < b; u++) {
      c->n_osv[i0 + u] = kh[u];
      c->Qp[i0 + u] = mem + off;
      off += (size_t)kh[u] * nv;
      c->Wp[i0 + u] = mem + off;
      off += kh[u];
      qd[u] = c->Qp[i0 + u];
      qd[b + u] = c->Wp[i0 + u];
    }
    CK(cudaMemcpyAsync(qtab.p, qd.data(), 2 * b * sizeof(double*), cudaMemcpyHostToDevice, c->st));
    launch_pack_q((double*)Vm.p, (double*)wm.p, b, nv, kmax, (int*)km.p, (double* const*)qtab.p,
                  (double* const*)qtab.p + b, c->st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->st));
  }
  TRY(check_err_flag(c, "OSV build"));
  for (int i = 0; i < n; i++)
    if (c->n_osv[i] == 0) return fail(c, OSVMP2_E_NUMERIC, "orbital %d has no OSV above l_osv", i);
  TRY(upload(c, c->n_osv_d, c->n_osv));
  TRY(upload(c, c->Q_d, c->Qp));
  CK(cudaStreamSynchronize(c->st));
  c->have_osv = true;
  if (n_osv_host) std::copy(c->n_osv.begin(), c->n_osv.end(), n_osv_host);
  return OSVMP2_OK;
}

int osvmp2_get_osv(osvmp2_ctx* c, int32_t i, double* Q, double* w) {
  if (!c) return OSVMP2_E_ARG;
  if (!c->have_osv) return fail(c, OSVMP2_E_STATE, "no OSVs built");
  if (i < 0 || i >= c->sys.n_occ) return fail(c, OSVMP2_E_ARG, "orbital %d out of range", i);
  const size_t k = c->n_osv[i];
  if (Q) CK(cudaMemcpyAsync(Q, c->Qp[i], k * c->sys.n_vir * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  if (w) CK(cudaMemcpyAsync(w, c->Wp[i], k * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  return OSVMP2_OK;
}

int osvmp2_pair_integrals(osvmp2_ctx* c, const int32_t* pairs, int64_t n_pairs, osvmp2_prec prec) {
  if (!c) return OSVMP2_E_ARG;
  c->err.clear();
  if (n_pairs < 0 || (n_pairs > 0 && !pairs)) return fail(c, OSVMP2_E_ARG, "bad pair list");
  std::vector<std::pair<int, int>> req;
  for (int64_t p = 0; p < n_pairs; p++) req.push_back({pairs[2 * p], pairs[2 * p + 1]});
  CK(cudaSetDevice(c->device));
  return ensure_pairs(c, req, prec);
}

int osvmp2_get_pair_blocks(osvmp2_ctx* c, int32_t i, int32_t j, double* K, double* S, double* F) {
  if (!c) return OSVMP2_E_ARG;
  if (!c->have_osv) return fail(c, OSVMP2_E_STATE, "no OSVs built");
  const int n = c->sys.n_occ;
  if (i < 0 || j < i || j >= n) return fail(c, OSVMP2_E_ARG, "pair (%d,%d) invalid", i, j);
  const int pid = c->pair_id[(size_t)i * n + j];
  if (pid < 0) return fail(c, OSVMP2_E_STATE, "pair (%d,%d) not built", i, j);
  const int m = c->m_h[pid];
  if (K) CK(cudaMemcpyAsync(K, c->K_h[pid], (size_t)m * m * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  // S and F assembled on the host side of the copy from their blocks
  int blocks[2] = {i, j};
  const int nb = (i == j) ? 1 : 2;
  int roff = 0;
  for (int a = 0; a < nb; a++) {
    int coff = 0;
    for (int b = 0; b < nb; b++) {
      const int x = blocks[a], y = blocks[b];
      const int nx = c->n_osv[x], ny = c->n_osv[y];
      const int lo = std::min(x, y), hi = std::max(x, y);
      const int id = c->sf_id[(size_t)lo * n + hi];
      std::vector<double> hs((size_t)c->n_osv[lo] * c->n_osv[hi]), hf(hs.size());
      CK(cudaMemcpyAsync(hs.data(), c->S_h[id], hs.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st));
      CK(cudaMemcpyAsync(hf.data(), c->F_h[id], hf.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st));
      CK(cudaStreamSynchronize(c->st));
      std::vector<double> bs((size_t)nx * ny), bf(bs.size());
      for (int r = 0; r < nx; r++)
        for (int q = 0; q < ny; q++) {
          const size_t src = (x <= y) ? (size_t)r * ny + q : (size_t)q * nx + r;
          bs[(size_t)r * ny + q] = hs[src];
          bf[(size_t)r * ny + q] = hf[src];
        }
      for (int r = 0; r < nx; r++) {
        if (S) CK(cudaMemcpy(S + (size_t)(roff + r) * m + coff, bs.data() + (size_t)r * ny, ny * sizeof(double),
                             cudaMemcpyHostToDevice));
        if (F) CK(cudaMemcpy(F + (size_t)(roff + r) * m + coff, bf.data() + (size_t)r * ny, ny * sizeof(double),
                             cudaMemcpyHostToDevice));
      }
      coff += ny;
    }
    roff += c->n_osv[blocks[a]];
  }
  CK(cudaStreamSynchronize(c->st));
  return OSVMP2_OK;
}

int osvmp2_get_precond(osvmp2_ctx* c, int32_t i, int32_t j, double* X, double* et, int32_t* r_out) {
  if (!c) return OSVMP2_E_ARG;
  if (!c->have_osv) return fail(c, OSVMP2_E_STATE, "no OSVs built");
  const int n = c->sys.n_occ;
  if (i < 0 || j < i || j >= n) return fail(c, OSVMP2_E_ARG, "pair (%d,%d) invalid", i, j);
  const int pid = c->pair_id[(size_t)i * n + j];
  if (pid < 0) return fail(c, OSVMP2_E_STATE, "pair (%d,%d) not built", i, j);
  const int m = c->m_h[pid];
  if (X) CK(cudaMemcpyAsync(X, c->X_h[pid], (size_t)m * m * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  if (et) CK(cudaMemcpyAsync(et, c->et_h[pid], (size_t)m * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (r_out) *r_out = c->r_h[pid];
  return OSVMP2_OK;
}

int osvmp2_solve(osvmp2_ctx* c, const int32_t* orbs, int32_t n_orbs, osvmp2_prec prec, double* e_out,
                 double* pair_e_out, int32_t* iters_out) {
  if (!c) return OSVMP2_E_ARG;
  c->err.clear();
  if (!c->have_osv) return fail(c, OSVMP2_E_STATE, "osvmp2_build_osv has not been called");
  if (!orbs || n_orbs <= 0 || !e_out) return fail(c, OSVMP2_E_ARG, "orbs, n_orbs > 0 and e_out are required");
  const int n = c->sys.n_occ;
  for (int a = 0; a < n_orbs; a++) {
    if (orbs[a] < 0 || orbs[a] >= n) return fail(c, OSVMP2_E_ARG, "orbital %d out of range", orbs[a]);
    if (a > 0 && orbs[a] <= orbs[a - 1]) return fail(c, OSVMP2_E_ARG, "orbs must be strictly ascending");
  }
  CK(cudaSetDevice(c->device));
  std::vector<std::pair<int, int>> req;
  for (int a = 0; a < n_orbs; a++)
    for (int b = a; b < n_orbs; b++) req.push_back({orbs[a], orbs[b]});
  TRY(ensure_pairs(c, req, prec));
  const int np = (int)req.size();
  size_t tot = 0;
  int max_m = 0;
  for (auto& p : req) {
    const int m = pair_dim_h(c, p.first, p.second);
    tot += 4 * (size_t)m * m;
    max_m = std::max(max_m, m);
  }
  const int n_cta = std::min(np, 2 * c->num_sms);
  Tmp mem, wmem, ptrs, orbd, pe, pu;
  TRY(tmp_alloc(c, mem, tot * sizeof(double)));
  TRY(tmp_alloc(c, wmem, (size_t)n_cta * 2 * max_m * max_m * sizeof(double)));
  TRY(tmp_alloc(c, ptrs, (size_t)(4 * np + 2 * n_cta) * sizeof(double*)));
  TRY(tmp_alloc(c, orbd, n_orbs * sizeof(int)));
  TRY(tmp_alloc(c, pe, (np + 1) * sizeof(double)));
  TRY(tmp_alloc(c, pu, (np + 1) * sizeof(double)));
  std::vector<double*> hp(4 * np + 2 * n_cta);
  size_t off = 0;
  for (int q = 0; q < np; q++) {
    const size_t m2 = (size_t)pair_dim_h(c, req[q].first, req[q].second) * pair_dim_h(c, req[q].first, req[q].second);
    for (int u = 0; u < 4; u++) { hp[u * np + q] = (double*)mem.p + off; off += m2; }
  }
  for (int u = 0; u < 2 * n_cta; u++) hp[4 * np + u] = (double*)wmem.p + (size_t)u * max_m * max_m;
  CK(cudaMemcpyAsync(ptrs.p, hp.data(), hp.size() * sizeof(double*), cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(orbd.p, orbs, n_orbs * sizeof(int), cudaMemcpyHostToDevice, c->st));
  double** P = (double**)ptrs.p;
  SubDev sd{n_orbs, (const int*)orbd.p, P, P + np, P + 2 * np, P + 3 * np, P + 4 * np, (double*)pe.p, (double*)pu.p};
  const Tables t = tables(c);
  launch_sub_prepare(t, sd, np, n_cta, c->st);
  CK(cudaGetLastError());
  double e_prev = 0.0, e = 0.0, um = 0.0;
  int it = 1;
  bool conv = false;
  for (; it <= c->opts.max_iter; it++) {
    ph_begin(c, OSVMP2_PH_SUBSOLVE);
    launch_sub_residual(t, sd, np, n_cta, c->st);
    launch_sub_update(t, sd, np, n_cta, c->st);
    ph_end(c, OSVMP2_PH_SUBSOLVE, 0.0);
    CK(cudaGetLastError());
    double h[2];
    CK(cudaMemcpyAsync(&h[0], (double*)pe.p + np, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaMemcpyAsync(&h[1], (double*)pu.p + np, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    ph_collect(c);
    e = h[0];
    um = h[1];
    if (!std::isfinite(e) || !std::isfinite(um)) return fail(c, OSVMP2_E_NUMERIC, "non-finite energy in solve");
    if (um < c->opts.tol_update && std::fabs(e - e_prev) < c->opts.tol_energy) { conv = true; break; }
    e_prev = e;
  }
  *e_out = e;
  if (iters_out) *iters_out = std::min(it, c->opts.max_iter);
  if (pair_e_out) {
    CK(cudaMemcpyAsync(pair_e_out, pe.p, np * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
  }
  if (!conv) return fail(c, OSVMP2_E_NOCONV, "solve did not converge in %d iterations (max|update| %.3e)",
                         c->opts.max_iter, um);
  return OSVMP2_OK;
}

int osvmp2_mbe3_fragments(const double* r_occ, int32_t n_occ, double r2, double r3, int64_t cap, int32_t* orbs_out,
                          int32_t* weights_out, int64_t* n_out) {
  if (!r_occ || n_occ <= 0 || !n_out || r2 < 0 || r3 < 0) return OSVMP2_E_ARG;
  std::vector<Frag> fr;
  enumerate_fragments(r_occ, n_occ, r2, r3, fr);
  *n_out = (int64_t)fr.size();
  if (orbs_out || weights_out) {
    if (cap < (int64_t)fr.size()) return OSVMP2_E_ARG;
    for (size_t f = 0; f < fr.size(); f++) {
      if (orbs_out)
        for (int u = 0; u < 3; u++) orbs_out[3 * f + u] = fr[f].orbs[u];
      if (weights_out) weights_out[f] = fr[f].weight;
    }
  }
  return OSVMP2_OK;
}

// Mixed form: the overlaps Sigma_(lo,hi) = U_lo^T U_hi of every pair couple that
// a coupling term of some fragment uses (pair p with the pairs (a,c), (c,b) of
// its fragment), each computed once on the tensor cores from the U slices.
struct SigmaStore {
  Tmp data, off, hi, pos;
  SigmaTable tab{};
};
int build_sigma_table(osvmp2_ctx* c, SigmaStore& ss) {
  const int n = c->sys.n_occ, npairs = (int)c->K_h.size();
  std::vector<std::pair<int, int>> cps;
  for (const Frag& fr : c->frags) {
    int orbs[3], nc = 0;
    for (int u = 0; u < 3; u++)
      if (fr.orbs[u] >= 0) orbs[nc++] = fr.orbs[u];
    auto pid_of = [&](int x, int y) {
      const int a = std::min(orbs[x], orbs[y]), b = std::max(orbs[x], orbs[y]);
      return c->pair_id[(size_t)a * n + b];
    };
    for (int a = 0; a < nc; a++)
      for (int b = a; b < nc; b++) {
        const int P = pid_of(a, b);
        for (int k = 0; k < nc; k++) {
          if (k != b) { const int Q = pid_of(a, k); if (Q != P) cps.push_back({std::min(P, Q), std::max(P, Q)}); }
          if (k != a) { const int Q = pid_of(k, b); if (Q != P) cps.push_back({std::min(P, Q), std::max(P, Q)}); }
        }
      }
  }
  std::sort(cps.begin(), cps.end());
  cps.erase(std::unique(cps.begin(), cps.end()), cps.end());
  std::vector<int> off(npairs + 1, 0), hi(cps.size());
  std::vector<long long> pos(cps.size());
  long long tot = 0;
  for (size_t u = 0; u < cps.size(); u++) {
    off[cps[u].first + 1]++;
    hi[u] = cps[u].second;
    pos[u] = tot;
    tot += (long long)c->r_h[cps[u].first] * c->r_h[cps[u].second];
  }
  for (int q = 0; q < npairs; q++) off[q + 1] += off[q];
  TRY(tmp_alloc(c, ss.data, (size_t)std::max<long long>(tot, 1) * sizeof(float)));
  TRY(tmp_alloc(c, ss.off, off.size() * sizeof(int)));
  TRY(tmp_alloc(c, ss.hi, std::max<size_t>(hi.size(), 1) * sizeof(int)));
  TRY(tmp_alloc(c, ss.pos, std::max<size_t>(pos.size(), 1) * sizeof(long long)));
  CK(cudaMemcpyAsync(ss.off.p, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice, c->st));
  if (!cps.empty()) {
    CK(cudaMemcpyAsync(ss.hi.p, hi.data(), hi.size() * sizeof(int), cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(ss.pos.p, pos.data(), pos.size() * sizeof(long long), cudaMemcpyHostToDevice, c->st));
  }
  ss.tab = SigmaTable{(const int*)ss.off.p, (const int*)ss.hi.p, (const long long*)ss.pos.p, (const float*)ss.data.p};
  // tensor-core tiles, grouped by the U slice stores of the two pairs
  std::map<std::pair<const float*, const float*>, std::vector<tc::Job>> groups;
  for (size_t u = 0; u < cps.size(); u++) {
    const int lo = cps[u].first, hq = cps[u].second;
    const int rl = c->r_h[lo], rh = c->r_h[hq];
    if (!c->us_base_h[lo] || !c->us_base_h[hq]) return fail(c, OSVMP2_E_STATE, "pair without U slices");
    auto& js = groups[{c->us_base_h[lo], c->us_base_h[hq]}];
    for (int m0 = 0; m0 < rl; m0 += tc::BM)
      for (int n0 = 0; n0 < rh; n0 += tc::BN) {
        tc::Job jb;
        jb.a_row = (int)(c->us_row_h[lo] + m0);
        jb.a_sstride = rl;
        jb.b_row = (int)(c->us_row_h[hq] + n0);
        jb.b_sstride = rh;
        jb.m_valid = std::min(tc::BM, rl - m0);
        jb.n_valid = std::min(tc::BN, rh - n0);
        jb.out = (float*)ss.data.p + pos[u] + (size_t)m0 * rh + n0;
        jb.ld_out = rh;
        jb.m0 = m0;
        jb.n0 = n0;
        jb.s = 0.0;
        js.push_back(jb);
      }
  }
  for (auto& g : groups) {
    const float* A = g.first.first;
    const float* B = g.first.second;
    long long ar = 0, br = 0;
    for (int q = 0; q < npairs; q++) {
      if (c->us_base_h[q] == A) ar = c->us_alloc_rows_h[q];
      if (c->us_base_h[q] == B) br = c->us_alloc_rows_h[q];
    }
    Tmp jd;
    TRY(tmp_alloc(c, jd, g.second.size() * sizeof(tc::Job)));
    CK(cudaMemcpyAsync(jd.p, g.second.data(), g.second.size() * sizeof(tc::Job), cudaMemcpyHostToDevice, c->st));
    if (launch_rows_tc(A, ar, B, br, c->sys.n_vir, c->us_ldv, (const tc::Job*)jd.p, (int)g.second.size(), c->err_d,
                       c->st))
      return fail(c, OSVMP2_E_CUDA, "tensor-map encoding for the pair-couple overlaps failed");
    CK(cudaGetLastError());
  }
  return 0;
}

// Distance-rule fragment list of osvmp2_mbe3_energy / osvmp2_energy_grad into c->frags.
static int distance_fragments(osvmp2_ctx* c, double r2, double r3, double* e_out) {
  if (!c) return OSVMP2_E_ARG;
  c->err.clear();
  if (!c->have_osv) return fail(c, OSVMP2_E_STATE, "osvmp2_build_osv has not been called");
  if (!e_out) return fail(c, OSVMP2_E_ARG, "e_out is required");
  if (c->r_occ.empty()) return fail(c, OSVMP2_E_ARG, "system has no r_occ (needed for fragment lists)");
  if (!(r2 >= 0) || !(r3 >= 0)) return fail(c, OSVMP2_E_ARG, "cutoffs must be >= 0");
  CK(cudaSetDevice(c->device));
  enumerate_fragments(c->r_occ.data(), c->sys.n_occ, r2, r3, c->frags);
  c->weak.clear();
  c->weak_e.clear();
  return 0;
}

// MBE(3) energy of the fragments in c->frags; with tstore != NULL the converged
// amplitudes of every fragment are kept (fragment f at tstore + toff[f], local
// pairs a<=b in order).
static int mbe3_core(osvmp2_ctx* c, osvmp2_prec prec, double* e_out, osvmp2_mbe_stats* stats, Tmp* tstore,
                     std::vector<long long>* toff) {
  const int n = c->sys.n_occ;
  const int nf = (int)c->frags.size();
  std::vector<std::pair<int, int>> req;
  int64_t ns = 0, npair = 0, ntri = 0;
  for (auto& f : c->frags) {
    const int nc = (f.orbs[1] < 0) ? 1 : (f.orbs[2] < 0 ? 2 : 3);
    if (nc == 1) { ns++; req.push_back({f.orbs[0], f.orbs[0]}); }
    else if (nc == 2) { npair++; req.push_back({f.orbs[0], f.orbs[1]}); }
    else ntri++;
  }
  TRY(ensure_pairs(c, req, prec));
  // processing order: largest estimated cost first
  std::vector<int> order(nf);
  std::vector<double> cost(nf, 0.0);
  int max_m = 0;
  for (int f = 0; f < nf; f++) {
    order[f] = f;
    const Frag& fr = c->frags[f];
    for (int a = 0; a < 3; a++)
      for (int b = a; b < 3; b++) {
        if (fr.orbs[a] < 0 || fr.orbs[b] < 0) continue;
        const double m = pair_dim_h(c, fr.orbs[a], fr.orbs[b]);
        cost[f] += m * m * m;
        max_m = std::max(max_m, (int)m);
      }
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<int> orbs_h(3 * (size_t)nf), w_h(nf);
  for (int f = 0; f < nf; f++) {
    for (int u = 0; u < 3; u++) orbs_h[3 * f + u] = c->frags[f].orbs[u];
    w_h[f] = c->frags[f].weight;
  }
  // scratch sized for the largest launch: the mixed solver's autotuner tries up to 3 CTAs per SM
  int n_cta = std::max(1, std::min(nf, (prec == OSVMP2_MIXED ? 3 : 2) * c->num_sms));
  Tmp d_orbs, d_order, d_w, d_out, d_cnt, d_scr;
  TRY(tmp_alloc(c, d_orbs, orbs_h.size() * sizeof(int)));
  TRY(tmp_alloc(c, d_order, nf * sizeof(int)));
  TRY(tmp_alloc(c, d_w, nf * sizeof(int)));
  TRY(tmp_alloc(c, d_out, nf * sizeof(FragOut)));
  TRY(tmp_alloc(c, d_cnt, sizeof(int)));
  const size_t per_cta = (prec == OSVMP2_MIXED) ? frag_mixed_scratch_doubles(max_m) : frag_scratch_doubles(max_m);
  TRY(tmp_alloc(c, d_scr, (size_t)n_cta * per_cta * sizeof(double)));
  CK(cudaMemcpyAsync(d_orbs.p, orbs_h.data(), orbs_h.size() * sizeof(int), cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(d_order.p, order.data(), nf * sizeof(int), cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(d_w.p, w_h.data(), nf * sizeof(int), cudaMemcpyHostToDevice, c->st));
  Tmp d_toff;
  double* tdst = nullptr;
  if (tstore) {
    toff->assign(nf, 0);
    long long tot = 0;
    for (int f = 0; f < nf; f++) {
      (*toff)[f] = tot;
      const Frag& fr = c->frags[f];
      for (int a = 0; a < 3; a++)
        for (int b = a; b < 3; b++)
          if (fr.orbs[a] >= 0 && fr.orbs[b] >= 0) {
            const long long m = pair_dim_h(c, fr.orbs[a], fr.orbs[b]);
            tot += m * m;
          }
    }
    TRY(tmp_alloc(c, *tstore, (size_t)tot * sizeof(double)));
    TRY(tmp_alloc(c, d_toff, nf * sizeof(long long)));
    CK(cudaMemcpyAsync(d_toff.p, toff->data(), nf * sizeof(long long), cudaMemcpyHostToDevice, c->st));
    tdst = (double*)tstore->p;
  }
  SolveOpts so{c->opts.tol_update, c->opts.tol_energy, c->opts.max_iter};
  SigmaStore sig;
  ph_begin(c, OSVMP2_PH_SOLVE);
  if (prec == OSVMP2_MIXED) {
    CK(cudaMemsetAsync(c->err_d, 0, sizeof(int), c->st));
    ph_begin(c, OSVMP2_PH_SIGMA);
    TRY(build_sigma_table(c, sig));
    ph_end(c, OSVMP2_PH_SIGMA, 0.0);
    const Tables tb = tables(c);
    auto solve = [&](const SolvePlan& pl, cudaStream_t st) {
      SolveOpts o = so;
      o.tiles = pl.tiles;
      const int nc = std::max(1, std::min(nf, pl.ctas_per_sm * c->num_sms));
      launch_frag_solve_mixed(tb, (const int*)d_orbs.p, (const int*)d_order.p, nf, max_m, o, sig.tab,
                              (double*)d_scr.p, nc, (int*)d_cnt.p, (FragOut*)d_out.p, tdst,
                              (const long long*)d_toff.p, c->err_d, pl.ctas_per_sm, st);
    };
    // autotuner: the first call for a (fragment count, largest pair order) times
    // every candidate plan on the full solve and keeps the fastest
    const std::pair<int, int> key{nf, max_m};
    auto it = c->plans.find(key);
    if (it == c->plans.end()) {
      SolvePlan best;
      if (c->opts.no_autotune == 2) best.ctas_per_sm = 3;
      if (!c->opts.no_autotune) {
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        float best_ms = 1e30f;
        for (int cps = 1; cps <= 3; cps++)
          for (int tl = 0; tl <= 1; tl++) {
            SolvePlan pl;
            pl.ctas_per_sm = cps;
            pl.tiles = tl;
            CK(cudaEventRecord(e0, c->st));
            solve(pl, c->st);
            CK(cudaEventRecord(e1, c->st));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best_ms) {
              best_ms = ms;
              best = pl;
            }
          }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        best.tuned = true;
        best.ms = best_ms;
        CK(cudaMemsetAsync(c->err_d, 0, sizeof(int), c->st));
      }
      it = c->plans.emplace(key, best).first;
    }
    c->last_plan = it->second;
    // the solve and the MBE(3) sum replayed as one CUDA graph (recorded on a
    // private stream, launched on the ctx stream; an instantiated graph is
    // updated in place when only its arguments changed)
    bool graphed = false;
    ph_begin(c, OSVMP2_PH_K_FRAGSOLVE);
    if (!c->cap_st) cudaStreamCreateWithFlags(&c->cap_st, cudaStreamNonBlocking);
    if (c->cap_st && cudaStreamBeginCapture(c->cap_st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      solve(it->second, c->cap_st);
      launch_weighted_sum((const FragOut*)d_out.p, (const int*)d_w.p, nf, c->scal_d, c->cap_st);
      cudaGraph_t g = nullptr;
      if (cudaStreamEndCapture(c->cap_st, &g) == cudaSuccess && g) {
        if (c->solve_exec) {
          cudaGraphExecUpdateResultInfo info;
          if (cudaGraphExecUpdate(c->solve_exec, g, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(c->solve_exec);
            c->solve_exec = nullptr;
          }
        }
        if (!c->solve_exec && cudaGraphInstantiate(&c->solve_exec, g, 0) != cudaSuccess) {
          cudaGetLastError();
          c->solve_exec = nullptr;
        }
        if (c->solve_exec && cudaGraphLaunch(c->solve_exec, c->st) == cudaSuccess) graphed = true;
        cudaGraphDestroy(g);
      }
      cudaGetLastError();
    }
    if (!graphed) {
      solve(it->second, c->st);
      launch_weighted_sum((const FragOut*)d_out.p, (const int*)d_w.p, nf, c->scal_d, c->st);
    }
    ph_end(c, OSVMP2_PH_K_FRAGSOLVE, 0.0);
  } else {
    ph_begin(c, OSVMP2_PH_K_FRAGSOLVE);
    launch_frag_solve(tables(c), (const int*)d_orbs.p, (const int*)d_order.p, nf, max_m, so, (double*)d_scr.p, n_cta,
                      (int*)d_cnt.p, (FragOut*)d_out.p, tdst, (const long long*)d_toff.p, c->st);
    launch_weighted_sum((const FragOut*)d_out.p, (const int*)d_w.p, nf, c->scal_d, c->st);
    ph_end(c, OSVMP2_PH_K_FRAGSOLVE, 0.0);
  }
  CK(cudaGetLastError());
  ph_end(c, OSVMP2_PH_SOLVE, 0.0);
  ph_begin(c, OSVMP2_PH_MBE_SUM);   // (inside the solve phase: the sum is part of the same graph)
  ph_end(c, OSVMP2_PH_MBE_SUM, 2.0 * nf);
  c->frag_out.resize(nf);
  CK(cudaMemcpyAsync(c->frag_out.data(), d_out.p, nf * sizeof(FragOut), cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(e_out, c->scal_d, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  ph_collect(c);
  if (prec == OSVMP2_MIXED) TRY(check_err_flag(c, "mixed fragment solve"));
  double f_solve = 0.0;
  for (int f = 0; f < nf; f++)
    f_solve += (prec == OSVMP2_MIXED) ? fragment_mixed_flops(c, c->frags[f], c->frag_out[f].iters)
                                      : c->frag_out[f].iters * fragment_iter_flops(c, c->frags[f]);
  c->flops[OSVMP2_PH_SOLVE] += f_solve;
  c->flops[OSVMP2_PH_K_FRAGSOLVE] += f_solve;
  int unconv = 0, maxit = 0;
  int64_t worst = -1;
  double maxu = 0.0;
  for (int f = 0; f < nf; f++) {
    const FragOut& o = c->frag_out[f];
    maxit = std::max(maxit, o.iters);
    maxu = std::max(maxu, o.umax);
    if (o.status) {
      unconv++;
      if (worst < 0) worst = f;
    }
  }
  if (stats) {
    stats->n_single = ns;
    stats->n_pair = npair;
    stats->n_triple = ntri;
    stats->n_pair_blocks = (int64_t)c->K_h.size();
    stats->max_iter_used = maxit;
    stats->n_unconverged = unconv;
    stats->worst_fragment = worst;
    stats->max_update = maxu;
    stats->flops = f_solve;
    stats->n_weak = 0;
  }
  if (unconv)
    return fail(c, OSVMP2_E_NOCONV, "%d fragment(s) did not converge; first is fragment %lld", unconv,
                (long long)worst);
  return OSVMP2_OK;
}

int osvmp2_mbe3_energy(osvmp2_ctx* c, double r2, double r3, osvmp2_prec prec, double* e_out,
                       osvmp2_mbe_stats* stats) {
  TRY(distance_fragments(c, r2, r3, e_out));
  return mbe3_core(c, prec, e_out, stats, nullptr, nullptr);
}

int osvmp2_pair_screening(osvmp2_ctx* c, const osvmp2_screen* sc, double* s2b_out, int32_t* class_out,
                          int64_t* counts) {
  if (!c) return OSVMP2_E_ARG;
  c->err.clear();
  if (!c->have_osv) return fail(c, OSVMP2_E_STATE, "osvmp2_build_osv has not been called");
  if (!screen_valid(sc)) return fail(c, OSVMP2_E_ARG, "invalid screening thresholds");
  CK(cudaSetDevice(c->device));
  const int n = c->sys.n_occ;
  std::vector<double> s2b;
  TRY(compute_s2b(c, s2b));
  int64_t cnt[3] = {0, 0, 0};
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) {
      const double v = s2b[(size_t)i * n + j];
      const int cl = (i == j || v >= sc->s2b_close) ? 2 : (v >= sc->s2b_distant ? 1 : 0);
      if (class_out) class_out[(size_t)i * n + j] = cl;
      if (i < j) cnt[2 - cl]++;
    }
  if (s2b_out) std::copy(s2b.begin(), s2b.end(), s2b_out);
  if (counts) std::copy(cnt, cnt + 3, counts);
  return OSVMP2_OK;
}

int osvmp2_mbe3_energy_screened(osvmp2_ctx* c, const osvmp2_screen* sc, osvmp2_prec prec, double* e_out,
                                double* e_weak_out, osvmp2_mbe_stats* stats) {
  if (!c) return OSVMP2_E_ARG;
  c->err.clear();
  if (!c->have_osv) return fail(c, OSVMP2_E_STATE, "osvmp2_build_osv has not been called");
  if (!e_out) return fail(c, OSVMP2_E_ARG, "e_out is required");
  if (!screen_valid(sc)) return fail(c, OSVMP2_E_ARG, "invalid screening thresholds");
  if (prec != OSVMP2_FP64 && prec != OSVMP2_MIXED) return fail(c, OSVMP2_E_ARG, "unknown precision %d", (int)prec);
  CK(cudaSetDevice(c->device));
  const int n = c->sys.n_occ, nx = c->sys.n_aux;
  const bool mixed = prec == OSVMP2_MIXED;
  std::vector<double> s2b;
  TRY(compute_s2b(c, s2b));
  std::vector<std::pair<int, int>> weak;
  screened_fragments(s2b.data(), n, *sc, c->frags, weak);
  c->weak.clear();
  c->weak_e.clear();
  Tmp tstore;
  std::vector<long long> toff;
  double e_cl = 0.0;
  TRY(mbe3_core(c, prec, &e_cl, stats, weak.empty() ? nullptr : &tstore, &toff));
  double e_weak = 0.0;
  if (!weak.empty()) {
    ph_begin(c, OSVMP2_PH_WEAK);
    std::vector<int> need(n, 0);
    for (auto& w : weak) need[w.first] = need[w.second] = 1;
    // T_(ii,ii) of Eq. (tmbediag): the weighted (ii) amplitudes of the clusters containing i
    std::vector<std::vector<GradContrib>> con(n);
    for (size_t f = 0; f < c->frags.size(); f++) {
      const Frag& fr = c->frags[f];
      int orbs[3], nc = 0;
      for (int u = 0; u < 3; u++)
        if (fr.orbs[u] >= 0) orbs[nc++] = fr.orbs[u];
      long long off = toff[f];
      for (int a = 0; a < nc; a++)
        for (int b = a; b < nc; b++) {
          const long long m = pair_dim_h(c, orbs[a], orbs[b]);
          if (a == b && need[orbs[a]] && fr.weight != 0)
            con[orbs[a]].push_back(GradContrib{(const double*)tstore.p + off, fr.weight});
          off += m * m;
        }
    }
    std::vector<DiagJob> dj;
    std::vector<GradContrib> cflat;
    std::vector<size_t> doff(n, 0);
    size_t tsz = 0;
    int max_n = 1;
    for (int i = 0; i < n; i++) {
      if (!need[i]) continue;
      const int pid = c->pair_id[(size_t)i * n + i];
      if (pid < 0) return fail(c, OSVMP2_E_STATE, "diagonal pair (%d,%d) not built", i, i);
      DiagJob d{i, pid, (int)cflat.size(), 0, nullptr};
      for (auto& x : con[i]) cflat.push_back(x);
      d.c1 = (int)cflat.size();
      doff[i] = tsz;
      tsz += (size_t)c->n_osv[i] * c->n_osv[i];
      max_n = std::max(max_n, c->n_osv[i]);
      dj.push_back(d);
    }
    Tmp tdiag, d_dj, d_cf, dscr;
    TRY(tmp_alloc(c, tdiag, tsz * sizeof(double)));
    for (auto& d : dj) d.T = (double*)tdiag.p + doff[d.i];
    TRY(tmp_alloc(c, d_dj, dj.size() * sizeof(DiagJob)));
    TRY(tmp_alloc(c, d_cf, std::max<size_t>(1, cflat.size()) * sizeof(GradContrib)));
    const int n_cta_d = std::max(1, std::min((int)dj.size(), 2 * c->num_sms));
    TRY(tmp_alloc(c, dscr, (size_t)n_cta_d * 2 * max_n * max_n * sizeof(double)));
    CK(cudaMemcpyAsync(d_dj.p, dj.data(), dj.size() * sizeof(DiagJob), cudaMemcpyHostToDevice, c->st));
    if (!cflat.empty())
      CK(cudaMemcpyAsync(d_cf.p, cflat.data(), cflat.size() * sizeof(GradContrib), cudaMemcpyHostToDevice, c->st));
    launch_diag_amp(tables(c), (const DiagJob*)d_dj.p, (int)dj.size(), (const GradContrib*)d_cf.p, mixed ? 1 : 0,
                    (double*)dscr.p, max_n, n_cta_d, c->st);
    CK(cudaGetLastError());
    // S_(i,j) of the weak pairs
    TRY(ensure_sf_blocks(c, weak));
    // diagonal projections B~_i^(i) (Eq. osv_imua): the FP64 form's own; the mixed form
    // forms them for the weak-pair orbitals in double-float.  Eigenbases of F_(i,i):
    // the preconditioners of the diagonal pairs (exact in the FP64 form, the mixed
    // basis otherwise; k_weak then iterates on the raw-basis residual).
    std::vector<const double*> bii(n, nullptr), xi(n, nullptr), ei(n, nullptr);
    Tmp projm, d_pj;
    for (int i = 0; i < n; i++) {
      if (!need[i]) continue;
      const int pid = c->pair_id[(size_t)i * n + i];
      if (c->r_h[pid] != c->n_osv[i])
        return fail(c, OSVMP2_E_NUMERIC, "diagonal pair (%d,%d): preconditioner rank %d below %d", i, i, c->r_h[pid],
                    c->n_osv[i]);
      xi[i] = c->X_h[pid];
      ei[i] = c->et_h[pid];
      if (!mixed) {
        const int id = c->bt_id[(size_t)i * n + i];
        if (id < 0) return fail(c, OSVMP2_E_STATE, "projection of orbital %d not built", i);
        bii[i] = c->bt_h[id];
      }
    }
    if (mixed) {
      std::vector<ProjJob> pj;
      size_t psz = 0;
      for (int i = 0; i < n; i++)
        if (need[i]) psz += (size_t)nx * c->n_osv[i];
      TRY(tmp_alloc(c, projm, psz * sizeof(double)));
      size_t po = 0;
      double fl = 0.0;
      for (int i = 0; i < n; i++) {
        if (!need[i]) continue;
        double* out = (double*)projm.p + po;
        pj.push_back(ProjJob{i, i, out});
        bii[i] = out;
        po += (size_t)nx * c->n_osv[i];
        fl += 2.0 * nx * (double)c->sys.n_vir * c->n_osv[i];
      }
      TRY(tmp_alloc(c, d_pj, pj.size() * sizeof(ProjJob)));
      CK(cudaMemcpyAsync(d_pj.p, pj.data(), pj.size() * sizeof(ProjJob), cudaMemcpyHostToDevice, c->st));
      launch_project_df(bsrc(c), tables(c), (const ProjJob*)d_pj.p, (int)pj.size(), c->st);
      CK(cudaGetLastError());
      c->flops[OSVMP2_PH_WEAK] += fl;
    }
    std::vector<WeakJob> wj;
    double fl = 0.0;
    for (auto& w : weak) {
      const int i = w.first, j = w.second;
      const int id = c->sf_id[(size_t)i * n + j];
      WeakJob jb{i, j, bii[i], bii[j], c->S_h[id], (const double*)tdiag.p + doff[i],
                 (const double*)tdiag.p + doff[j], xi[i], xi[j], ei[i], ei[j], c->n_osv[i], c->n_osv[j],
                 c->F_h[c->sf_id[(size_t)i * n + i]], c->F_h[c->sf_id[(size_t)j * n + j]]};
      wj.push_back(jb);
      const double ni = c->n_osv[i], nj = c->n_osv[j];
      fl += 2.0 * nx * ni * nj + 2.0 * (ni * ni * nj + ni * nj * nj) * 3.0;
    }
    Tmp d_wj, wscr, we;
    const int n_cta_w = std::max(1, std::min((int)wj.size(), 2 * c->num_sms));
    TRY(tmp_alloc(c, d_wj, wj.size() * sizeof(WeakJob)));
    TRY(tmp_alloc(c, wscr, (size_t)n_cta_w * 6 * max_n * max_n * sizeof(double)));
    TRY(tmp_alloc(c, we, wj.size() * sizeof(double)));
    CK(cudaMemcpyAsync(d_wj.p, wj.data(), wj.size() * sizeof(WeakJob), cudaMemcpyHostToDevice, c->st));
    launch_weak(tables(c), nx, (const WeakJob*)d_wj.p, (int)wj.size(), (double*)wscr.p, max_n, n_cta_w,
                (double*)we.p, mixed ? 1 : 0, c->st);
    CK(cudaGetLastError());
    ph_end(c, OSVMP2_PH_WEAK, fl);
    c->weak_e.resize(wj.size());
    CK(cudaMemcpyAsync(c->weak_e.data(), we.p, wj.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    ph_collect(c);
    c->weak = weak;
    for (double v : c->weak_e) {
      if (!std::isfinite(v)) return fail(c, OSVMP2_E_NUMERIC, "non-finite weak-pair energy");
      e_weak += v;
    }
  }
  if (stats) stats->n_weak = (int64_t)weak.size();
  *e_out = e_cl + e_weak;
  if (e_weak_out) *e_weak_out = e_weak;
  return OSVMP2_OK;
}

int osvmp2_weak_results(osvmp2_ctx* c, int64_t* n_out, int32_t* pairs, double* energies) {
  if (!c || !n_out) return OSVMP2_E_ARG;
  *n_out = (int64_t)c->weak.size();
  for (size_t q = 0; q < c->weak.size(); q++) {
    if (pairs) {
      pairs[2 * q] = c->weak[q].first;
      pairs[2 * q + 1] = c->weak[q].second;
    }
    if (energies) energies[q] = q < c->weak_e.size() ? c->weak_e[q] : 0.0;
  }
  return OSVMP2_OK;
}

int osvmp2_localize_pm(osvmp2_ctx* c, const double* C, int32_t n_ao, int32_t n_occ, const int32_t* atom_ao,
                       int32_t n_atom, double l_loc, int32_t max_sweeps, double* U, double* L_out, int32_t* sweeps_out) {
  if (!c) return OSVMP2_E_ARG;
  c->err.clear();
  if (!C || !U || !atom_ao || n_occ < 1 || n_atom < 1 || n_ao < n_occ || max_sweeps < 1 || !(l_loc >= 0.0))
    return fail(c, OSVMP2_E_ARG, "localize: bad arguments");
  if (atom_ao[0] != 0 || atom_ao[n_atom] != n_ao)
    return fail(c, OSVMP2_E_ARG, "localize: atom_ao must run from 0 to n_ao");
  for (int a = 0; a < n_atom; a++)
    if (atom_ao[a + 1] < atom_ao[a]) return fail(c, OSVMP2_E_ARG, "localize: atom_ao must be ascending");
  if ((double)n_occ * n_occ * n_atom > 4e9) return fail(c, OSVMP2_E_ARG, "localize: charge tensor too large");
  CK(cudaSetDevice(c->device));
  Tmp P, ao, out, stat, part, bar;
  TRY(tmp_alloc(c, P, (size_t)n_occ * n_occ * n_atom * sizeof(double)));
  TRY(tmp_alloc(c, ao, (size_t)(n_atom + 1) * sizeof(int)));
  TRY(tmp_alloc(c, out, 2 * sizeof(double)));
  TRY(tmp_alloc(c, stat, 2 * sizeof(int)));
  TRY(tmp_alloc(c, part, 4 * (size_t)std::max(1, std::min(n_atom, c->num_sms)) * sizeof(double)));
  TRY(tmp_alloc(c, bar, 2 * sizeof(unsigned)));
  CK(cudaMemcpyAsync(ao.p, atom_ao, (size_t)(n_atom + 1) * sizeof(int), cudaMemcpyHostToDevice, c->st));
  CK(cudaMemsetAsync(c->err_d, 0, sizeof(int), c->st));
  ph_begin(c, OSVMP2_PH_LOCALIZE);
  // whole-GPU form (atoms over a cooperative grid) when its CTAs can all be resident,
  // else the one-CTA form; both follow the same sequence of rotations
  if (!launch_pm_localize_grid(C, n_occ, (const int*)ao.p, n_atom, l_loc, max_sweeps, (double*)P.p, U,
                               (double*)out.p, (int*)stat.p, (double*)part.p, (unsigned*)bar.p, c->err_d, c->num_sms,
                               c->st))
    launch_pm_localize(C, n_ao, n_occ, (const int*)ao.p, n_atom, l_loc, max_sweeps, (double*)P.p, U, (double*)out.p,
                       (int*)stat.p, c->num_sms, c->st);
  ph_end(c, OSVMP2_PH_LOCALIZE, 0.0);
  CK(cudaGetLastError());
  TRY(check_err_flag(c, "localize"));
  double ho[2];
  int hs[2];
  CK(cudaMemcpyAsync(ho, out.p, sizeof ho, cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(hs, stat.p, sizeof hs, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  ph_collect(c);
  if (L_out) *L_out = ho[0];
  if (sweeps_out) *sweeps_out = hs[0];
  if (!std::isfinite(ho[0])) return fail(c, OSVMP2_E_NUMERIC, "localize: non-finite functional");
  if (!hs[1]) return fail(c, OSVMP2_E_NOCONV, "localize: dL = %.3e after %d sweeps", ho[1], hs[0]);
  return OSVMP2_OK;
}

int osvmp2_profile(osvmp2_ctx* c, double* ms, double* flops, double* bytes, int64_t* calls, int reset) {
  if (!c) return OSVMP2_E_ARG;
  CK(cudaStreamSynchronize(c->st));
  ph_collect(c);
  for (int ph = 0; ph < OSVMP2_NPHASE; ph++) {
    if (ms) ms[ph] = c->ms[ph];
    if (flops) flops[ph] = c->flops[ph];
    if (bytes) bytes[ph] = c->bytes[ph];
    if (calls) calls[ph] = c->calls[ph];
    if (reset) { c->ms[ph] = 0.0; c->flops[ph] = 0.0; c->bytes[ph] = 0.0; c->calls[ph] = 0; }
  }
  return OSVMP2_OK;
}

int osvmp2_fragment_results(osvmp2_ctx* c, int64_t* n_out, int32_t* orbs, int32_t* weights, double* energies) {
  if (!c || !n_out) return OSVMP2_E_ARG;
  const size_t nf = c->frags.size();
  *n_out = (int64_t)nf;
  for (size_t f = 0; f < nf; f++) {
    if (orbs)
      for (int u = 0; u < 3; u++) orbs[3 * f + u] = c->frags[f].orbs[u];
    if (weights) weights[f] = c->frags[f].weight;
    if (energies) energies[f] = (f < c->frag_out.size()) ? c->frag_out[f].energy : 0.0;
  }
  return OSVMP2_OK;
}

// OSV response of the relaxed gradient (FP64 form), added to the frozen outputs:
// dE/dQ_x from the exchange part per pair and the rest per fragment, then per batch
// of orbitals T_xx again, all its eigenpairs, the response Z_x and its chain rule.
static int relax_osv(osvmp2_ctx* c, const std::vector<std::pair<int, int>>& plist,
                     const std::vector<GradPairJob>& pjobs, const double* tstore, const std::vector<long long>& toff,
                     int max_m, double* dE_dB, double* dE_df, double* dE_de, double* gap_out) {
  const int n = c->sys.n_occ, nv = c->sys.n_vir, nx = c->sys.n_aux;
  const int np = (int)plist.size(), nf = (int)c->frags.size();
  const Tables t = tables(c);
  const BSrc bs = bsrc(c);
  auto bt = [&](int a, int x) -> const double* {
    const int id = c->bt_id[(size_t)a * n + x];
    return id >= 0 ? (const double*)c->bt_h[id] : nullptr;
  };
  double fl = 0.0;
  ph_begin(c, OSVMP2_PH_RELAX);
  // exchange part per stored pair
  std::vector<size_t> koff(np + 1, 0);
  for (int q = 0; q < np; q++) koff[q + 1] = koff[q] + (size_t)nv * pair_dim_h(c, plist[q].first, plist[q].second);
  Tmp dk, kscr, d_kj;
  TRY(tmp_alloc(c, dk, std::max<size_t>(1, koff[np]) * sizeof(double)));
  std::vector<RelaxKJob> kj(np);
  for (int q = 0; q < np; q++) {
    const int i = plist[q].first, j = plist[q].second;
    RelaxKJob& k = kj[q];
    k.i = i;
    k.j = j;
    k.W = pjobs[q].W;
    k.bt_ii = bt(i, i);
    k.bt_ij = (i != j) ? bt(i, j) : nullptr;
    k.bt_ji = (i != j) ? bt(j, i) : nullptr;
    k.bt_jj = (i != j) ? bt(j, j) : nullptr;
    if (!k.bt_ii || (i != j && (!k.bt_ij || !k.bt_ji || !k.bt_jj)))
      return fail(c, OSVMP2_E_STATE, "relaxed gradient: the projections of pair (%d, %d) are missing", i, j);
    k.out = (double*)dk.p + koff[q];
    const double m = pair_dim_h(c, i, j);
    fl += 4.0 * nx * m * m + 4.0 * nv * (double)nx * m;
  }
  const int n_cta_k = std::max(1, std::min(np, 2 * c->num_sms));
  TRY(tmp_alloc(c, kscr, (size_t)n_cta_k * 2 * nx * std::max(max_m, 1) * sizeof(double)));
  TRY(tmp_alloc(c, d_kj, std::max<size_t>(1, kj.size()) * sizeof(RelaxKJob)));
  if (np) CK(cudaMemcpyAsync(d_kj.p, kj.data(), kj.size() * sizeof(RelaxKJob), cudaMemcpyHostToDevice, c->st));
  launch_relax_kpart(t, bs, (const RelaxKJob*)d_kj.p, np, (double*)kscr.p, n_cta_k, max_m, c->st);
  CK(cudaGetLastError());
  // the rest per fragment, into one slot per (fragment, orbital)
  std::vector<std::vector<RelaxGTerm>> gt(n);
  size_t slot_total = 0;
  for (int f = 0; f < nf; f++)
    if (c->frags[f].weight != 0)
      for (int u = 0; u < 3; u++)
        if (c->frags[f].orbs[u] >= 0) slot_total += (size_t)nv * c->n_osv[c->frags[f].orbs[u]];
  Tmp slots, fscr, d_fj;
  TRY(tmp_alloc(c, slots, std::max<size_t>(1, slot_total) * sizeof(double)));
  std::vector<RelaxFragJob> fj;
  size_t so = 0;
  for (int f = 0; f < nf; f++) {
    const Frag& fr = c->frags[f];
    if (fr.weight == 0) continue;
    RelaxFragJob jb{};
    jb.no = 0;
    jb.c = (double)fr.weight;
    jb.T = tstore + toff[f];
    for (int u = 0; u < 3; u++)
      if (fr.orbs[u] >= 0) {
        const int x = fr.orbs[u];
        jb.orbs[jb.no] = x;
        jb.slot[jb.no] = (double*)slots.p + so;
        gt[x].push_back(RelaxGTerm{jb.slot[jb.no], c->n_osv[x], 0});
        so += (size_t)nv * c->n_osv[x];
        jb.no++;
      }
    double rows = 0.0;
    for (int a = 0; a < jb.no; a++) rows += c->n_osv[jb.orbs[a]];
    for (int a = 0; a < jb.no; a++)
      for (int b = a; b < jb.no; b++) {
        const double m = pair_dim_h(c, jb.orbs[a], jb.orbs[b]);
        fl += 2.0 * (8.0 * m * m * m + (double)nv * m * (m + rows));   // self terms, Q_x products
        for (int k = 0; k < jb.no; k++)                                  // couplings (x, y) = (k, b), (a, k)
          for (int s2 = 0; s2 < 2; s2++) {
            const int x = s2 ? a : k, y = s2 ? k : b;
            const double mq = pair_dim_h(c, jb.orbs[std::min(x, y)], jb.orbs[std::max(x, y)]);
            fl += 4.0 * (mq * mq * m + mq * m * m);
          }
      }
    fj.push_back(jb);
  }
  // one CTA per fragment in flight, two per SM (112 registers x 256 threads each), their scratch
  // within a quarter of the free memory
  const size_t scr_per = 8 * (size_t)std::max(max_m, 1) * std::max(max_m, 1) + (size_t)nv * std::max(max_m, 1);
  int n_cta_f = std::max(1, std::min((int)fj.size(), 2 * c->num_sms));
  {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) == cudaSuccess)
      n_cta_f = (int)std::max<size_t>(1, std::min<size_t>((size_t)n_cta_f, fr / 4 / (scr_per * sizeof(double))));
    else
      cudaGetLastError();
  }
  TRY(tmp_alloc(c, fscr, (size_t)n_cta_f * scr_per * sizeof(double)));
  TRY(tmp_alloc(c, d_fj, std::max<size_t>(1, fj.size()) * sizeof(RelaxFragJob)));
  if (!fj.empty())
    CK(cudaMemcpyAsync(d_fj.p, fj.data(), fj.size() * sizeof(RelaxFragJob), cudaMemcpyHostToDevice, c->st));
  launch_relax_frag(t, c->sys.e_vir, (const RelaxFragJob*)d_fj.p, (int)fj.size(), (double*)fscr.p, scr_per, n_cta_f,
                    max_m, c->st);
  CK(cudaGetLastError());
  // G_x: fragment slots (fragment order), then the exchange parts (pair order)
  for (int q = 0; q < np; q++) {
    const int i = plist[q].first, j = plist[q].second, m = pair_dim_h(c, i, j);
    gt[i].push_back(RelaxGTerm{(const double*)dk.p + koff[q], m, 0});
    if (i != j) gt[j].push_back(RelaxGTerm{(const double*)dk.p + koff[q], m, c->n_osv[i]});
  }
  std::vector<RelaxGJob> gj(n);
  std::vector<RelaxGTerm> gflat;
  std::vector<size_t> goff(n + 1, 0);
  for (int x = 0; x < n; x++) goff[x + 1] = goff[x] + (size_t)nv * c->n_osv[x];
  Tmp gmem, d_gj, d_gt;
  TRY(tmp_alloc(c, gmem, goff[n] * sizeof(double)));
  for (int x = 0; x < n; x++) {
    gj[x] = RelaxGJob{x, (int)gflat.size(), 0, (double*)gmem.p + goff[x]};
    for (auto& tm : gt[x]) gflat.push_back(tm);
    gj[x].t1 = (int)gflat.size();
  }
  TRY(tmp_alloc(c, d_gj, gj.size() * sizeof(RelaxGJob)));
  TRY(tmp_alloc(c, d_gt, std::max<size_t>(1, gflat.size()) * sizeof(RelaxGTerm)));
  CK(cudaMemcpyAsync(d_gj.p, gj.data(), gj.size() * sizeof(RelaxGJob), cudaMemcpyHostToDevice, c->st));
  if (!gflat.empty())
    CK(cudaMemcpyAsync(d_gt.p, gflat.data(), gflat.size() * sizeof(RelaxGTerm), cudaMemcpyHostToDevice, c->st));
  launch_relax_gather(nv, c->n_osv_d, (const RelaxGJob*)d_gj.p, n, (const RelaxGTerm*)d_gt.p, c->st);
  CK(cudaGetLastError());
  // per batch of orbitals: T_xx, all its eigenpairs, the response and its chain rule
  const size_t V2 = (size_t)nv * nv;
  const size_t per = (4 * V2 + 2 * (size_t)nv * nv + 3 * (size_t)nv + 1 + eig_osv_scratch_doubles(nv, nv)) * sizeof(double);
  int nb = (int)std::max<size_t>(1, std::min<size_t>((size_t)n, ((size_t)8 << 30) / per));
  nb = std::min(nb, 4 * c->num_sms);
  Tmp Tm, Tc, Vm, wm, km, em, Zm, Ym, Xm, dem, dfm, d_rj;
  TRY(tmp_alloc(c, Tm, (size_t)nb * V2 * sizeof(double)));
  TRY(tmp_alloc(c, Tc, (size_t)nb * V2 * sizeof(double)));
  TRY(tmp_alloc(c, Vm, (size_t)nb * V2 * sizeof(double)));
  TRY(tmp_alloc(c, wm, (size_t)nb * nv * sizeof(double)));
  TRY(tmp_alloc(c, km, (size_t)nb * sizeof(int)));
  TRY(tmp_alloc(c, em, (size_t)nb * eig_osv_scratch_doubles(nv, nv) * sizeof(double)));
  TRY(tmp_alloc(c, Zm, (size_t)nb * V2 * sizeof(double)));
  TRY(tmp_alloc(c, Ym, (size_t)nb * V2 * sizeof(double)));
  TRY(tmp_alloc(c, Xm, (size_t)nb * V2 * sizeof(double)));
  TRY(tmp_alloc(c, dem, (size_t)nb * nv * sizeof(double)));
  TRY(tmp_alloc(c, dfm, (size_t)nb * sizeof(double)));
  TRY(tmp_alloc(c, d_rj, (size_t)nb * sizeof(RelaxRJob)));
  double gap = INFINITY;
  std::vector<double> wh((size_t)nb * nv);
  std::vector<RelaxRJob> rj(nb);
  for (int i0 = 0; i0 < n; i0 += nb) {
    const int b = std::min(nb, n - i0);
    launch_tii(bs, c->sys.e_vir, c->sys.f_occ, n, i0, b, (double*)Tm.p, c->st);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(Tc.p, Tm.p, (size_t)b * V2 * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    launch_eig_osv((double*)Tm.p, b, nv, 0.0, nv, (double*)Vm.p, (double*)wm.p, (int*)km.p, (double*)em.p, c->err_d,
                   false, c->st);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(wh.data(), wm.p, (size_t)b * nv * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    TRY(check_err_flag(c, "relaxed gradient: eigen-decomposition of T_ii"));
    for (int u = 0; u < b; u++) {
      const int x = i0 + u, nk = c->n_osv[x];
      const double* w = wh.data() + (size_t)u * nv;
      int cnt = 0;
      while (cnt < nv && (c->l_osv <= 0.0 || w[cnt] >= c->l_osv)) cnt++;
      if (cnt != nk)
        return fail(c, OSVMP2_E_NUMERIC,
                    "relaxed gradient: orbital %d has %d eigenvalues of T_ii above l_osv in FP64, %d OSVs built", x,
                    cnt, nk);
      if (nk < nv) {
        const double g = w[nk - 1] - w[nk];
        if (!(g > 0.0))
          return fail(c, OSVMP2_E_NUMERIC, "relaxed gradient: no eigenvalue gap at the OSV cut of orbital %d", x);
        gap = std::min(gap, g);
      }
      rj[u] = RelaxRJob{x, (const double*)Vm.p + u * V2, (const double*)wm.p + (size_t)u * nv,
                        (const double*)Tc.p + u * V2, (const double*)gmem.p + goff[x], (double*)Zm.p + u * V2,
                        (double*)Ym.p + u * V2, (double*)Xm.p + u * V2, (double*)dem.p + (size_t)u * nv,
                        (double*)dfm.p + u};
      const double nd = nv - nk;
      fl += (double)nv * nv * nx + 9.0 * (double)nv * nv * nv + 4.0 * nd * nk * nv + 4.0 * (double)nv * nv * nk +
            2.0 * (double)nv * nv * nx;
    }
    CK(cudaMemcpyAsync(d_rj.p, rj.data(), (size_t)b * sizeof(RelaxRJob), cudaMemcpyHostToDevice, c->st));
    launch_relax_resp(t, bs, c->sys.e_vir, (const RelaxRJob*)d_rj.p, b, dE_dB, dE_de, dE_df, c->st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->st));   // rj is rewritten by the next batch
  }
  ph_end(c, OSVMP2_PH_RELAX, fl);
  if (gap_out) *gap_out = gap;
  return OSVMP2_OK;
}

static int energy_grad_impl(osvmp2_ctx* c, double r2, double r3, osvmp2_prec prec, double* e_out, double* dE_dB,
                            double* dE_df, double* dE_de, osvmp2_mbe_stats* stats, bool relaxed, double* gap_out) {
  if (!c) return OSVMP2_E_ARG;
  Tmp tstore;
  std::vector<long long> toff;
  TRY(distance_fragments(c, r2, r3, e_out));
  TRY(mbe3_core(c, prec, e_out, stats, &tstore, &toff));
  const int n = c->sys.n_occ, nv = c->sys.n_vir, nx = c->sys.n_aux;
  const int nf = (int)c->frags.size();
  // unique pairs of the fragment list, each with its (fragment-ordered) contributions
  std::vector<int> pidx((size_t)n * n, -1);
  std::vector<std::pair<int, int>> plist;
  std::vector<std::vector<GradContrib>> contr;
  int max_m = 0;
  for (int f = 0; f < nf; f++) {
    const Frag& fr = c->frags[f];
    int orbs[3], nc = 0;
    for (int u = 0; u < 3; u++)
      if (fr.orbs[u] >= 0) orbs[nc++] = fr.orbs[u];
    long long off = toff[f];
    for (int a = 0; a < nc; a++)
      for (int b = a; b < nc; b++) {
        const int i = orbs[a], j = orbs[b];
        const long long m = pair_dim_h(c, i, j);
        max_m = std::max(max_m, (int)m);
        int& q = pidx[(size_t)i * n + j];
        if (q < 0) {
          q = (int)plist.size();
          plist.push_back({i, j});
          contr.emplace_back();
        }
        if (fr.weight != 0) contr[q].push_back(GradContrib{(const double*)tstore.p + off, fr.weight});
        off += m * m;
      }
  }
  const int np = (int)plist.size();
  size_t wh = 0;
  for (auto& p : plist) wh += 2 * (size_t)pair_dim_h(c, p.first, p.second) * pair_dim_h(c, p.first, p.second);
  std::vector<GradPairJob> pjobs;
  std::vector<GradContrib> cflat;
  Tmp whm;
  TRY(tmp_alloc(c, whm, wh * sizeof(double)));
  {
    size_t o = 0;
    for (int q = 0; q < np; q++) {
      const size_t m2 = (size_t)pair_dim_h(c, plist[q].first, plist[q].second) *
                        pair_dim_h(c, plist[q].first, plist[q].second);
      GradPairJob jb{plist[q].first, plist[q].second, (int)cflat.size(), 0, (double*)whm.p + o,
                     (double*)whm.p + o + m2};
      for (auto& cb : contr[q]) cflat.push_back(cb);
      jb.c1 = (int)cflat.size();
      o += 2 * m2;
      pjobs.push_back(jb);
    }
  }
  const Tables t = tables(c);
  const int n_cta = std::max(1, std::min(np, 2 * c->num_sms));
  Tmp d_pj, d_cf, scr;
  TRY(tmp_alloc(c, d_pj, pjobs.size() * sizeof(GradPairJob)));
  TRY(tmp_alloc(c, d_cf, std::max<size_t>(1, cflat.size()) * sizeof(GradContrib)));
  const size_t scr_d = std::max((size_t)2 * max_m * max_m, (size_t)nv * max_m);
  TRY(tmp_alloc(c, scr, (size_t)n_cta * scr_d * sizeof(double)));
  CK(cudaMemcpyAsync(d_pj.p, pjobs.data(), pjobs.size() * sizeof(GradPairJob), cudaMemcpyHostToDevice, c->st));
  if (!cflat.empty())
    CK(cudaMemcpyAsync(d_cf.p, cflat.data(), cflat.size() * sizeof(GradContrib), cudaMemcpyHostToDevice, c->st));
  double fl = 0.0;
  for (int q = 0; q < np; q++) {
    const double m = pair_dim_h(c, plist[q].first, plist[q].second);
    fl += (double)contr[q].size() * (plist[q].first == plist[q].second ? 4.0 : 8.0) * m * m * m;
  }
  const bool mixed = prec == OSVMP2_MIXED;
  ph_begin(c, OSVMP2_PH_GRAD);
  if (mixed)
    launch_gradm_pair(t, (const GradPairJob*)d_pj.p, np, (const GradContrib*)d_cf.p, (double*)scr.p, n_cta, max_m,
                      c->st);
  else
    launch_grad_pair(t, (const GradPairJob*)d_pj.p, np, (const GradContrib*)d_cf.p, (double*)scr.p, n_cta, max_m,
                     c->st);
  CK(cudaGetLastError());
  Tmp dpair;
  if (dE_de) {
    TRY(tmp_alloc(c, dpair, (size_t)np * nv * sizeof(double)));
    if (mixed)
      launch_gradm_de(t, (const GradPairJob*)d_pj.p, np, (double*)scr.p, n_cta, max_m, (double*)dpair.p, dE_de, c->st);
    else
      launch_grad_de(t, (const GradPairJob*)d_pj.p, np, (double*)scr.p, n_cta, max_m, (double*)dpair.p, dE_de, c->st);
    CK(cudaGetLastError());
  }
  Tmp gfrag, d_fptr, d_flist, d_orbs, d_w, d_toff;
  if (dE_df) {
    std::vector<int> fptr(n + 1, 0), flist, orbs_h(3 * (size_t)nf), w_h(nf);
    std::vector<std::vector<int>> per(n);
    for (int f = 0; f < nf; f++) {
      for (int u = 0; u < 3; u++) {
        orbs_h[3 * f + u] = c->frags[f].orbs[u];
        if (c->frags[f].orbs[u] >= 0) per[c->frags[f].orbs[u]].push_back(f);
      }
      w_h[f] = c->frags[f].weight;
    }
    for (int k = 0; k < n; k++) {
      fptr[k + 1] = fptr[k] + (int)per[k].size();
      for (int f : per[k]) flist.push_back(f);
    }
    TRY(tmp_alloc(c, gfrag, (size_t)nf * 9 * sizeof(double)));
    TRY(tmp_alloc(c, d_fptr, fptr.size() * sizeof(int)));
    TRY(tmp_alloc(c, d_flist, std::max<size_t>(1, flist.size()) * sizeof(int)));
    TRY(tmp_alloc(c, d_orbs, orbs_h.size() * sizeof(int)));
    TRY(tmp_alloc(c, d_w, w_h.size() * sizeof(int)));
    TRY(tmp_alloc(c, d_toff, toff.size() * sizeof(long long)));
    CK(cudaMemcpyAsync(d_fptr.p, fptr.data(), fptr.size() * sizeof(int), cudaMemcpyHostToDevice, c->st));
    if (!flist.empty())
      CK(cudaMemcpyAsync(d_flist.p, flist.data(), flist.size() * sizeof(int), cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(d_orbs.p, orbs_h.data(), orbs_h.size() * sizeof(int), cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(d_w.p, w_h.data(), w_h.size() * sizeof(int), cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(d_toff.p, toff.data(), toff.size() * sizeof(long long), cudaMemcpyHostToDevice, c->st));
    const int n_cta_f = std::max(1, std::min(nf, 2 * c->num_sms));
    Tmp scr_f;
    TRY(tmp_alloc(c, scr_f, (size_t)n_cta_f * 2 * max_m * max_m * sizeof(double)));
    if (mixed)
      launch_gradm_df(t, (const int*)d_orbs.p, (const int*)d_w.p, (const double*)tstore.p,
                      (const long long*)d_toff.p, nf, max_m, (double*)scr_f.p, n_cta_f, (double*)gfrag.p,
                      (const int*)d_fptr.p, (const int*)d_flist.p, dE_df, c->st);
    else
      launch_grad_df(t, (const int*)d_orbs.p, (const int*)d_w.p, (const double*)tstore.p,
                     (const long long*)d_toff.p, nf, max_m, (double*)scr_f.p, n_cta_f, (double*)gfrag.p,
                     (const int*)d_fptr.p, (const int*)d_flist.p, dE_df, c->st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->st));
  }
  Tmp ymem, d_yj, d_yt, d_bj, d_bt;
  if (dE_dB && mixed) {
    // Z = op(W~) G_partner per (pair, side); dB_o = 4 sum U_p Z over the pairs of o
    std::vector<GradZJob> zj;
    std::vector<std::vector<GradMBTerm>> per(n);
    size_t zsz = 0;
    int max_r = 0;
    for (int q = 0; q < np; q++) {
      const int i = plist[q].first, j = plist[q].second, pid = c->pair_id[(size_t)i * n + j];
      const int r = c->r_h[pid];
      max_r = std::max(max_r, r);
      zsz += (size_t)r * nx * (i == j ? 1 : 2);
    }
    TRY(tmp_alloc(c, ymem, std::max<size_t>(1, zsz) * sizeof(float)));
    size_t zo = 0;
    for (int q = 0; q < np; q++) {
      const int i = plist[q].first, j = plist[q].second, pid = c->pair_id[(size_t)i * n + j];
      const int r = c->r_h[pid];
      float* Zi = (float*)ymem.p + zo;
      zo += (size_t)r * nx;
      zj.push_back(GradZJob{r, 0, pjobs[q].W, c->Gj_h[pid], Zi});      // for dB_i: W~ G_j
      per[i].push_back(GradMBTerm{r, c->U_h[pid], Zi});
      fl += 2.0 * r * (double)r * nx + 2.0 * nv * (double)r * nx;
      if (i != j) {
        float* Zj = (float*)ymem.p + zo;
        zo += (size_t)r * nx;
        zj.push_back(GradZJob{r, 1, pjobs[q].W, c->Gi_h[pid], Zj});    // for dB_j: W~^T G_i
        per[j].push_back(GradMBTerm{r, c->U_h[pid], Zj});
        fl += 2.0 * r * (double)r * nx + 2.0 * nv * (double)r * nx;
      }
    }
    std::vector<GradBJob> bj;
    std::vector<GradMBTerm> bt;
    for (int o = 0; o < n; o++) {
      if (per[o].empty()) continue;
      GradBJob b{o, (int)bt.size(), 0};
      for (auto& tm : per[o]) bt.push_back(tm);
      b.t1 = (int)bt.size();
      bj.push_back(b);
    }
    TRY(tmp_alloc(c, d_yj, zj.size() * sizeof(GradZJob)));
    TRY(tmp_alloc(c, d_bj, bj.size() * sizeof(GradBJob)));
    TRY(tmp_alloc(c, d_bt, bt.size() * sizeof(GradMBTerm)));
    CK(cudaMemcpyAsync(d_yj.p, zj.data(), zj.size() * sizeof(GradZJob), cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(d_bj.p, bj.data(), bj.size() * sizeof(GradBJob), cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(d_bt.p, bt.data(), bt.size() * sizeof(GradMBTerm), cudaMemcpyHostToDevice, c->st));
    CK(cudaMemsetAsync(dE_dB, 0, (size_t)n * nv * nx * sizeof(double), c->st));
    launch_gradm_Z(nx, (const GradZJob*)d_yj.p, (int)zj.size(), max_r, c->st);
    CK(cudaGetLastError());
    launch_gradm_dB(nv, nx, (const GradBJob*)d_bj.p, (int)bj.size(), (const GradMBTerm*)d_bt.p, dE_dB, c->st);
    CK(cudaGetLastError());
  }
  if (dE_dB && !mixed) {
    // combos (o, x): x = o and every partner of o in the pair list
    std::vector<std::vector<int>> partners(n);
    for (auto& p : plist)
      if (p.first != p.second) {
        partners[p.first].push_back(p.second);
        partners[p.second].push_back(p.first);
      }
    auto bt = [&](int a, int x) { return (const double*)c->bt_h[c->bt_id[(size_t)a * n + x]]; };
    auto Wp = [&](int i, int j) { return (const double*)pjobs[pidx[(size_t)i * n + j]].W; };
    std::vector<GradYJob> yj;
    std::vector<GradYTerm> yt;
    std::vector<GradBJob> bj;
    std::vector<GradBTerm> btm;
    size_t ysz = 0;
    int max_n = 0;
    std::vector<int> has(n, 0);
    for (auto& p : plist) { has[p.first] = 1; has[p.second] = 1; }
    for (int o = 0; o < n; o++) {
      if (!has[o]) continue;
      std::sort(partners[o].begin(), partners[o].end());
      std::vector<int> xs;
      xs.push_back(o);
      for (int x : partners[o]) xs.push_back(x);
      std::sort(xs.begin(), xs.end());
      GradBJob b{o, (int)btm.size(), 0};
      for (int x : xs) {
        GradYJob y{o, x, (int)yt.size(), 0, nullptr};
        if (x == o) {
          for (auto& p : plist) {
            if (p.first == o && p.second == o) yt.push_back(GradYTerm{o, o, 0, 0, Wp(o, o), bt(o, o), nullptr});
            else if (p.first == o) yt.push_back(GradYTerm{o, p.second, 0, 0, Wp(o, p.second), bt(p.second, o),
                                                          bt(p.second, p.second)});
            else if (p.second == o) yt.push_back(GradYTerm{p.first, o, 1, c->n_osv[p.first], Wp(p.first, o),
                                                           bt(p.first, p.first), bt(p.first, o)});
          }
        } else if (o < x) {
          yt.push_back(GradYTerm{o, x, 0, c->n_osv[o], Wp(o, x), bt(x, o), bt(x, x)});
        } else {
          yt.push_back(GradYTerm{x, o, 1, 0, Wp(x, o), bt(x, x), bt(x, o)});
        }
        y.t1 = (int)yt.size();
        y.Y = (double*)(uintptr_t)ysz;    // offset, fixed below
        ysz += (size_t)c->n_osv[x] * nx;
        max_n = std::max(max_n, c->n_osv[x]);
        btm.push_back(GradBTerm{x, (const double*)(uintptr_t)(ysz - (size_t)c->n_osv[x] * nx)});
        yj.push_back(y);
      }
      b.t1 = (int)btm.size();
      bj.push_back(b);
    }
    TRY(tmp_alloc(c, ymem, ysz * sizeof(double)));
    for (auto& y : yj) y.Y = (double*)ymem.p + (uintptr_t)y.Y;
    for (auto& b : btm) b.Y = (const double*)ymem.p + (uintptr_t)b.Y;
    TRY(tmp_alloc(c, d_yj, yj.size() * sizeof(GradYJob)));
    TRY(tmp_alloc(c, d_yt, yt.size() * sizeof(GradYTerm)));
    TRY(tmp_alloc(c, d_bj, bj.size() * sizeof(GradBJob)));
    TRY(tmp_alloc(c, d_bt, btm.size() * sizeof(GradBTerm)));
    CK(cudaMemcpyAsync(d_yj.p, yj.data(), yj.size() * sizeof(GradYJob), cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(d_yt.p, yt.data(), yt.size() * sizeof(GradYTerm), cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(d_bj.p, bj.data(), bj.size() * sizeof(GradBJob), cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(d_bt.p, btm.data(), btm.size() * sizeof(GradBTerm), cudaMemcpyHostToDevice, c->st));
    for (auto& tm : yt) {
      const double m = pair_dim_h(c, tm.pi, tm.pj);
      (void)m;
    }
    for (auto& y : yj)
      for (int q = y.t0; q < y.t1; q++) fl += 2.0 * c->n_osv[y.x] * (double)pair_dim_h(c, yt[q].pi, yt[q].pj) * nx;
    for (auto& b : btm) fl += 2.0 * nv * (double)c->n_osv[b.x] * nx;
    CK(cudaMemsetAsync(dE_dB, 0, (size_t)n * nv * nx * sizeof(double), c->st));
    launch_grad_Y(t, nx, (const GradYJob*)d_yj.p, (int)yj.size(), (const GradYTerm*)d_yt.p, max_n, c->st);
    CK(cudaGetLastError());
    launch_grad_dB(t, nx, (const GradBJob*)d_bj.p, (int)bj.size(), (const GradBTerm*)d_bt.p, dE_dB, c->st);
    CK(cudaGetLastError());
  }
  ph_end(c, OSVMP2_PH_GRAD, fl);
  if (relaxed) TRY(relax_osv(c, plist, pjobs, (const double*)tstore.p, toff, max_m, dE_dB, dE_df, dE_de, gap_out));
  CK(cudaStreamSynchronize(c->st));
  ph_collect(c);
  return check_err_flag(c, "gradient");
}

int osvmp2_energy_grad(osvmp2_ctx* c, double r2, double r3, osvmp2_prec prec, double* e_out, double* dE_dB,
                       double* dE_df, double* dE_de, osvmp2_mbe_stats* stats) {
  return energy_grad_impl(c, r2, r3, prec, e_out, dE_dB, dE_df, dE_de, stats, false, nullptr);
}

int osvmp2_energy_grad_relaxed(osvmp2_ctx* c, double r2, double r3, double* e_out, double* dE_dB, double* dE_df,
                               double* dE_de, osvmp2_mbe_stats* stats, double* min_gap_out) {
  if (!c) return OSVMP2_E_ARG;
  c->err.clear();
  if (!c->have_osv) return fail(c, OSVMP2_E_STATE, "no OSVs built");
  if (c->opts.osv_method != 0)
    return fail(c, OSVMP2_E_ARG, "the relaxed gradient needs exact OSVs (opts.osv_method 0)");
  return energy_grad_impl(c, r2, r3, OSVMP2_FP64, e_out, dE_dB, dE_df, dE_de, stats, true, min_gap_out);
}

}  // extern "C"
