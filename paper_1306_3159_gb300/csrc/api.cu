// C ABI of libibrd and the host-side drivers: multigrid V-cycle level loop,
// flexible GMRES, the reaction-limited and saddle-point operators, and the
// approximate Schur-complement preconditioner of Appendix A.
//
// Every arithmetic step runs in the CUDA kernels of grid_kernels.cu,
// blob_kernels.cu and krylov_kernels.cu; the host only sequences launches and
// reads back scalars (norms, residual estimates) to steer the iteration.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <tuple>
#include <type_traits>
#include <utility>
#include <vector>

#include "internal.h"
#include "schur_block.h"

namespace ibrd {

struct ArgError {
  ibrd_status code;
  std::string msg;
};

namespace {

// Device scalar slots.
enum Slot {
  S_BB = 0,   // ||b||^2
  S_SQ,       // ||w||^2 after orthogonalisation
  S_RES,      // residual estimate |g_{j+1}|
  S_MEAN,     // mean of a field (V-cycle projection)
  S_MEANX,    // mean of the V-cycle result
  S_GSUM,     // sum of g (saddle preconditioner)
  S_LBAR,     // lambda-bar of Appendix A
  S_CBAR,     // c-bar of Appendix A
  S_TMP,      // scratch
  S_TMP2,
  S_NORM,     // sqrt of S_SQ
  S_G32SUM,   // sum of the FP32-rounded source (saddle preconditioner)
  S_BMEAN1,   // mean of g~ (saddle preconditioner)
  S_XMEAN1,   // mean of c~* (saddle preconditioner)
  S_RFLAG,    // Gram-Schmidt second pass taken in this iteration (0/1)
  S_RCOUNT,   // second passes taken in this solve
  S_WAIT,     // nonzero bits: a bounded device wait gave up (written as an int)
  S_XMAX,     // largest |x| of a residual's iterate (its bits; fixed-point scale)
  S_PMEAN,    // mean of a block-preconditioned inner vector (IBRD_PRECOND_BLOCK)
  S_HHAT,     // Gram-Schmidt: the new basis vector's norm estimated before the pass
  S_HINV,     // its reciprocal
  S_RHO2,     // squared norm of the stored (scaled) new basis vector
  S_UB = 64,  // mean of S U_j for the inner iterations j = 0..m (64 slots)
  S_UX = 128, // mean of A~^-1 S U_j (64 slots)
  S_COUNT = 192
};

__global__ void k_bmean1(double* out, const double* sum32, const double* sum64, double inv_n) {
  if (threadIdx.x == 0) *out = (*sum32 - *sum64) * inv_n;
}

__global__ void k_scalar_affine(double* dst, const double* src, double a) {
  if (threadIdx.x == 0) *dst = a * (*src);
}

__global__ void k_check_rates(const double* __restrict__ k, int n, int* __restrict__ flag) {
  int bad = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    bad |= !(isfinite(k[i]) && k[i] >= 0.0);
  bad = __syncthreads_or(bad);
  if (bad && threadIdx.x == 0) atomicOr(flag, 1);
}

__global__ void k_set_gvec(double* gvec, int m, const double* beta) {
  const int i = threadIdx.x;
  if (i <= m) gvec[i] = (i == 0) ? *beta : 0.0;
}

template <typename T>
struct Hier {
  std::vector<T*> x, b;                       // levels >= 1 (index = level)
  std::vector<T*> y;                          // smoothing scratch, every level
  T* f0 = nullptr;                            // level-0 scratch fields (mixed path)
  T* f1 = nullptr;
  std::vector<std::pair<double, T*>> tables;  // coarsest Green's tables by shift
  std::vector<std::pair<double, T*>> hartley; // exact-level transform tables by shift (FP32)
};

struct Level {
  Dims d;
  double h;
};

}  // namespace

// Launch profiler of one handle: counts every launch and, when timing is on,
// brackets each launch with a pair of CUDA events on the launch stream.
struct Profiler {
  bool timing = false;
  unsigned mask = 0;      // classes timed when timing is on
  double min_bytes = 0.0; // only launches with at least this many algorithmic bytes are timed
  bool overflow = false;
  long long launches = 0;
  long long count[P_NCLASS] = {};
  double bytes[P_NCLASS] = {};
  double max_bytes[P_NCLASS] = {};
  double timed_bytes[P_NCLASS] = {};
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<std::pair<int, size_t>> pending;
  std::vector<double> pending_bytes;
  int open_cls = -1;
  size_t open_idx = 0;
};

// Launch shapes the autotuner chose for one handle, by element size, kernel
// and level grid.
struct Tuning {
  struct Entry {
    int elem, kind;
    Dims d;
    SweepShape s;
  };
  std::vector<Entry> e;
  // context of kernels with bounded device waits
  int* wait_err = nullptr;              // device flag set when a wait gives up
  unsigned wait_limit = kDefaultWaitLimit;  // tries per wait
  SweepShape* find(int elem, int kind, Dims d) {
    for (auto& x : e)
      if (x.elem == elem && x.kind == kind && x.d.nx == d.nx && x.d.ny == d.ny && x.d.nz == d.nz) return &x.s;
    return nullptr;
  }
};

namespace {
thread_local Profiler* t_prof = nullptr;
thread_local Tuning* t_tune = nullptr;
constexpr size_t kMaxEvents = 1 << 20;
}  // namespace

const SweepShape* tuned_sweep(int elem, int kind, Dims d) {
  Tuning* t = t_tune;
  if (!t || t->e.empty()) return nullptr;
  const SweepShape* x = t->find(elem, kind, d);
  return (x && (x->tx || x->zc)) ? x : nullptr;
}

int* wait_error_flag() { return t_tune ? t_tune->wait_err : nullptr; }
unsigned wait_limit() { return t_tune ? t_tune->wait_limit : kDefaultWaitLimit; }

void prof_begin(int cls, cudaStream_t s) {
  Profiler* p = t_prof;
  if (!p || !p->timing || p->overflow || !((p->mask >> cls) & 1u)) return;
  if (p->used + 2 > p->pool.size()) {
    if (p->pool.size() + 4096 > kMaxEvents) {
      p->overflow = true;
      return;
    }
    for (int i = 0; i < 4096; ++i) {
      cudaEvent_t e;
      IBRD_CUDA(cudaEventCreate(&e));
      p->pool.push_back(e);
    }
  }
  IBRD_CUDA(cudaEventRecord(p->pool[p->used], s));
  p->open_idx = p->used;
  p->open_cls = cls;
  p->used += 2;
}

void prof_end(int cls, cudaStream_t s, const char* what, double bytes) {
  check_launch(what);
  Profiler* p = t_prof;
  if (!p) return;
  p->launches++;
  p->count[cls]++;
  p->bytes[cls] += bytes;
  if (bytes > p->max_bytes[cls]) p->max_bytes[cls] = bytes;
  if (p->open_cls == cls) {
    p->open_cls = -1;
    if (bytes < p->min_bytes) {
      p->used -= 2;  // not timed: return the unused event pair
      return;
    }
    IBRD_CUDA(cudaEventRecord(p->pool[p->open_idx + 1], s));
    p->pending.emplace_back(cls, p->open_idx);
    p->pending_bytes.push_back(bytes);
  }
}

}  // namespace ibrd

using namespace ibrd;

struct ibrd_grid_s {
  int dev = 0;
  Dims d{};
  double h = 1, chi = 1, alpha = 0;
  int kernel = 4;
  int precision = IBRD_FP64;
  cudaStream_t s = nullptr;
  std::vector<Level> levels;
  int small_from = 0;           // first level handled by the single-CTA coarse V-cycle
  int exact32 = -1;             // FP32 V-cycles: level solved exactly by the Hartley transform (-1: none)
  Hier<double> h64;
  Hier<float> h32;
  BlobSet blobs;
  double* scal = nullptr;       // S_COUNT device scalars
  double* partial = nullptr;    // kRedBlocks * kDotGroup
  double* host = nullptr;       // pinned host scalars
  int* dflag = nullptr;
  unsigned* ticket = nullptr;  // last-CTA ticket of the fused reduction tails (0 between uses)
  // Krylov workspace
  double* V = nullptr;
  double* Z = nullptr;
  size_t vlen = 0;        // length of the current solve's vectors
  size_t vcap_elems = 0;  // capacity of V and Z (doubles each)
  double *H = nullptr, *cs = nullptr, *sn = nullptr, *gvec = nullptr, *yv = nullptr, *hb2 = nullptr;
  double* vsc = nullptr;  // inverse norms of the stored Krylov basis vectors (restart + 2)
  int hcap = 0;
  double *xs = nullptr, *bs = nullptr;  // saddle [c; lambda] solution and rhs
  size_t xs_cap = 0;
  // iterative refinement: FP64 residual, its FP32 copy and the FP32 correction
  double* ir_r = nullptr;
  float *ir_r32 = nullptr, *ir_d32 = nullptr;
  size_t ir_cap = 0;
  // preconditioner workspaces (FP64 and FP32 fields)
  double *p64[4] = {nullptr, nullptr, nullptr, nullptr};
  float *p32[4] = {nullptr, nullptr, nullptr, nullptr};
  // N-vector workspaces
  double *nv[4] = {nullptr, nullptr, nullptr, nullptr};
  double *U = nullptr, *Hs = nullptr, *scs = nullptr, *ssn = nullptr, *sg = nullptr;
  int ncap = -1, ucap = 0;
  double gamma_diag = 0.0;      // M_11 for the diagonal preconditioner
  bool gamma_valid = false;
  // block preconditioner of the Schur complement (IBRD_PRECOND_BLOCK): slots
  // (kBlockMax per blob), counts, rows, FP32 positions; built for one blob
  // configuration (blob_version, bumped by ibrd_set_blobs) and cutoff
  int* blk_idx = nullptr;
  int* blk_cnt = nullptr;
  float* blk_val = nullptr;
  float4* blk_pos = nullptr;
  int blk_cap = 0;
  long blob_version = 0;
  long blk_version = -1;
  double blk_cutoff = 0.0;
  // counters of the current solve
  long vcycles = 0;
  long inner = 0;
  long reorths = 0;
  long refinements = 0;
  Profiler prof;
  Tuning tune;  // launch shapes from ibrd_autotune
  // CUDA graphs of preconditioner applications, one per Krylov index j
  struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    long long launches = 0;
    long long count[P_NCLASS] = {};
    double bytes[P_NCLASS] = {};
    long vcycles = 0, inner = 0;  // solver counters one application adds
    int seen = 0;
  };
  std::map<std::string, std::vector<GraphEntry>> graphs;  // by configuration key
  cudaStream_t cap_stream = nullptr;
  // whole refinement solves as one graph each (opts.graphs == 2), by key
  struct SolveGraph {
    cudaGraph_t graph = nullptr;     // kept: a batch graph embeds it as a child graph
    cudaGraphExec_t exec = nullptr;
    int seen = 0;
    // launches one pass of each part adds (for the launch counter)
    long long l_init = 0, l_ref = 0, l_cyc = 0, l_true = 0;
    std::vector<long long> l_it;     // per Krylov index
    long vc_per_app = 0, inner_per_app = 0;
  };
  std::map<std::string, SolveGraph> sgraphs;
  void* gst = nullptr;               // device state of a graph solve
  double* ghist = nullptr;           // device residual history of a graph solve
  std::vector<cudaStream_t> cap_pool;  // streams that capture conditional bodies
  std::string err;
};

namespace ibrd {
namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

template <typename T>
T* dalloc(size_t n) {
  T* p = nullptr;
  IBRD_CUDA(cudaMalloc(&p, sizeof(T) * (n ? n : 1)));
  return p;
}

// The wait flag is an int written into the low bytes of a zeroed double slot.
bool wait_bits(double v) {
  unsigned long long u;
  std::memcpy(&u, &v, sizeof(u));
  return u != 0;
}

double host_scalar(ibrd_grid g, int slot) {
  IBRD_CUDA(cudaMemcpyAsync(g->host, g->scal + slot, sizeof(double), cudaMemcpyDeviceToHost, g->s));
  IBRD_CUDA(cudaStreamSynchronize(g->s));
  return g->host[0];
}

// S = h^-3 J^T (Sec. III.A): the spreading kernels take h^-3 in their scale.
double inv_h3(ibrd_grid g) { return 1.0 / (g->h * g->h * g->h); }

Stencil stencil(double h, double chi, double shift) {
  const double off = chi / (h * h);
  return Stencil{shift + 6.0 * off, off};
}

template <typename T>
Hier<T>& hier(ibrd_grid g);
template <>
Hier<double>& hier<double>(ibrd_grid g) { return g->h64; }
template <>
Hier<float>& hier<float>(ibrd_grid g) { return g->h32; }

template <typename T>
void ensure_hier(ibrd_grid g) {
  Hier<T>& H = hier<T>(g);
  if (!H.x.empty()) return;
  const size_t L = g->levels.size();
  H.x.assign(L, nullptr);
  H.b.assign(L, nullptr);
  H.y.assign(L, nullptr);
  for (size_t l = 0; l < L; ++l) {
    if (l > 0) {
      H.x[l] = dalloc<T>(g->levels[l].d.n());
      H.b[l] = dalloc<T>(g->levels[l].d.n());
    }
    if (l + 1 < L) H.y[l] = dalloc<T>(g->levels[l].d.n());
  }
}

// Hartley tables of the FP32 exact level for a shift.
const float* hartley_table(ibrd_grid g, double shift) {
  Hier<float>& H = g->h32;
  for (auto& e : H.hartley)
    if (e.first == shift) return e.second;
  const Level& le = g->levels[g->exact32];
  float* t = dalloc<float>(hartley_table_size(le.d));
  launch_hartley_tables(t, le.d, stencil(le.h, g->chi, shift), shift == 0.0 ? 1 : 0, g->s);
  H.hartley.emplace_back(shift, t);
  return t;
}

template <typename T>
const T* coarse_table(ibrd_grid g, double shift) {
  Hier<T>& H = hier<T>(g);
  for (auto& e : H.tables)
    if (e.first == shift) return e.second;
  const Level& lc = g->levels.back();
  T* t = dalloc<T>(lc.d.n());
  launch_coarse_table<T>(t, lc.d, stencil(lc.h, g->chi, shift), shift == 0.0 ? 1 : 0, g->s);
  H.tables.emplace_back(shift, t);
  return t;
}

// Levels l .. L-1 of the hierarchy as the single-CTA coarse V-cycle sees them.
CoarseLevels small_levels(ibrd_grid g, int l, double shift) {
  CoarseLevels cl{};
  cl.n = (int)g->levels.size() - l;
  int tot = 0;
  for (int i = 0; i < cl.n; ++i) {
    const Level& li = g->levels[l + i];
    const Stencil si = stencil(li.h, g->chi, shift);
    cl.nx[i] = li.d.nx;
    cl.ny[i] = li.d.ny;
    cl.nz[i] = li.d.nz;
    cl.off[i] = tot;
    auto lg = [](int v) { return (v & (v - 1)) == 0 ? __builtin_ctz((unsigned)v) : -1; };
    cl.lgx[i] = lg(li.d.nx);
    cl.lgy[i] = lg(li.d.ny);
    cl.diag[i] = si.diag;
    cl.offd[i] = si.off;
    tot += (int)li.d.n();
  }
  cl.total = tot;
  return cl;
}

// One V-cycle on level l for A_l x = b - bshift (bshift nullable). Smoothing
// sweeps ping-pong between x and the level's scratch field. If part is
// non-null (finest level only) the last smoothing sweep also writes per-CTA
// sums of the new x there; the return value is their count (0: none).
template <typename T>
int vcycle_level(ibrd_grid g, int l, const T* b, const double* bshift, T* x, bool zero, double shift, int nu1,
                 int nu2, double* part) {
  Hier<T>& H = hier<T>(g);
  const Level& lv = g->levels[l];
  const Stencil st = stencil(lv.h, g->chi, shift);
  if (sizeof(T) == 4 && l == g->exact32) {
    // FP32 hierarchy: this level is solved exactly
    launch_hartley_solve(hartley_table(g, shift), reinterpret_cast<const float*>(b), bshift,
                         reinterpret_cast<float*>(x), lv.d, g->s);
    return 0;
  }
  if (l == (int)g->levels.size() - 1) {
    // Exact coarsest solve. A constant shift of b only changes the mean, which
    // the singular pseudo-inverse ignores; the nonsingular case never shifts.
    launch_coarse_solve<T>(coarse_table<T>(g, shift), b, x, lv.d, g->s);
    return 0;
  }
  // the coarse end of the hierarchy runs in one CTA out of shared memory
  // (FP64 V-cycles, and FP32 ones on grids without an exact level)
  if (l >= g->small_from && !(sizeof(T) == 4 && g->exact32 >= 0)) {
    const CoarseLevels cl = small_levels(g, l, shift);
    launch_vcycle_small<T>(cl, b, x, bshift, coarse_table<T>(g, shift), zero, nu1, nu2, g->s);
    return 0;
  }
  const int part_cap = kRedBlocks * kDotGroup;
  T* cur = x;
  T* oth = H.y[l];
  bool first = zero;
  int np = 0;
  if (sizeof(T) == 4 && nu1 == 1 && zero && zero_restrict_rows_ok(lv.d) && aligned16(b) && aligned16(cur) &&
      wait_error_flag()) {
    // rows of 128 or 256 cells: the single pre-smoothing sweep from zero and
    // the restriction in one pass, row-resident and fed by TMA
    prof_begin(P_RBGS32, g->s);
    launch_zero_restrict_rows(reinterpret_cast<const float*>(b), bshift, reinterpret_cast<float*>(cur),
                              reinterpret_cast<float*>(H.b[l + 1]), lv.d, st, zero_restrict_rows_default_zc(lv.d),
                              g->s);
    prof_end(P_RBGS32, g->s, "zero_restrict_rows", 8.5 * sizeof(T) / 4.0 * lv.d.n());
  } else if (sizeof(T) == 4 && nu1 == 1 && zero && zero_restrict_ok(lv.d) && aligned16(b) && aligned16(cur) &&
             lv.d.n() <= (size_t(1) << 21)) {
    // the single pre-smoothing sweep from zero and the restriction in one pass
    // (levels up to 128^3 cells; on larger ones the kernel is bound by its
    // shared-memory traffic and the two streaming kernels are faster)
    launch_zero_restrict(reinterpret_cast<const float*>(b), bshift, reinterpret_cast<float*>(cur),
                         reinterpret_cast<float*>(H.b[l + 1]), lv.d, st, g->s);
  } else {
    if (nu1 == 0 && zero) IBRD_CUDA(cudaMemsetAsync(x, 0, sizeof(T) * lv.d.n(), g->s));
    for (int sweep = 0; sweep < nu1; ++sweep) {
      if (launch_rb_sweep<T>(cur, oth, b, bshift, lv.d, st, first, nullptr, 0, g->s) >= 0) std::swap(cur, oth);
      first = false;
    }
    launch_resid_restrict<T>(cur, b, bshift, H.b[l + 1], lv.d, st, g->s);
  }
  vcycle_level<T>(g, l + 1, H.b[l + 1], nullptr, H.x[l + 1], true, shift, nu1, nu2, nullptr);
  int sweep = 0;
  if (nu2 >= 1) {
    // the coarse-grid correction inside the first post-smoothing sweep
    const int r = launch_prolong_sweep<T>(H.x[l + 1], cur, oth, b, bshift, lv.d, st, nu2 == 1 ? part : nullptr,
                                          part_cap, g->s);
    if (r >= 0) {
      std::swap(cur, oth);
      np = nu2 == 1 ? r : 0;
      sweep = 1;
    }
  }
  if (sweep == 0) launch_prolong8<T>(H.x[l + 1], cur, lv.d, g->s);
  for (; sweep < nu2; ++sweep) {
    const bool last = (sweep == nu2 - 1);
    const int r = launch_rb_sweep<T>(cur, oth, b, bshift, lv.d, st, false, last ? part : nullptr, part_cap, g->s);
    if (r >= 0) std::swap(cur, oth);
    np = last ? (r > 0 ? r : 0) : np;
  }
  if (cur != x) IBRD_CUDA(cudaMemcpyAsync(x, cur, sizeof(T) * lv.d.n(), cudaMemcpyDeviceToDevice, g->s));
  return np;
}

// What a singular (shift = 0) V-cycle does with the mean of its result.
enum class XMean {
  Project,  // subtract it: the restricted inverse of Appendix A (mean-zero result)
  Report,   // write it to *xmean and leave x unprojected
  Ignore    // leave x unprojected; the caller's use is invariant to a constant
};

// One V-cycle on the finest level for (shift I - chi L) x = b. When shift is
// 0 (periodic, singular) the right-hand side is taken with its mean removed
// (bmean: that mean if the caller knows it, else computed here) and the
// result's mean is handled as `xm` says.
template <typename T>
void vcycle(ibrd_grid g, const T* b, T* x, bool zero, double shift, int nu1, int nu2, const double* bmean = nullptr,
            XMean xm = XMean::Project, double* xmean = nullptr) {
  ensure_hier<T>(g);
  const Dims d = g->d;
  const bool singular = (shift == 0.0);
  const double* bshift = nullptr;
  if (singular) {
    if (!bmean) {
      launch_sum<T>(b, d.n(), g->partial, g->scal + S_MEAN, 1.0 / (double)d.n(), g->s, g->ticket);
      bmean = g->scal + S_MEAN;
    }
    bshift = bmean;
  }
  const bool want = singular && xm != XMean::Ignore;
  const int np = vcycle_level<T>(g, 0, b, bshift, x, zero, shift, nu1, nu2, want ? g->partial : nullptr);
  if (want) {
    double* mout = (xm == XMean::Report && xmean) ? xmean : g->scal + S_MEANX;
    if (np > 0)
      launch_finalize(g->partial, np, mout, 1.0 / (double)d.n(), g->s);
    else
      launch_sum<T>(x, d.n(), g->partial, mout, 1.0 / (double)d.n(), g->s, g->ticket);
    if (xm == XMean::Project) launch_sub_scalar<T>(x, d.n(), mout, g->s);
  }
  g->vcycles++;
}

// n V-cycles; the mean options apply to every cycle (the last one's report
// is the result's).
template <typename T>
void vcycles(ibrd_grid g, const T* b, T* x, bool zero, double shift, int n, int nu1, int nu2,
             const double* bmean = nullptr, XMean xm = XMean::Project, double* xmean = nullptr) {
  for (int i = 0; i < n; ++i) {
    const XMean m = (i + 1 < n && xm == XMean::Report) ? XMean::Ignore : xm;
    vcycle<T>(g, b, x, zero && i == 0, shift, nu1, nu2, bmean, m, xmean);
  }
}

// ---------------------------------------------------------------- Krylov
// A linear operator with its preconditioner on vectors of type E (FP64 or
// FP32 Krylov vectors).
template <typename E>
struct LinOp {
  virtual ~LinOp() = default;
  virtual void apply(const E* x, E* y) = 0;
  // r = b - K x
  virtual void residual(const E* b, const E* x, E* r) = 0;
  virtual void precond(const E* v, E* z) = 0;
  // everything a preconditioner application depends on besides v and z
  virtual std::string key() const = 0;
  // device operands apply and residual read beyond the handle's own arrays
  virtual std::string operands() const { return std::string(); }
};

void drop_batch_graphs_of(ibrd_grid g);

void free_graphs(ibrd_grid g) {
  drop_batch_graphs_of(g);  // a batch graph bakes in this handle's launches too
  for (auto& kv : g->graphs)
    for (auto& e : kv.second)
      if (e.exec) cudaGraphExecDestroy(e.exec);
  g->graphs.clear();
  for (auto& kv : g->sgraphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
  }
  g->sgraphs.clear();
}

// Apply the preconditioner z = P(v) for Krylov index j. The launch sequence
// of one application is fixed for a given configuration and j (all buffers
// and device scalars have fixed addresses), so from the second encounter on
// it is captured once into a CUDA graph and replayed with one launch. The
// first encounter runs directly, which also performs any lazy allocation.
// Capture happens on a private stream (the legacy default stream cannot be
// captured); the graph is launched on the handle's stream. While per-launch
// timing is on the sequence always runs directly.
template <typename E>
void run_precond(ibrd_grid g, LinOp<E>& op, int j, const E* v, E* z, bool use_graphs) {
  Profiler& p = g->prof;
  if (!use_graphs || p.timing) {
    op.precond(v, z);
    return;
  }
  // blob data enters the graphs through device arrays (whose contents may
  // change between solves) and through the blob and covered-cell counts and
  // array addresses (which may not)
  const BlobSet& bl = g->blobs;
  char sig[256];
  std::snprintf(sig, sizeof sig, "|%d|%d|%p|%p|%p|%p|%p|%p|%p|%p|%zu", bl.n, bl.n_cells, (void*)g->V, (void*)g->Z,
                (void*)bl.idx, (void*)bl.w32, (void*)bl.w64, (void*)bl.cells, (void*)bl.cell_tile,
                (void*)bl.tile_blobs, g->vlen);
  const std::string key = op.key() + sig;
  if (g->graphs.size() > 16 && !g->graphs.count(key)) free_graphs(g);
  auto& list = g->graphs[key];
  if ((int)list.size() <= j) list.resize(j + 1);
  auto& e = list[j];
  if (!e.exec) {
    if (e.seen == 0) {
      e.seen = 1;
      op.precond(v, z);
      return;
    }
    if (!g->cap_stream) IBRD_CUDA(cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking));
    const long long l0 = p.launches;
    long long c0[P_NCLASS];
    double b0[P_NCLASS];
    for (int c = 0; c < P_NCLASS; ++c) {
      c0[c] = p.count[c];
      b0[c] = p.bytes[c];
    }
    const long v0 = g->vcycles, i0 = g->inner;
    cudaStream_t user = g->s;
    g->s = g->cap_stream;
    cudaGraph_t graph = nullptr;
    IBRD_CUDA(cudaStreamBeginCapture(g->s, cudaStreamCaptureModeRelaxed));
    try {
      op.precond(v, z);
    } catch (...) {
      cudaStreamEndCapture(g->s, &graph);
      if (graph) cudaGraphDestroy(graph);
      g->s = user;
      throw;
    }
    const cudaError_t ec = cudaStreamEndCapture(g->s, &graph);
    g->s = user;
    if (ec != cudaSuccess) throw CudaError{ec, "cudaStreamEndCapture"};
    const cudaError_t ei = cudaGraphInstantiate(&e.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      e.exec = nullptr;
      throw CudaError{ei, "cudaGraphInstantiate"};
    }
    // the capture counted launches (and V-cycles) that did not run; keep
    // them per graph and add them at each replay
    e.vcycles = g->vcycles - v0;
    e.inner = g->inner - i0;
    g->vcycles = v0;
    g->inner = i0;
    e.launches = p.launches - l0;
    p.launches = l0;
    for (int c = 0; c < P_NCLASS; ++c) {
      e.count[c] = p.count[c] - c0[c];
      e.bytes[c] = p.bytes[c] - b0[c];
      p.count[c] = c0[c];
      p.bytes[c] = b0[c];
    }
  }
  IBRD_CUDA(cudaGraphLaunch(e.exec, g->s));
  g->vcycles += e.vcycles;
  g->inner += e.inner;
  p.launches += e.launches;
  for (int c = 0; c < P_NCLASS; ++c) {
    p.count[c] += e.count[c];
    p.bytes[c] += e.bytes[c];
  }
}

// The Krylov bases V ((restart+1) vectors) and Z (restart vectors) of length
// n live in two blocks that are only ever grown, so the reaction (n = N_c) and
// saddle (n = N_c + N) solves of one handle, in either precision, share them
// without reallocating. Vectors start every ld elements, ld = n rounded up to
// 32 elements (128-byte aligned vectors for the 16-byte copies of the
// smoother and the 4-vector Krylov kernels). Returns ld.
template <typename E>
size_t ensure_krylov(ibrd_grid g, size_t n, int restart) {
  const size_t ld = (n + 31) & ~size_t(31);
  const size_t need = (ld * (size_t)(restart + 1) * sizeof(E) + 7) / 8;  // in doubles
  if (need > g->vcap_elems) {
    free_graphs(g);
    cudaFree(g->V);
    cudaFree(g->Z);
    g->V = g->Z = nullptr;
    g->V = dalloc<double>(need);
    g->Z = dalloc<double>(need);
    g->vcap_elems = need;
  }
  g->vlen = ld * sizeof(E);
  if (g->hcap < restart) {
    cudaFree(g->H);
    cudaFree(g->cs);
    cudaFree(g->sn);
    cudaFree(g->gvec);
    cudaFree(g->yv);
    cudaFree(g->hb2);
    cudaFree(g->vsc);
    g->H = dalloc<double>((size_t)(restart + 1) * restart);
    g->cs = dalloc<double>(restart);
    g->sn = dalloc<double>(restart);
    g->gvec = dalloc<double>(restart + 1);
    g->yv = dalloc<double>(restart);
    g->hb2 = dalloc<double>(restart + 1);
    g->vsc = dalloc<double>(restart + 2);
    const std::vector<double> ones((size_t)restart + 2, 1.0);  // V[0] is always normalised exactly
    IBRD_CUDA(cudaMemcpyAsync(g->vsc, ones.data(), sizeof(double) * ones.size(), cudaMemcpyHostToDevice, g->s));
    IBRD_CUDA(cudaStreamSynchronize(g->s));
    g->hcap = restart;
  }
  return ld;
}

// w (= V[j+1]) <- w - sum_{i<=j} h_i v_i, the projections h written into
// H[:, j], h_{j+1,j} (the norm of w after) into H[j+1, j], ||w||^2 before into
// S_TMP and h_{j+1,j}^2 into S_SQ; then V[j+1] is the new basis vector. Stored
// basis vectors need not have norm 1: V[i] = v_i / vsc[i], vsc[i] its inverse
// norm, and every projection and coefficient carries that factor. Classical
// Gram-Schmidt. Without a second pass (eta <= 0) the pass that subtracts the
// projections also scales the new vector by the reciprocal of its norm as
// estimated from them, and the exact norm of what it stored, taken in the same
// pass, fixes h_{j+1,j} and vsc[j+1] (no separate normalisation pass). With the
// DGKS second pass (threshold eta, decided on the device, its kernels
// returning at once when it is not needed) the vector is normalised after it.
// Without the second pass and with at most kDotGroup - 1 basis vectors the
// reductions of both passes, the norm bookkeeping and the Givens step of
// column j run in the last CTA of the multi-dot and multi-axpy launches;
// returns true when the Givens step is done.
template <typename E>
bool orthogonalize(ibrd_grid g, int j, size_t n, size_t ld, int ldh, double eta) {
  E* V = reinterpret_cast<E*>(g->V);
  E* w = V + (size_t)(j + 1) * ld;
  double* hcol = g->H + (size_t)j * ldh;
  double* vs = g->vsc;
  double* sc = g->scal;
  const int nb = j + 1;  // basis vectors V[0..j]
  if (eta <= 0.0 && nb + 1 <= kDotGroup) {
    DotTail dt;
    dt.ticket = g->ticket;
    dt.out = hcol;
    dt.scale = vs;
    dt.nscale = nb;
    dt.nb = nb;
    dt.ww = sc + S_TMP;
    dt.hhat = sc + S_HHAT;
    dt.hinv = sc + S_HINV;
    launch_multidot(V, ld, nb + 1, w, n, g->partial, g->s, nullptr, &dt);
    AxpyTail at;
    at.ticket = g->ticket;
    at.rho2 = sc + S_RHO2;
    at.hhat = sc + S_HHAT;
    at.hsub = hcol + nb;
    at.vscale = vs + nb;
    at.sq = sc + S_SQ;
    at.H = g->H;
    at.ldh = ldh;
    at.j = j;
    at.cs = g->cs;
    at.sn = g->sn;
    at.gvec = g->gvec;
    at.res = sc + S_RES;
    launch_multi_axpy(w, V, ld, nb, hcol, -1.0, n, g->partial, g->s, nullptr, vs, sc + S_HINV, &at);
    return true;
  }
  // pass 1: dots of V[0..j+1] (the last is <w, w>, unscaled)
  for (int g0 = 0; g0 < nb + 1; g0 += kDotGroup) {
    const int m = std::min(kDotGroup, nb + 1 - g0);
    launch_multidot(V + (size_t)g0 * ld, ld, m, w, n, g->partial, g->s);
    launch_reduce_partials(g->partial, m, hcol + g0, g->s, nullptr, vs + g0, std::max(0, std::min(m, nb - g0)));
  }
  if (eta <= 0.0) {
    launch_gs_norm_estimate(hcol, nb, sc + S_TMP, sc + S_HHAT, sc + S_HINV, g->s);
    for (int g0 = 0; g0 < nb; g0 += kDotGroup) {
      const int m = std::min(kDotGroup, nb - g0);
      const bool last = g0 + m >= nb;
      launch_multi_axpy(w, V + (size_t)g0 * ld, ld, m, hcol + g0, -1.0, n, last ? g->partial : nullptr, g->s,
                        nullptr, vs + g0, last ? sc + S_HINV : nullptr);
    }
    launch_reduce_partials(g->partial, 1, sc + S_RHO2, g->s);
    launch_gs_norm_fix(sc + S_RHO2, sc + S_HHAT, hcol + nb, vs + nb, sc + S_SQ, g->s);
    return false;
  }
  IBRD_CUDA(cudaMemcpyAsync(sc + S_TMP, hcol + nb, sizeof(double), cudaMemcpyDeviceToDevice, g->s));
  for (int g0 = 0; g0 < nb; g0 += kDotGroup) {
    const int m = std::min(kDotGroup, nb - g0);
    const bool last = g0 + m >= nb;
    launch_multi_axpy(w, V + (size_t)g0 * ld, ld, m, hcol + g0, -1.0, n, last ? g->partial : nullptr, g->s,
                      nullptr, vs + g0);
  }
  launch_reduce_partials(g->partial, 1, sc + S_SQ, g->s);
  const double* gate = sc + S_RFLAG;
  launch_reorth_flag(sc + S_TMP, sc + S_SQ, eta, sc + S_RFLAG, sc + S_RCOUNT, g->s);
  for (int g0 = 0; g0 < nb; g0 += kDotGroup) {
    const int m = std::min(kDotGroup, nb - g0);
    launch_multidot(V + (size_t)g0 * ld, ld, m, w, n, g->partial, g->s, gate);
    launch_reduce_partials(g->partial, m, g->hb2 + g0, g->s, gate, vs + g0, m);
  }
  for (int g0 = 0; g0 < nb; g0 += kDotGroup) {
    const int m = std::min(kDotGroup, nb - g0);
    const bool last = g0 + m >= nb;
    launch_multi_axpy(w, V + (size_t)g0 * ld, ld, m, g->hb2 + g0, -1.0, n, last ? g->partial : nullptr, g->s,
                      gate, vs + g0);
  }
  launch_reduce_partials(g->partial, 1, sc + S_SQ, g->s, gate);
  launch_vec_add_small(hcol, g->hb2, nb, g->s, gate);
  launch_gs_norm_unit(sc + S_SQ, hcol + nb, vs + nb, g->s);
  launch_scale_by_inv<E>(w, w, n, hcol + nb, 1.0, g->s);
  return false;
}

struct SolveResult {
  ibrd_status st = IBRD_OK;
  int iters = 0;
  double rel = 0;
};

// Where the per-iteration residual estimates go: entry = scale * |g_{j+1}| / ||b||.
struct History {
  double* buf = nullptr;
  int cap = 0;
  int len = 0;
  double scale = 1.0;
  void add(double v) {
    if (buf && len < cap) buf[len++] = scale * v;
  }
};

// Right-preconditioned flexible GMRES (Saad 1993) with true-residual restarts,
// on vectors of type E, to relative residual tol in at most max_iter
// iterations. With trust_estimate the solve ends as soon as the Givens
// residual estimate meets tol (no true residual is formed then): used for the
// inner solves of iterative refinement, whose caller forms the true residual
// itself.
template <typename E>
SolveResult fgmres(ibrd_grid g, LinOp<E>& op, const E* b, E* x, size_t n, const ibrd_solve_opts& o, double tol,
                   int max_iter, bool zero_guess, History& hist, bool trust_estimate = false,
                   const double* b_sq = nullptr, double b_norm = -1.0) {
  SolveResult R;
  const int m = std::max(1, o.restart);
  const size_t ld = ensure_krylov<E>(g, n, m);
  IBRD_CUDA(cudaMemsetAsync(g->scal + S_RCOUNT, 0, sizeof(double), g->s));
  const int ldh = m + 1;
  E* V = reinterpret_cast<E*>(g->V);
  E* Z = reinterpret_cast<E*>(g->Z);
  // ||b||: from the caller when it already holds it (b_sq: ||b||^2 on the
  // device, b_norm: ||b|| on the host), else one reduction
  const bool known = b_sq && b_norm >= 0.0;
  double bnorm = b_norm;
  if (!known) {
    launch_dot<E>(b, b, n, g->partial, g->scal + S_BB, 1.0, g->s, g->ticket);
    bnorm = std::sqrt(host_scalar(g, S_BB));
  }
  if (!std::isfinite(bnorm)) {
    R.st = IBRD_ERR_NONFINITE;
    return R;
  }
  if (bnorm == 0.0) {
    IBRD_CUDA(cudaMemsetAsync(x, 0, sizeof(E) * n, g->s));
    return R;
  }
  // r0 = b - K x0; from a zero guess with ||b|| known, V[0] is scaled
  // straight from b
  bool first_from_b = false;
  double beta;
  if (zero_guess && known) {
    IBRD_CUDA(cudaMemsetAsync(x, 0, sizeof(E) * n, g->s));
    launch_sqrt_scalar(b_sq, g->scal + S_NORM, g->s);
    beta = bnorm;
    first_from_b = true;
  } else {
    if (zero_guess) {
      IBRD_CUDA(cudaMemsetAsync(x, 0, sizeof(E) * n, g->s));
      IBRD_CUDA(cudaMemcpyAsync(V, b, sizeof(E) * n, cudaMemcpyDeviceToDevice, g->s));
    } else {
      op.residual(b, x, V);
    }
    launch_dot<E>(V, V, n, g->partial, g->scal + S_TMP2, 1.0, g->s, g->ticket);
    launch_sqrt_scalar(g->scal + S_TMP2, g->scal + S_NORM, g->s);
    beta = std::sqrt(host_scalar(g, S_TMP2));
  }
  while (true) {
    R.rel = beta / bnorm;
    if (!std::isfinite(R.rel)) {
      R.st = IBRD_ERR_NONFINITE;
      break;
    }
    if (R.rel <= tol) break;
    if (R.iters >= max_iter) {
      R.st = IBRD_ERR_NOT_CONVERGED;
      break;
    }
    // V[0] = r / beta, gvec = [beta, 0, ...]
    launch_scale_by_inv<E>(first_from_b ? b : V, V, n, g->scal + S_NORM, 1.0, g->s);
    first_from_b = false;
    prof_begin(P_SMALL, g->s);
    k_set_gvec<<<1, 64, 0, g->s>>>(g->gvec, m, g->scal + S_NORM);
    prof_end(P_SMALL, g->s, "set_gvec");
    int k = 0;
    bool breakdown = false, estimate_met = false;
    double res_last = 0.0;
    for (int j = 0; j < m; ++j) {
      E* vj = V + (size_t)j * ld;
      E* zj = Z + (size_t)j * ld;
      E* w = V + (size_t)(j + 1) * ld;
      run_precond<E>(g, op, j, vj, zj, o.graphs != 0);
      op.apply(zj, w);
      if (!orthogonalize<E>(g, j, n, ld, ldh, o.reorth_eta))
        launch_givens(g->H, ldh, j, g->cs, g->sn, g->gvec, g->scal + S_RES, g->s);
      // one host read per iteration: residual estimate and the norms
      IBRD_CUDA(cudaMemcpyAsync(g->host, g->scal, sizeof(double) * (S_WAIT + 1), cudaMemcpyDeviceToHost, g->s));
      IBRD_CUDA(cudaStreamSynchronize(g->s));
      const double res = g->host[S_RES], sq = g->host[S_SQ], ww = g->host[S_TMP];
      if (wait_bits(g->host[S_WAIT])) {
        R.st = IBRD_ERR_TIMEOUT;
        break;
      }
      // breakdown: w lies in the span of V (a zero or negligible new column,
      // relative to the rounding of E); V[j+1] is then not used again
      const double floor_sq = sizeof(E) == 4 ? 1e-12 : 1e-28;
      const bool tiny = !(sq > floor_sq * ww) || sq <= 0.0;
      k = j + 1;
      R.iters++;
      res_last = res;
      hist.add(res / bnorm);
      if (!std::isfinite(res) || !std::isfinite(sq)) {
        R.st = IBRD_ERR_NONFINITE;
        break;
      }
      if (tiny) {
        breakdown = true;
        break;
      }
      if (res / bnorm <= tol) {
        estimate_met = true;
        break;
      }
      if (R.iters >= max_iter) break;
    }
    if (R.st == IBRD_ERR_NONFINITE || R.st == IBRD_ERR_TIMEOUT) break;
    // x += Z y
    launch_backsolve(g->H, ldh, k, g->gvec, g->yv, g->s);
    for (int g0 = 0; g0 < k; g0 += kDotGroup) {
      const int mm = std::min(kDotGroup, k - g0);
      launch_multi_axpy(x, Z + (size_t)g0 * ld, ld, mm, g->yv + g0, 1.0, n, nullptr, g->s);
    }
    if (trust_estimate && (estimate_met || breakdown)) {
      R.rel = res_last / bnorm;
      break;
    }
    // true residual
    op.residual(b, x, V);
    launch_dot<E>(V, V, n, g->partial, g->scal + S_TMP2, 1.0, g->s, g->ticket);
    launch_sqrt_scalar(g->scal + S_TMP2, g->scal + S_NORM, g->s);
    beta = std::sqrt(host_scalar(g, S_TMP2));
    if (breakdown && beta / bnorm > tol) {
      R.rel = beta / bnorm;
      // an invariant subspace was found but the true residual disagrees:
      // restart once more unless nothing changes
      if (R.iters >= max_iter) {
        R.st = IBRD_ERR_BREAKDOWN;
        break;
      }
    }
  }
  g->reorths += (long)host_scalar(g, S_RCOUNT);
  return R;
}

// FP64 solve of K x = b through FP32 Krylov iterations (iterative refinement):
// the residual r = b - K x is formed in FP64 (op64), the correction solves
// K d = r / ||r|| by FP32 FGMRES (op32, FP32 preconditioner) to relative
// residual max(inner_tol, tol ||b|| / (2 ||r||)), and x += ||r|| d in FP64.
// Each refinement step multiplies the FP64 residual by about the inner
// tolerance until the FP64 rounding floor, so the stopping test below is on
// the true FP64 residual, as for the FP64 solver.
SolveResult refine(ibrd_grid g, LinOp<double>& op64, LinOp<float>& op32, const double* b, double* x, size_t n,
                   const ibrd_solve_opts& o, bool zero_guess, History& hist) {
  SolveResult R;
  if (g->ir_cap < n) {
    cudaFree(g->ir_r);
    cudaFree(g->ir_r32);
    cudaFree(g->ir_d32);
    g->ir_r = nullptr;
    g->ir_r32 = g->ir_d32 = nullptr;
    g->ir_r = dalloc<double>(n);
    g->ir_r32 = dalloc<float>(n);
    g->ir_d32 = dalloc<float>(n);
    g->ir_cap = n;
  }
  double* r = g->ir_r;
  launch_dot<double>(b, b, n, g->partial, g->scal + S_BB, 1.0, g->s, g->ticket);
  const double bnorm = std::sqrt(host_scalar(g, S_BB));
  if (!std::isfinite(bnorm)) {
    R.st = IBRD_ERR_NONFINITE;
    return R;
  }
  if (bnorm == 0.0) {
    IBRD_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, g->s));
    return R;
  }
  // The FP32 right-hand side of a refinement step is sigma r, sigma a power
  // of two that brings the expected norm of r near 1 (FP32 squares stay in
  // range); the step's correction is then divided by sigma.
  double sigma = 1.0;
  auto set_sigma = [&](double expect) { sigma = std::ldexp(1.0, -std::ilogb(std::max(expect, 1e-300))); };
  double r32norm = 0.0;  // ||sigma r|| of the FP32 right-hand side, ||.||^2 kept in S_TMP2
  auto to_f32 = [&](const double* v) {
    launch_convert_sq(v, g->ir_r32, n, sigma, g->partial, g->scal + S_TMP2, g->s, g->ticket);
    r32norm = std::sqrt(host_scalar(g, S_TMP2));
    return r32norm / sigma;
  };
  double rnorm;
  set_sigma(bnorm);
  if (zero_guess) {
    IBRD_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, g->s));
    to_f32(b);
    rnorm = bnorm;
  } else {
    op64.residual(b, x, r);
    rnorm = to_f32(r);
  }
  int stalled = 0;
  while (true) {
    R.rel = rnorm / bnorm;
    if (!std::isfinite(R.rel)) {
      R.st = IBRD_ERR_NONFINITE;
      break;
    }
    if (R.rel <= o.tol) break;
    if (R.iters >= o.max_iter) {
      R.st = IBRD_ERR_NOT_CONVERGED;
      break;
    }
    // three refinement steps in a row that do not halve the residual: the
    // FP32 corrections no longer improve the FP64 iterate
    if (stalled >= 3) {
      R.st = IBRD_ERR_NOT_CONVERGED;
      break;
    }
    const double tol_in = std::max(o.inner_tol, 0.5 * o.tol / R.rel);
    hist.scale = R.rel;
    const SolveResult I =
        fgmres<float>(g, op32, g->ir_r32, g->ir_d32, n, o, tol_in, o.max_iter - R.iters, true, hist, true,
                      g->scal + S_TMP2, r32norm);
    R.iters += I.iters;
    g->refinements++;
    if (I.st == IBRD_ERR_NONFINITE || I.st == IBRD_ERR_TIMEOUT) {
      R.st = I.st;
      break;
    }
    launch_add_scaled(1.0 / sigma, g->ir_d32, x, n, g->s);
    op64.residual(b, x, r);
    set_sigma(rnorm * std::max(I.rel, 1e-7));
    const double rn = to_f32(r);
    stalled = (rn > 0.5 * rnorm) ? stalled + 1 : 0;
    rnorm = rn;
  }
  return R;
}

// ---------------------------------------------------------------- device-terminated refinement
// The refinement solve of `refine` as ONE CUDA graph whose loops end on the
// device: the refinement steps and the FGMRES restart cycles are conditional
// WHILE nodes, Krylov index j of a cycle is a conditional IF node (its kernels
// keep the fixed addresses of V[j], Z[j], H[:, j]), and the solution update of
// a cycle with k columns is body k of a SWITCH node. One-thread control kernels
// after each Givens rotation, cycle and refinement step take the decisions the
// host loop takes (same tests, same order) and set the conditions, so a solve
// is one graph launch and one host read at the end. The state lives in device
// memory (GState); the residual history goes to a device buffer.
enum : int { GF_MET = 1, GF_BREAKDOWN = 2, GF_NONFINITE = 4, GF_TIMEOUT = 8 };
constexpr int kGHistCap = 4096;

// Parameters of a graph solve, rewritten before every launch (the head of GState).
struct GParams {
  double tol, inner_tol, floor_sq;
  int max_iter, restart;
};
struct GState {
  double tol, inner_tol, floor_sq;
  int max_iter, restart;
  double bnorm, rnorm, sigma, rel;         // refinement: ||b||, ||r||, scale, ||r|| / ||b||
  double tol_in, bn_in, rel_in, res_last;  // inner FGMRES of the current step
  double hist_scale;
  int iters, it_in, max_in, stalled, status, refinements, cycles, trues, k, flags, hist_len, zero_x;
  long long upd_launches;
  int jcount[64];                          // iterations run at each Krylov index
};

__device__ __forceinline__ void gset(cudaGraphConditionalHandle h, bool v) { cudaGraphSetConditional(h, v ? 1u : 0u); }

// after ||b||^2 (scal[S_BB]) and, with a guess, ||sigma r||^2 (scal[S_TMP2])
__global__ void k_g_init(GState* st, const double* __restrict__ scal, int zero_guess, int phase,
                         cudaGraphConditionalHandle h_ref) {
  if (threadIdx.x != 0) return;
  if (phase == 0) {
    st->iters = st->stalled = st->status = st->refinements = st->cycles = st->trues = st->hist_len = 0;
    st->zero_x = 0;
    st->upd_launches = 0;
    for (int j = 0; j < 64; ++j) st->jcount[j] = 0;
    const double bn = sqrt(scal[S_BB]);
    st->bnorm = bn;
    st->sigma = ldexp(1.0, -ilogb(fmax(bn, 1e-300)));
    st->rnorm = bn;
    st->rel = 1.0;
  }
  const double bn = st->bnorm;
  bool go = false;
  if (!isfinite(bn)) {
    st->status = IBRD_ERR_NONFINITE;
  } else if (bn == 0.0) {
    st->rel = 0.0;
    st->zero_x = 1;
  } else if (phase == 0 && !zero_guess) {
    go = false;  // the residual of the guess decides (phase 1)
  } else {
    if (phase == 1) {
      st->rnorm = sqrt(scal[S_TMP2]) / st->sigma;
      st->rel = st->rnorm / bn;
    }
    const double rel = st->rel;
    if (!isfinite(rel))
      st->status = IBRD_ERR_NONFINITE;
    else if (rel <= st->tol)
      st->status = IBRD_OK;
    else if (st->iters >= st->max_iter)
      st->status = IBRD_ERR_NOT_CONVERGED;
    else
      go = true;
  }
  gset(h_ref, go);
}

// start of a refinement step: the inner FGMRES solves for sigma r (norm in S_TMP2)
__global__ void k_g_ref_begin(GState* st, double* __restrict__ scal, cudaGraphConditionalHandle h_cyc) {
  if (threadIdx.x != 0) return;
  st->tol_in = fmax(st->inner_tol, 0.5 * st->tol / st->rel);
  st->hist_scale = st->rel;
  const double bn = sqrt(scal[S_TMP2]);
  st->bn_in = bn;
  scal[S_NORM] = bn;
  st->max_in = st->max_iter - st->iters;
  st->it_in = 0;
  st->flags = 0;
  st->rel_in = 1.0;
  bool go = true;
  if (!isfinite(bn)) {
    st->flags |= GF_NONFINITE;
    go = false;
  } else if (bn == 0.0 || st->max_in <= 0) {
    go = false;
  }
  gset(h_cyc, go);
}

struct IfHandles {
  cudaGraphConditionalHandle h[61];
};

// start of a restart cycle: index 0 runs, the others wait for their predecessor
__global__ void k_g_cyc_begin(GState* st, IfHandles hs, int m) {
  if (threadIdx.x != 0) return;
  st->k = 0;
  st->cycles++;
  st->flags &= ~(GF_MET | GF_BREAKDOWN);
  for (int j = 0; j < m; ++j) gset(hs.h[j], j == 0);
}

// after the Givens rotation of index j: the host loop's per-iteration tests
__global__ void k_g_it_ctrl(GState* st, const double* __restrict__ scal, double* __restrict__ hist, int j, int m,
                            cudaGraphConditionalHandle h_next, cudaGraphConditionalHandle h_k) {
  if (threadIdx.x != 0) return;
  const double res = scal[S_RES], sq = scal[S_SQ], ww = scal[S_TMP];
  unsigned long long wb;
  const double wv = scal[S_WAIT];
  memcpy(&wb, &wv, sizeof(wb));
  const bool tiny = !(sq > st->floor_sq * ww) || sq <= 0.0;
  st->k = j + 1;
  st->iters++;
  st->it_in++;
  st->jcount[j]++;
  st->res_last = res;
  if (st->hist_len < kGHistCap) hist[st->hist_len++] = st->hist_scale * (res / st->bn_in);
  if (wb != 0)
    st->flags |= GF_TIMEOUT;
  else if (!isfinite(res) || !isfinite(sq))
    st->flags |= GF_NONFINITE;
  else if (tiny)
    st->flags |= GF_BREAKDOWN;
  else if (res / st->bn_in <= st->tol_in)
    st->flags |= GF_MET;
  const bool bad = st->flags & (GF_NONFINITE | GF_TIMEOUT);
  const bool cont = !(st->flags & (GF_MET | GF_BREAKDOWN)) && !bad && st->it_in < st->max_in && j + 1 < m;
  if (j + 1 < m) gset(h_next, cont);
  if (!cont) {
    // the cycle ends here: its update uses k columns (none after a fault)
    const int k = bad ? 0 : j + 1;
    cudaGraphSetConditional(h_k, (unsigned)k);
    st->upd_launches += k ? 1 + (k + 7) / 8 : 0;
  }
}

// end of a cycle's update: trust the estimate after convergence or breakdown
// (as the refinement's inner solves do), else form the true residual
__global__ void k_g_cyc_ctrl1(GState* st, cudaGraphConditionalHandle h_true, cudaGraphConditionalHandle h_cyc) {
  if (threadIdx.x != 0) return;
  const int f = st->flags;
  bool tr = false;
  if (f & (GF_NONFINITE | GF_TIMEOUT)) {
  } else if (f & (GF_MET | GF_BREAKDOWN)) {
    st->rel_in = st->res_last / st->bn_in;
  } else {
    tr = true;
  }
  if (tr) st->trues++;
  gset(h_true, tr);
  if (!tr) gset(h_cyc, false);
}

__global__ void k_g_cyc_ctrl2(GState* st, const double* __restrict__ scal, cudaGraphConditionalHandle h_cyc) {
  if (threadIdx.x != 0) return;
  const double beta = sqrt(scal[S_TMP2]);
  st->rel_in = beta / st->bn_in;
  bool go = false;
  if (!isfinite(st->rel_in))
    st->flags |= GF_NONFINITE;
  else
    go = st->rel_in > st->tol_in && st->it_in < st->max_in;
  gset(h_cyc, go);
}

// after the inner solve: stop on a fault, else update x
__global__ void k_g_upd_gate(GState* st, cudaGraphConditionalHandle h_upd, cudaGraphConditionalHandle h_ref) {
  if (threadIdx.x != 0) return;
  const int f = st->flags;
  const bool bad = f & (GF_NONFINITE | GF_TIMEOUT);
  if (bad) {
    st->status = (f & GF_TIMEOUT) ? IBRD_ERR_TIMEOUT : IBRD_ERR_NONFINITE;
    gset(h_ref, false);
  }
  gset(h_upd, !bad);
}

__global__ void k_g_sigma(GState* st) {
  if (threadIdx.x != 0) return;
  st->sigma = ldexp(1.0, -ilogb(fmax(st->rnorm * fmax(st->rel_in, 1e-7), 1e-300)));
}

__global__ void k_g_ref_ctrl(GState* st, const double* __restrict__ scal, cudaGraphConditionalHandle h_ref) {
  if (threadIdx.x != 0) return;
  st->refinements++;
  const double rn = sqrt(scal[S_TMP2]) / st->sigma;
  st->stalled = (rn > 0.5 * st->rnorm) ? st->stalled + 1 : 0;
  st->rnorm = rn;
  st->rel = rn / st->bnorm;
  bool go = false;
  if (!isfinite(st->rel))
    st->status = IBRD_ERR_NONFINITE;
  else if (st->rel <= st->tol)
    st->status = IBRD_OK;
  else if (st->iters >= st->max_iter || st->stalled >= 3)
    st->status = IBRD_ERR_NOT_CONVERGED;
  else
    go = true;
  gset(h_ref, go);
}

// Stream capture into conditional bodies: a conditional node is added after
// the work captured so far on g->s; each body is captured on a stream of the
// handle's pool (one per nesting depth) with g->s pointing at it.
struct GCapture {
  ibrd_grid g;
  int depth = 0;
  long long* counter;  // launch counter of the part being captured
  cudaStream_t stream(int d) {
    while ((int)g->cap_pool.size() <= d) {
      cudaStream_t st = nullptr;
      IBRD_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
      g->cap_pool.push_back(st);
    }
    return g->cap_pool[d];
  }
  cudaGraph_t current_graph() {
    cudaStreamCaptureStatus cs;
    cudaGraph_t graph = nullptr;
    IBRD_CUDA(cudaStreamGetCaptureInfo(g->s, &cs, nullptr, &graph, nullptr, nullptr, nullptr));
    if (cs != cudaStreamCaptureStatusActive) throw CudaError{cudaErrorStreamCaptureInvalidated, "graph solve capture"};
    return graph;
  }
  cudaGraphConditionalHandle handle() {
    cudaGraphConditionalHandle h;
    IBRD_CUDA(cudaGraphConditionalHandleCreate(&h, current_graph(), 0, 0));
    return h;
  }
  template <typename F>
  void conditional(cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type, int nbody, F&& fill) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t graph = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* ed = nullptr;
    size_t nd = 0;
    IBRD_CUDA(cudaStreamGetCaptureInfo(g->s, &cs, nullptr, &graph, &deps, &ed, &nd));
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = type;
    p.conditional.size = (unsigned)nbody;
    cudaGraphNode_t node;
    IBRD_CUDA(cudaGraphAddNode(&node, graph, deps, ed, nd, &p));
    IBRD_CUDA(cudaStreamUpdateCaptureDependencies(g->s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaStream_t outer = g->s;
    ++depth;
    for (int b = 0; b < nbody; ++b) {
      cudaStream_t sb = stream(depth);
      IBRD_CUDA(cudaStreamBeginCaptureToGraph(sb, p.conditional.phGraph_out[b], nullptr, nullptr, 0,
                                              cudaStreamCaptureModeRelaxed));
      g->s = sb;
      try {
        fill(b);
      } catch (...) {
        cudaGraph_t dummy;
        cudaStreamEndCapture(sb, &dummy);
        g->s = outer;
        --depth;
        throw;
      }
      cudaGraph_t out = nullptr;
      IBRD_CUDA(cudaStreamEndCapture(sb, &out));
      g->s = outer;
    }
    --depth;
  }
};

// Record a refinement solve (b, x as in `refine`) onto g->s, which is being
// captured; SG receives the launch counts of its parts.
void capture_refine(ibrd_grid g, LinOp<double>& op64, LinOp<float>& op32, const double* b, double* x, size_t n,
                    const ibrd_solve_opts& o, bool zero_guess, ibrd_grid_s::SolveGraph& SG) {
  Profiler& p = g->prof;
  const int m = std::max(1, o.restart);
  const size_t ld = ensure_krylov<float>(g, n, m);
  const int ldh = m + 1;
  float* V = reinterpret_cast<float*>(g->V);
  float* Z = reinterpret_cast<float*>(g->Z);
  GState* st = reinterpret_cast<GState*>(g->gst);
  double* sc = g->scal;
  GCapture C{g, 0, nullptr};
  const long long l00 = p.launches;
  long long c00[P_NCLASS];
  double b00[P_NCLASS];
  for (int c = 0; c < P_NCLASS; ++c) {
    c00[c] = p.count[c];
    b00[c] = p.bytes[c];
  }
  const long v00 = g->vcycles, i00 = g->inner;
  auto mark = [&]() { return p.launches; };  // counts library launches (the control kernels add 1 each below)
  {
    cudaGraphConditionalHandle h_ref = C.handle();
    long long t0 = mark();
    launch_dot<double>(b, b, n, g->partial, sc + S_BB, 1.0, g->s, g->ticket);
    k_g_init<<<1, 32, 0, g->s>>>(st, sc, zero_guess ? 1 : 0, 0, h_ref);
    if (zero_guess) {
      IBRD_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, g->s));
      launch_convert_sq(b, g->ir_r32, n, &st->sigma, g->partial, sc + S_TMP2, g->s, g->ticket);
    } else {
      op64.residual(b, x, g->ir_r);
      launch_convert_sq(g->ir_r, g->ir_r32, n, &st->sigma, g->partial, sc + S_TMP2, g->s, g->ticket);
      k_g_init<<<1, 32, 0, g->s>>>(st, sc, 0, 1, h_ref);
    }
    SG.l_init = mark() - t0 + (zero_guess ? 1 : 2);
    C.conditional(h_ref, cudaGraphCondTypeWhile, 1, [&](int) {
      cudaGraphConditionalHandle h_cyc = C.handle(), h_upd = C.handle();
      k_g_ref_begin<<<1, 32, 0, g->s>>>(st, sc, h_cyc);
      IBRD_CUDA(cudaMemsetAsync(g->ir_d32, 0, sizeof(float) * n, g->s));
      IBRD_CUDA(cudaMemcpyAsync(V, g->ir_r32, sizeof(float) * n, cudaMemcpyDeviceToDevice, g->s));
      C.conditional(h_cyc, cudaGraphCondTypeWhile, 1, [&](int) {
        IfHandles hs{};
        for (int j = 0; j < m; ++j) hs.h[j] = C.handle();
        cudaGraphConditionalHandle h_k = C.handle(), h_true = C.handle();
        const long long c0 = mark();
        k_g_cyc_begin<<<1, 32, 0, g->s>>>(st, hs, m);
        launch_scale_by_inv<float>(V, V, n, sc + S_NORM, 1.0, g->s);
        prof_begin(P_SMALL, g->s);
        k_set_gvec<<<1, 64, 0, g->s>>>(g->gvec, m, sc + S_NORM);
        prof_end(P_SMALL, g->s, "set_gvec");
        SG.l_cyc = mark() - c0 + 2;  // with the cycle's two control kernels
        SG.l_it.assign(m, 0);
        for (int j = 0; j < m; ++j) {
          C.conditional(hs.h[j], cudaGraphCondTypeIf, 1, [&](int) {
            const long long a0 = mark();
            const long va = g->vcycles, ia = g->inner;
            float* vj = V + (size_t)j * ld;
            float* zj = Z + (size_t)j * ld;
            float* w = V + (size_t)(j + 1) * ld;
            op32.precond(vj, zj);
            if (j == 0) {
              SG.vc_per_app = g->vcycles - va;
              SG.inner_per_app = g->inner - ia;
            }
            op32.apply(zj, w);
            if (!orthogonalize<float>(g, j, n, ld, ldh, o.reorth_eta))
              launch_givens(g->H, ldh, j, g->cs, g->sn, g->gvec, sc + S_RES, g->s);
            k_g_it_ctrl<<<1, 32, 0, g->s>>>(st, sc, g->ghist, j, m, j + 1 < m ? hs.h[j + 1] : hs.h[j], h_k);
            SG.l_it[j] = mark() - a0 + 1;
          });
        }
        C.conditional(h_k, cudaGraphCondTypeSwitch, m + 1, [&](int k) {
          if (k == 0) return;
          launch_backsolve(g->H, ldh, k, g->gvec, g->yv, g->s);
          for (int g0 = 0; g0 < k; g0 += kDotGroup) {
            const int mm = std::min(kDotGroup, k - g0);
            launch_multi_axpy(g->ir_d32, Z + (size_t)g0 * ld, ld, mm, g->yv + g0, 1.0, n, nullptr, g->s);
          }
        });
        k_g_cyc_ctrl1<<<1, 32, 0, g->s>>>(st, h_true, h_cyc);
        C.conditional(h_true, cudaGraphCondTypeIf, 1, [&](int) {
          const long long q0 = mark();
          op32.residual(g->ir_r32, g->ir_d32, V);
          launch_dot<float>(V, V, n, g->partial, sc + S_TMP2, 1.0, g->s, g->ticket);
          launch_sqrt_scalar(sc + S_TMP2, sc + S_NORM, g->s);
          k_g_cyc_ctrl2<<<1, 32, 0, g->s>>>(st, sc, h_cyc);
          SG.l_true = mark() - q0 + 1;
        });
      });
      k_g_upd_gate<<<1, 32, 0, g->s>>>(st, h_upd, h_ref);
      C.conditional(h_upd, cudaGraphCondTypeIf, 1, [&](int) {
        const long long u0 = mark();
        launch_add_divided(&st->sigma, g->ir_d32, x, n, g->s);
        op64.residual(b, x, g->ir_r);
        k_g_sigma<<<1, 32, 0, g->s>>>(st);
        launch_convert_sq(g->ir_r, g->ir_r32, n, &st->sigma, g->partial, sc + S_TMP2, g->s, g->ticket);
        k_g_ref_ctrl<<<1, 32, 0, g->s>>>(st, sc, h_ref);
        // a refinement step: its begin and gate kernels, this body and its two control kernels
        SG.l_ref = mark() - u0 + 4;
      });
    });
  }
  // the capture counted launches and V-cycles that did not run
  p.launches = l00;
  for (int c = 0; c < P_NCLASS; ++c) {
    p.count[c] = c00[c];
    p.bytes[c] = b00[c];
  }
  g->vcycles = v00;
  g->inner = i00;
}

void ensure_graph_state(ibrd_grid g) {
  if (!g->gst) g->gst = dalloc<unsigned char>(sizeof(GState));
  if (!g->ghist) g->ghist = dalloc<double>(kGHistCap);
  if (!g->cap_stream) IBRD_CUDA(cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking));
}

// Build the graph of one refinement solve.
void build_refine_graph(ibrd_grid g, LinOp<double>& op64, LinOp<float>& op32, const double* b, double* x,
                        size_t n, const ibrd_solve_opts& o, bool zero_guess, ibrd_grid_s::SolveGraph& SG) {
  ensure_graph_state(g);
  cudaStream_t user = g->s;
  g->s = g->cap_stream;
  cudaGraph_t graph = nullptr;
  IBRD_CUDA(cudaStreamBeginCapture(g->s, cudaStreamCaptureModeRelaxed));
  try {
    capture_refine(g, op64, op32, b, x, n, o, zero_guess, SG);
  } catch (...) {
    cudaGraph_t dummy = nullptr;
    cudaStreamEndCapture(g->s, &dummy);
    if (dummy) cudaGraphDestroy(dummy);
    g->s = user;
    throw;
  }
  const cudaError_t ec = cudaStreamEndCapture(g->s, &graph);
  g->s = user;
  if (ec != cudaSuccess) throw CudaError{ec, "cudaStreamEndCapture (graph solve)"};
  SG.graph = graph;
  const cudaError_t ei = cudaGraphInstantiate(&SG.exec, graph, 0);
  if (ei != cudaSuccess) {
    SG.exec = nullptr;
    throw CudaError{ei, "cudaGraphInstantiate (graph solve)"};
  }
}

// Device state to host after a graph solve; fills R, the history and the
// handle's counters.
SolveResult finish_refine_graph(ibrd_grid g, const ibrd_grid_s::SolveGraph& SG, double* x, size_t n,
                                History& hist) {
  GState hs;
  IBRD_CUDA(cudaMemcpyAsync(&hs, g->gst, sizeof(GState), cudaMemcpyDeviceToHost, g->s));
  IBRD_CUDA(cudaStreamSynchronize(g->s));
  SolveResult R;
  R.st = (ibrd_status)hs.status;
  R.iters = hs.iters;
  R.rel = hs.rel;
  if (hs.zero_x) IBRD_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, g->s));
  const int nh = std::min(hs.hist_len, kGHistCap);
  if (hist.buf && nh > 0) {
    std::vector<double> hb(nh);
    IBRD_CUDA(cudaMemcpy(hb.data(), g->ghist, sizeof(double) * nh, cudaMemcpyDeviceToHost));
    for (double v : hb) {
      if (hist.len < hist.cap) hist.buf[hist.len] = v;
      hist.len++;
    }
    hist.len = std::min(hist.len, hist.cap);
  }
  g->refinements += hs.refinements;
  g->vcycles += (long)hs.iters * SG.vc_per_app;
  g->inner += (long)hs.iters * SG.inner_per_app;
  long long launches = 1 + SG.l_init + (long long)hs.refinements * SG.l_ref + (long long)hs.cycles * SG.l_cyc +
                       (long long)hs.trues * SG.l_true + hs.upd_launches;
  for (int j = 0; j < (int)SG.l_it.size() && j < 64; ++j) launches += (long long)hs.jcount[j] * SG.l_it[j];
  g->prof.launches += launches;
  return R;
}

// Everything baked into the graph of a refinement solve.
std::string refine_graph_key(ibrd_grid g, LinOp<double>& op64, LinOp<float>& op32, const double* b, double* x,
                             size_t n, const ibrd_solve_opts& o, bool zero_guess) {
  const BlobSet& bl = g->blobs;
  char sig[640];
  std::snprintf(sig, sizeof sig,
                "|G|%d|%d|%p|%p|%p|%p|%p|%p|%p|%p|%zu|%p|%p|%zu|%d|%d|%d|%.17g|%.17g|%.17g|%p|%p|%p|%p|%p|%u",
                bl.n, bl.n_cells, (void*)g->V, (void*)g->Z, (void*)bl.idx, (void*)bl.w32, (void*)bl.w64,
                (void*)bl.cells, (void*)bl.cell_tile, (void*)bl.tile_blobs, g->vlen, (const void*)b, (void*)x, n,
                o.restart, o.max_iter, zero_guess ? 1 : 0, o.tol, o.inner_tol, o.reorth_eta, (void*)g->ir_r,
                (void*)g->ir_r32, (void*)g->ir_d32, g->gst, (void*)g->ghist, g->tune.wait_limit);
  return op32.key() + op64.key() + op32.operands() + op64.operands() + sig;
}

// `refine` as one graph launch (built on the second solve of a configuration,
// when every lazy allocation has happened); null when the host loop should run.
ibrd_grid_s::SolveGraph* refine_graph_for(ibrd_grid g, LinOp<double>& op64, LinOp<float>& op32, const double* b,
                                          double* x, size_t n, const ibrd_solve_opts& o, bool zero_guess) {
  if (g->prof.timing || o.restart > 61) return nullptr;
  ensure_krylov<float>(g, n, std::max(1, o.restart));  // grows (and drops graphs) only before a key is taken
  ensure_graph_state(g);
  const std::string key = refine_graph_key(g, op64, op32, b, x, n, o, zero_guess);
  if (g->sgraphs.size() > 8 && !g->sgraphs.count(key)) free_graphs(g);
  auto& SG = g->sgraphs[key];
  if (SG.exec) return &SG;
  if (SG.seen == 0) {
    SG.seen = 1;
    return nullptr;
  }
  build_refine_graph(g, op64, op32, b, x, n, o, zero_guess, SG);
  return &SG;
}

static_assert(offsetof(GState, restart) == offsetof(GParams, restart) && sizeof(GParams) <= offsetof(GState, bnorm),
              "GParams is the head of GState");

// The parameters the control kernels read (before every launch of a solve graph).
void set_graph_params(ibrd_grid g, const ibrd_solve_opts& o) {
  GParams prm{o.tol, o.inner_tol, 1e-12, o.max_iter, o.restart};
  IBRD_CUDA(cudaMemcpyAsync(g->gst, &prm, sizeof(GParams), cudaMemcpyHostToDevice, g->s));
}

// The refinement solve: one graph launch when opts.graphs == 2 and its graph
// exists (from the second solve of a configuration on), else the host loop.
SolveResult run_refine(ibrd_grid g, LinOp<double>& op64, LinOp<float>& op32, const double* b, double* x, size_t n,
                       const ibrd_solve_opts& o, bool zero_guess, History& hist) {
  if (o.graphs == 2) {
    if (g->ir_cap >= n) {
      if (auto* SG = refine_graph_for(g, op64, op32, b, x, n, o, zero_guess)) {
        set_graph_params(g, o);
        IBRD_CUDA(cudaGraphLaunch(SG->exec, g->s));
        return finish_refine_graph(g, *SG, x, n, hist);
      }
    }
  }
  return refine(g, op64, op32, b, x, n, o, zero_guess, hist);
}

// ---------------------------------------------------------------- workspaces
template <typename T>
T* pfield(ibrd_grid g, int i);
template <>
double* pfield<double>(ibrd_grid g, int i) {
  if (!g->p64[i]) g->p64[i] = dalloc<double>(g->d.n());
  return g->p64[i];
}
template <>
float* pfield<float>(ibrd_grid g, int i) {
  if (!g->p32[i]) g->p32[i] = dalloc<float>(g->d.n());
  return g->p32[i];
}

void ensure_nvec(ibrd_grid g, int m) {
  const int n = g->blobs.n;
  if (g->ncap != n) {
    for (auto& p : g->nv) {
      cudaFree(p);
      p = nullptr;
    }
    for (auto& p : g->nv) p = dalloc<double>(std::max(n, 1));
    cudaFree(g->U);
    g->U = nullptr;
    g->ucap = 0;
    g->ncap = n;
  }
  if (g->ucap < m) {
    cudaFree(g->U);
    cudaFree(g->Hs);
    cudaFree(g->scs);
    cudaFree(g->ssn);
    cudaFree(g->sg);
    g->U = dalloc<double>((size_t)(m + 1) * std::max(n, 1));
    g->Hs = dalloc<double>((size_t)(m + 1) * m);
    g->scs = dalloc<double>(m);
    g->ssn = dalloc<double>(m);
    g->sg = dalloc<double>(m + 1);
    g->ucap = m;
  }
}

// ---------------------------------------------------------------- operators
// The FP64 residual of a solve in fixed point (launch_residual): within
// 2^-52 of its terms per cell, plus 2^-55 chi / h^2 max|c| from the scaling,
// which in cells far below the largest |c| can exceed the FP64 stencil's
// rounding; solves asking for relative residuals below kFxTolMin form it with
// the FP64 stencil.
constexpr double kFxTolMin = 1e-13;
double* fx_scratch(ibrd_grid g, const ibrd_solve_opts& o) { return o.tol >= kFxTolMin ? g->scal + S_XMAX : nullptr; }

// B c = alpha c - chi L c + S (kappa * J c)  (Eq. unsteady_system / steady_state)
// on Krylov vectors of type E; the preconditioner is V-cycles in T (FP32
// V-cycles inside FP64 FGMRES convert on the way in and out).
template <typename T, typename E = T>
struct ReactionOp : LinOp<E> {
  ibrd_grid g;
  const double* kappa;
  double sigma;
  ibrd_solve_opts o;
  ReactionOp(ibrd_grid g_, const double* k_, double sg, const ibrd_solve_opts& o_) : g(g_), kappa(k_), sigma(sg), o(o_) {}
  std::string key() const override {
    char buf[160];
    std::snprintf(buf, sizeof buf, "reaction|%zu|%zu|%d|%d|%d|%.17g", sizeof(T), sizeof(E), o.mg_cycles, o.nu1,
                  o.nu2, sigma);
    return buf;
  }
  std::string operands() const override {
    char buf[40];
    std::snprintf(buf, sizeof buf, "|k%p", (const void*)kappa);
    return buf;
  }
  void apply(const E* x, E* y) override {
    launch_interp<E>(g->blobs, g->d, x, 1.0, g->nv[0], g->s);
    launch_apply_A<E>(x, y, g->d, stencil(g->h, g->chi, g->alpha), g->s);
    launch_spread<E>(g->blobs, g->d, g->nv[0], kappa, inv_h3(g), y, 1, g->s);
  }
  void residual(const E* b, const E* x, E* r) override {
    launch_interp<E>(g->blobs, g->d, x, 1.0, g->nv[0], g->s);
    launch_residual<E>(x, b, r, g->d, stencil(g->h, g->chi, g->alpha), fx_scratch(g, o), g->s);
    launch_spread<E>(g->blobs, g->d, g->nv[0], kappa, -inv_h3(g), r, 1, g->s);
  }
  // n V-cycles of (sigma I - chi L) (Eq. Pinv_Poisson)
  void precond(const E* v, E* z) override {
    if constexpr (std::is_same<T, E>::value) {
      vcycles<T>(g, v, z, true, sigma, o.mg_cycles, o.nu1, o.nu2);
    } else {
      T* bt = pfield<T>(g, 0);
      T* xt = pfield<T>(g, 1);
      launch_convert<E, T>(v, bt, g->d.n(), 1.0, nullptr, g->s);
      vcycles<T>(g, bt, xt, true, sigma, o.mg_cycles, o.nu1, o.nu2);
      launch_convert<T, E>(xt, z, g->d.n(), 1.0, nullptr, g->s);
    }
  }
};

// K [c; lambda] = [A c + zeta S lambda; xi J c]  (Eq. saddle_point) on
// vectors [c; lambda] of type E. The preconditioner's V-cycles, spreading and
// interpolation run in T; its inner Schur GMRES basis has the vectors' type E.
template <typename T, typename E = T>
struct SaddleOp : LinOp<E> {
  ibrd_grid g;
  ibrd_solve_opts o;
  double zeta, xi;
  bool singular;
  SaddleOp(ibrd_grid g_, const ibrd_solve_opts& o_, double z, double x) : g(g_), o(o_), zeta(z), xi(x) {
    singular = (g->alpha == 0.0);
  }
  std::string key() const override {
    char buf[200];
    std::snprintf(buf, sizeof buf, "saddle|%zu|%zu|%d|%d|%d|%d|%d|%.17g|%.17g|%.17g|%.17g", sizeof(T), sizeof(E),
                  o.mg_cycles, o.nu1, o.nu2, o.schur_inner, o.precond, zeta, xi, g->alpha, g->gamma_diag);
    std::string k = buf;
    if (o.precond == IBRD_PRECOND_BLOCK) {
      std::snprintf(buf, sizeof buf, "|B%p|%p|%p", (void*)g->blk_idx, (void*)g->blk_cnt, (void*)g->blk_val);
      k += buf;
    }
    return k;
  }
  void apply(const E* x, E* y) override {
    const size_t nc = g->d.n();
    launch_apply_A<E>(x, y, g->d, stencil(g->h, g->chi, g->alpha), g->s);
    launch_spread<E, E>(g->blobs, g->d, x + nc, nullptr, zeta * inv_h3(g), y, 1, g->s);
    launch_interp<E, E>(g->blobs, g->d, x, xi, y + nc, g->s);
  }
  void residual(const E* b, const E* x, E* r) override {
    const size_t nc = g->d.n();
    launch_residual<E>(x, b, r, g->d, stencil(g->h, g->chi, g->alpha), fx_scratch(g, o), g->s);
    launch_spread<E, E>(g->blobs, g->d, x + nc, nullptr, -zeta * inv_h3(g), r, 1, g->s);
    launch_interp<E, E>(g->blobs, g->d, x, -xi, r + nc, g->s);
    launch_axpby<E>(1.0, b + nc, 1.0, r + nc, g->blobs.n, g->s);
  }
  // Appendix A, steps 1-5, with A~_n^-1 = n V-cycles and, for the approximate
  // Schur complement, m GMRES iterations on J A~_1^-1 S.
  //
  // When A is singular the restricted inverse needs mean-zero input and gives
  // mean-zero output. The means involved are known without extra passes over
  // the grid: spreading preserves sums (h^3 sum S u = sum u), so the mean of
  // S U_j comes from the N-vector U_j; the source's mean comes out of the
  // FP64 -> FP32 conversion; and the result means are summed inside the last
  // smoothing sweep. Where a constant offset of a field cancels (c~ is used
  // only through c~ + cbar with cbar = <f/xi - J c~> and J 1 = 1) the mean is
  // not formed at all.
  void precond(const E* v, E* z) override {
    const size_t nc = g->d.n();
    const int N = g->blobs.n;
    const E* vc = v;
    const E* vf = v + nc;
    E* zc = z;
    E* zl = z + nc;
    T* gt = pfield<T>(g, 0);   // g~
    T* cs = pfield<T>(g, 1);   // c~* then c~
    const double volume = (double)nc * g->h * g->h * g->h;
    const double shift = g->alpha;
    const double ih3 = inv_h3(g);
    double* sc = g->scal;
    // step 1: g~ = g - alpha V N^-1 S <g>, c~* = A~_n^-1 g~
    const double* bmean = nullptr;
    const double* xshift = nullptr;
    if (singular) {
      launch_convert_sum<E, T>(vc, gt, nc, g->partial, sc + S_GSUM, sc + S_G32SUM, g->s, g->ticket);
      // zeta S (lambda-bar 1) = (V / (N N_c)) sum(g) S 1; its total is sum(g)
      launch_spread_const<T>(g->blobs, g->d, sc + S_GSUM, -volume / ((double)N * (double)nc) * ih3, gt, g->s);
      prof_begin(P_SMALL, g->s);
      k_scalar_affine<<<1, 1, 0, g->s>>>(sc + S_LBAR, sc + S_GSUM, volume / (zeta * N * (double)nc));
      prof_end(P_SMALL, g->s, "lbar");
      prof_begin(P_SMALL, g->s);
      k_bmean1<<<1, 1, 0, g->s>>>(sc + S_BMEAN1, sc + S_G32SUM, sc + S_GSUM, 1.0 / (double)nc);
      prof_end(P_SMALL, g->s, "bmean");
      bmean = sc + S_BMEAN1;
      xshift = sc + S_XMEAN1;
      vcycles<T>(g, gt, cs, true, shift, o.mg_cycles, o.nu1, o.nu2, bmean, XMean::Report, sc + S_XMEAN1);
    } else {
      launch_convert<E, T>(vc, gt, nc, 1.0, nullptr, g->s);
      vcycles<T>(g, gt, cs, true, shift, o.mg_cycles, o.nu1, o.nu2);
    }
    // step 2: rhs = (zeta xi)^-1 (xi J c~* - f), with J applied to the
    // mean-zero c~* (J 1 = 1, so subtracting the mean of c~* from J c~*)
    double* rhs = g->nv[0];
    double* lam = g->nv[1];
    launch_interp<T>(g->blobs, g->d, cs, 1.0, rhs, g->s);
    launch_nvec_affine(rhs, rhs, N, 1.0 / zeta, xshift, vf, -1.0 / (zeta * xi), g->s);
    if (o.precond == IBRD_PRECOND_DIAG) {
      launch_convert<double, double>(rhs, lam, N, 1.0 / g->gamma_diag, nullptr, g->s);
      if (singular) {
        launch_sum<double>(lam, N, g->partial, sc + S_TMP, 1.0 / N, g->s, g->ticket);
        launch_sub_scalar<double>(lam, N, sc + S_TMP, g->s);
      }
    } else {
      const int m = std::max(1, o.schur_inner);
      T* fs = pfield<T>(g, 2);
      T* fx = pfield<T>(g, 3);
      // mean of S U_j = h^-3 sum(U_j) / N_c
      const double ub_scale = ih3 / (double)nc;
      // the inner basis has the Krylov vectors' precision E
      E* U = reinterpret_cast<E*>(g->U);
      // IBRD_PRECOND_BLOCK (alpha = 0 only): GMRES on P M~ lambda = P rhs, P
      // the block preconditioner, its outputs made mean-free like M~'s
      const bool blk = o.precond == IBRD_PRECOND_BLOCK;
      const double* start = rhs;
      if (blk) {
        double* prhs = g->nv[2];
        launch_block_apply<double, double>(g->blk_idx, g->blk_cnt, g->blk_val, rhs, nullptr, N, prhs, g->partial,
                                           g->s, g->ticket, sc + S_PMEAN, 1.0 / N);
        launch_sub_scalar<double>(prhs, N, sc + S_PMEAN, g->s);
        start = prhs;
      }
      launch_small_start<E>(start, U, N, g->sg, m, singular ? sc + S_UB : nullptr, ub_scale, g->s);
      for (int j = 0; j < m; ++j) {
        launch_spread<T, E>(g->blobs, g->d, U + (size_t)j * N, nullptr, ih3, fs, 0, g->s);
        if (singular)
          vcycle<T>(g, fs, fx, true, shift, o.nu1, o.nu2, sc + S_UB + j, XMean::Report, sc + S_UX + j);
        else
          vcycle<T>(g, fs, fx, true, shift, o.nu1, o.nu2);
        const double* wshift = singular ? sc + S_UX + j : nullptr;
        if (blk) {
          // J of the V-cycle result into scratch, P of it minus the result's
          // mean into the basis, whose own mean the Arnoldi step removes
          E* w = reinterpret_cast<E*>(g->nv[2]);
          launch_interp<T, E>(g->blobs, g->d, fx, 1.0, w, g->s);
          launch_block_apply<E, E>(g->blk_idx, g->blk_cnt, g->blk_val, w, wshift, N, U + (size_t)(j + 1) * N,
                                   g->partial, g->s, g->ticket, sc + S_PMEAN, 1.0 / N);
          wshift = sc + S_PMEAN;
        } else {
          launch_interp<T, E>(g->blobs, g->d, fx, 1.0, U + (size_t)(j + 1) * N, g->s);
        }
        launch_small_arnoldi<E>(U, N, j, g->Hs, m + 1, g->scs, g->ssn, g->sg, wshift,
                             singular && j + 1 < m ? sc + S_UB + j + 1 : nullptr, ub_scale, g->s);
        g->inner++;
      }
      launch_small_finish<E>(U, N, m, g->Hs, m + 1, g->sg, lam, singular ? 1 : 0, g->s);
    }
    // step 3: c~ = A~_n^-1 (g~ - zeta S lambda~) from c~*; lambda~ has mean
    // zero, so the right-hand side keeps the mean of g~
    launch_spread<T>(g->blobs, g->d, lam, nullptr, -zeta * ih3, gt, 1, g->s);
    if (singular)
      vcycles<T>(g, gt, cs, false, shift, o.mg_cycles, o.nu1, o.nu2, bmean, XMean::Ignore);
    else
      vcycles<T>(g, gt, cs, false, shift, o.mg_cycles, o.nu1, o.nu2);
    // steps 4-5: cbar = <f/xi - J c~>, c = c~ + cbar, lambda = lambda~ + lambda-bar
    if (singular) {
      double* t = g->nv[2];
      launch_interp<T>(g->blobs, g->d, cs, 1.0, t, g->s);
      launch_nvec_affine(t, t, N, -1.0, nullptr, vf, 1.0 / xi, g->s);
      launch_sum<double>(t, N, g->partial, sc + S_CBAR, 1.0 / N, g->s, g->ticket);
      launch_convert<double, E>(lam, zl, N, 1.0, sc + S_LBAR, g->s);
      launch_convert<T, E>(cs, zc, nc, 1.0, sc + S_CBAR, g->s);
    } else {
      launch_convert<double, E>(lam, zl, N, 1.0, nullptr, g->s);
      launch_convert<T, E>(cs, zc, nc, 1.0, nullptr, g->s);
    }
  }
};

__global__ void k_fill_or_scale(double* x, int n, double c, int scale) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = scale ? x[i] * c : c;
}

// Warm start of a saddle solve from a guess lambda0 of the multipliers (mode 1:
// the uniform share lambda0_i = h^3 sum(g) / (zeta N); mode 2: the caller's
// lambda, in x + N_c, scaled when A is singular to the solvability condition
// zeta sum(lambda) = h^3 sum(g), Appendix A). The grid part follows Appendix A
// steps 3-5 with lambda0 in place of the Schur solution: c~ = A~^-1 (g - zeta S
// lambda0) by `cycles` V-cycles in precision T and, when A is singular,
// c0 = c~ + cbar0 with cbar0 = <f/xi - J c~>. b = [g; f]; writes [c0; lambda0]
// into x.
template <typename T>
void saddle_warm_start(ibrd_grid g, const ibrd_solve_opts& o, const double* b, double* x, int mode, int cycles) {
  const size_t nc = g->d.n();
  const int N = g->blobs.n;
  const bool singular = (g->alpha == 0.0);
  const double h3 = g->h * g->h * g->h;
  double* sc = g->scal;
  double* lam = x + nc;
  launch_sum<double>(b, nc, g->partial, sc + S_TMP, h3 / o.zeta, g->s, g->ticket);
  if (mode == 2) launch_sum<double>(lam, N, g->partial, sc + S_TMP2, 1.0, g->s, g->ticket);
  IBRD_CUDA(cudaMemcpyAsync(g->host, sc + S_TMP, sizeof(double) * 2, cudaMemcpyDeviceToHost, g->s));
  IBRD_CUDA(cudaStreamSynchronize(g->s));
  const double total = g->host[0], lsum = mode == 2 ? g->host[1] : 0.0;
  const int nb = std::min(1024, (N + 255) / 256);
  prof_begin(P_SMALL, g->s);
  if (mode == 1 || (singular && !(std::isfinite(lsum) && lsum != 0.0)))
    k_fill_or_scale<<<nb, 256, 0, g->s>>>(lam, N, total / N, 0);
  else if (singular)
    k_fill_or_scale<<<nb, 256, 0, g->s>>>(lam, N, total / lsum, 1);
  prof_end(P_SMALL, g->s, "lambda0");
  // g - zeta S lambda0 (has mean zero when A is singular)
  T* rt = pfield<T>(g, 0);
  T* ct = pfield<T>(g, 1);
  IBRD_CUDA(cudaMemcpyAsync(x, b, sizeof(double) * nc, cudaMemcpyDeviceToDevice, g->s));
  launch_spread<double>(g->blobs, g->d, lam, nullptr, -o.zeta * inv_h3(g), x, 1, g->s);
  launch_convert<double, T>(x, rt, nc, 1.0, nullptr, g->s);
  vcycles<T>(g, rt, ct, true, g->alpha, std::max(1, cycles), o.nu1, o.nu2);
  if (singular) {
    double* t = g->nv[2];
    launch_interp<T>(g->blobs, g->d, ct, 1.0, t, g->s);
    launch_nvec_affine(t, t, N, -1.0, nullptr, b + nc, 1.0 / o.xi, g->s);
    launch_sum<double>(t, N, g->partial, sc + S_CBAR, 1.0 / N, g->s, g->ticket);
    launch_convert<T, double>(ct, x, nc, 1.0, sc + S_CBAR, g->s);
  } else {
    launch_convert<T, double>(ct, x, nc, 1.0, nullptr, g->s);
  }
}

// Warm start from the penalty form of the saddle point (Sec. II.B: the
// reaction-limited system with a large rate is a penalty method for the
// constrained one): relaxing xi J c = f to xi J c - (xi / kappa_p) lambda = f
// gives (A + zeta kappa_p S J) c = g + (zeta kappa_p / xi) S f and
// lambda = kappa_p (J c - f / xi). The first is a reaction-limited solve with
// the uniform rate zeta kappa_p (to relative residual o.penalty_tol, in the
// solve's precision mode); the pair starts the saddle solve. b = [g; f];
// writes [c; lambda] into x.
void saddle_penalty_start(ibrd_grid g, const ibrd_solve_opts& o, const double* b, double* x) {
  const size_t nc = g->d.n();
  const int N = g->blobs.n;
  const double kp = o.penalty_kappa;
  const double rate = o.zeta * kp;
  double* kappa = g->nv[3];
  const int nb = std::min(1024, (N + 255) / 256);
  prof_begin(P_SMALL, g->s);
  k_fill_or_scale<<<nb, 256, 0, g->s>>>(kappa, N, rate, 0);
  prof_end(P_SMALL, g->s, "penalty_kappa");
  double* bp = pfield<double>(g, 2);
  IBRD_CUDA(cudaMemcpyAsync(bp, b, sizeof(double) * nc, cudaMemcpyDeviceToDevice, g->s));
  launch_spread<double>(g->blobs, g->d, b + nc, nullptr, (o.zeta * kp / o.xi) * inv_h3(g), bp, 1, g->s);
  const double sigma = g->alpha > 0.0 ? g->alpha : rate * N / ((double)nc * g->h * g->h * g->h);
  ibrd_solve_opts op = o;
  op.tol = o.penalty_tol;
  History none;
  SolveResult R;
  if (o.precision == IBRD_FP64) {
    ReactionOp<double> r64(g, kappa, sigma, op);
    R = fgmres<double>(g, r64, bp, x, nc, op, op.tol, op.max_iter, true, none);
  } else if (o.precision == IBRD_MIXED_FP32) {
    ReactionOp<float, double> r(g, kappa, sigma, op);
    R = fgmres<double>(g, r, bp, x, nc, op, op.tol, op.max_iter, true, none);
  } else {
    ReactionOp<double> r64(g, kappa, sigma, op);
    ReactionOp<float> r32(g, kappa, sigma, op);
    R = refine(g, r64, r32, bp, x, nc, op, true, none);
  }
  if (R.st == IBRD_ERR_NONFINITE) throw ArgError{IBRD_ERR_NONFINITE, "penalty start: non-finite residual"};
  // lambda = kappa_p J c - (kappa_p / xi) f
  launch_interp<double>(g->blobs, g->d, x, kp, x + nc, g->s);
  launch_nvec_affine(x + nc, x + nc, N, 1.0, nullptr, b + nc, -kp / o.xi, g->s);
}

// M_11 = (J A^-1 S)_11 of blob 0 by V-cycle iteration to convergence (used by
// the diagonal preconditioner, Eq. Schur_diagonal).
double compute_gamma(ibrd_grid g, const ibrd_solve_opts& o) {
  const size_t nc = g->d.n();
  double* e = pfield<double>(g, 0);
  double* x = pfield<double>(g, 1);
  double* unit = g->nv[3];
  IBRD_CUDA(cudaMemsetAsync(unit, 0, sizeof(double) * g->blobs.n, g->s));
  const double one = 1.0;
  IBRD_CUDA(cudaMemcpyAsync(unit, &one, sizeof(double), cudaMemcpyHostToDevice, g->s));
  launch_spread<double>(g->blobs, g->d, unit, nullptr, inv_h3(g), e, 0, g->s);
  for (int it = 0; it < 40; ++it) vcycle<double>(g, e, x, it == 0, g->alpha, o.nu1, o.nu2);
  launch_interp<double>(g->blobs, g->d, x, 1.0, g->nv[2], g->s);
  IBRD_CUDA(cudaMemcpyAsync(g->host, g->nv[2], sizeof(double), cudaMemcpyDeviceToHost, g->s));
  IBRD_CUDA(cudaStreamSynchronize(g->s));
  (void)nc;
  return g->host[0];
}

// The block preconditioner of the Schur complement for the current blobs
// (IBRD_PRECOND_BLOCK; rebuilt when the blobs or the cutoff change): the
// Green's function model of M off the diagonal (Sec. IV.A's periodic
// constant, here for any box by an Ewald sum), gamma on it.
void ensure_block(ibrd_grid g, const ibrd_solve_opts& o) {
  const int N = g->blobs.n;
  if (N <= 0) return;
  const double lx = g->d.nx * g->h, ly = g->d.ny * g->h, lz = g->d.nz * g->h, V = lx * ly * lz;
  const double pi = 3.14159265358979323846;
  // by default about 12 neighbours at the mean density: (4/3) pi rc^3 N / V = 12
  double rc = o.block_cutoff > 0.0 ? o.block_cutoff : std::cbrt(9.0 * V / (pi * N));
  rc = std::min(rc, 0.5 * std::min(lx, std::min(ly, lz)));  // a unique minimum image
  if (g->blk_version == g->blob_version && g->blk_cutoff == rc && g->blk_cap >= N) return;
  if (g->blk_cap < N) {
    free_graphs(g);  // captured applications hold the old arrays' addresses
    cudaFree(g->blk_idx);
    cudaFree(g->blk_cnt);
    cudaFree(g->blk_val);
    cudaFree(g->blk_pos);
    g->blk_idx = g->blk_cnt = nullptr;
    g->blk_val = nullptr;
    g->blk_pos = nullptr;
    g->blk_cap = 0;
    g->blk_idx = dalloc<int>((size_t)N * kBlockMax);
    g->blk_cnt = dalloc<int>(N);
    g->blk_val = dalloc<float>((size_t)N * kBlockMax);
    g->blk_pos = dalloc<float4>(N);
    g->blk_cap = N;
  }
  BlockModel m;
  m.a = (float)(1.0 / (4.0 * pi * g->chi));
  m.c0 = (float)(periodic_constant(lx, ly, lz) / g->chi);
  m.c2 = (float)(1.0 / (6.0 * g->chi * V));
  m.diag = (float)g->gamma_diag;
  m.rmin = (float)(2.0 * g->h);  // inside two cells the kernels overlap and 1/r is no model
  launch_block_setup(g->blobs.q, N, lx, ly, lz, rc, m, g->blk_pos, g->blk_idx, g->blk_cnt, g->blk_val, g->s);
  g->blk_version = g->blob_version;
  g->blk_cutoff = rc;
}

// Whether a bounded device wait of this handle's kernels gave up since the
// last check (then the flag is cleared). Waits for the handle's stream.
bool take_wait_flag(ibrd_grid g) {
  const bool flag = wait_bits(host_scalar(g, S_WAIT));
  if (flag) IBRD_CUDA(cudaMemsetAsync(g->scal + S_WAIT, 0, sizeof(double), g->s));
  return flag;
}

// Entry points that only enqueue work check the flag when the stream is not
// being captured into a graph (a capture cannot synchronize).
void check_waits_if_not_capturing(ibrd_grid g, const char* name) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  IBRD_CUDA(cudaStreamIsCapturing(g->s, &cs));
  if (cs == cudaStreamCaptureStatusNone && take_wait_flag(g))
    throw ArgError{IBRD_ERR_TIMEOUT, std::string(name) + ": a bounded device wait gave up"};
}

ibrd_status fail(ibrd_grid g, ibrd_status st, const std::string& msg) {
  if (g) g->err = msg;
  return st;
}

struct ProfScope {
  Profiler* prev;
  Tuning* prev_tune;
  ProfScope(Profiler* p, Tuning* t) : prev(t_prof), prev_tune(t_tune) {
    t_prof = p;
    t_tune = t;
  }
  ~ProfScope() {
    t_prof = prev;
    t_tune = prev_tune;
  }
};

template <typename F>
ibrd_status guarded(ibrd_grid g, const char* name, F&& f) {
  if (!g) return IBRD_ERR_ARG;
  DeviceGuard dg(g->dev);
  ProfScope ps(&g->prof, &g->tune);
  try {
    g->err.clear();
    return f();
  } catch (const ArgError& e) {
    return fail(g, e.code, std::string(name) + ": " + e.msg);
  } catch (const CudaError& e) {
    const ibrd_status st = (e.code == cudaErrorMemoryAllocation) ? IBRD_ERR_OOM : IBRD_ERR_CUDA;
    cudaGetLastError();
    return fail(g, st, std::string(name) + ": " + e.what + ": " + cudaGetErrorString(e.code));
  } catch (const std::bad_alloc&) {
    return fail(g, IBRD_ERR_OOM, std::string(name) + ": host allocation failed");
  }
}

ibrd_solve_opts resolve_opts(ibrd_grid g, const ibrd_solve_opts* in) {
  ibrd_solve_opts o;
  ibrd_default_opts(&o);
  if (in) o = *in;
  if (o.precision < 0) o.precision = g->precision;
  if (o.xi <= 0.0) o.xi = o.zeta / (g->h * g->h * g->h);
  if (!(o.tol > 0.0) || o.restart < 1 || o.restart > 60 || o.max_iter < 0 || o.mg_cycles < 1 ||
      o.schur_inner < 1 || o.schur_inner > 60 || o.nu1 < 0 || o.nu2 < 0 || !(o.zeta != 0.0) ||
      !(o.reorth_eta >= 0.0) || !(o.inner_tol > 0.0 && o.inner_tol < 1.0) ||
      (o.precision != IBRD_FP64 && o.precision != IBRD_MIXED_FP32 && o.precision != IBRD_MIXED_REFINE) ||
      (o.precond != IBRD_PRECOND_SCHUR && o.precond != IBRD_PRECOND_DIAG && o.precond != IBRD_PRECOND_AUTO &&
       o.precond != IBRD_PRECOND_BLOCK) || !std::isfinite(o.block_cutoff) ||
      (o.lambda_guess != IBRD_GUESS_NONE && o.lambda_guess != IBRD_GUESS_UNIFORM &&
       o.lambda_guess != IBRD_GUESS_GIVEN && o.lambda_guess != IBRD_GUESS_PENALTY) || o.warm_cycles < 1 ||
      o.warm_cycles > 64 || !(o.penalty_kappa > 0.0) || !std::isfinite(o.penalty_kappa) ||
      !(o.penalty_tol > 0.0 && o.penalty_tol < 1.0))
    throw ArgError{IBRD_ERR_ARG, "invalid solver options"};
  // blob counts up to which the diagonal preconditioner solved faster than the
  // approximate Schur one at m = 5 (measured at 128^3 and 256^3, both
  // precisions, with the plain and the block-preconditioned inner GMRES;
  // above them the block-preconditioned one was never slower than the plain)
  if (o.precond == IBRD_PRECOND_AUTO)
    o.precond = g->blobs.n <= (o.precision == IBRD_FP64 ? 2048 : 512) ? IBRD_PRECOND_DIAG : IBRD_PRECOND_BLOCK;
  // the block preconditioner's model is the Green's function of -chi L
  // (alpha = 0); with a shift the plain inner GMRES runs
  if (o.precond == IBRD_PRECOND_BLOCK && g->alpha != 0.0) o.precond = IBRD_PRECOND_SCHUR;
  return o;
}

void fill_info(ibrd_solve_info* info, const SolveResult& R, ibrd_grid g, double t0) {
  if (!info) return;
  info->status = R.st;
  info->outer_iters = R.iters;
  info->inner_iters = (int)g->inner;
  info->vcycles = (int)g->vcycles;
  info->reorths = (int)g->reorths;
  info->refinements = (int)g->refinements;
  info->rel_residual = R.rel;
  info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count() - t0;
}

// Runs solve(i) for every i in [0, count) on `threads` host threads, largest
// estimated work (cells plus a blob term) first so that the longest solves do
// not start last. Each solve orders its GPU work on its own handle's stream, so
// solves whose handles have distinct streams overlap on the device. Returns the
// first non-OK status in index order.
template <typename F>
ibrd_status run_batch(int count, const ibrd_grid* grids, int threads, F&& solve) {
  if (count < 0 || (count > 0 && !grids)) return IBRD_ERR_ARG;
  if (count == 0) return IBRD_OK;
  std::vector<ibrd_grid> seen(grids, grids + count);
  std::sort(seen.begin(), seen.end());
  for (int i = 0; i < count; ++i)
    if (!seen[i] || (i > 0 && seen[i] == seen[i - 1])) return IBRD_ERR_ARG;  // null or shared handle
  if (threads <= 0) threads = 16;
  threads = std::max(1, std::min(std::min(threads, 64), count));
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  auto cost = [&](int i) { return (double)grids[i]->d.n() + 512.0 * grids[i]->blobs.n; };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
  std::vector<ibrd_status> st(count, IBRD_OK);
  std::atomic<int> next{0};
  auto worker = [&]() {
    for (;;) {
      const int k = next.fetch_add(1, std::memory_order_relaxed);
      if (k >= count) return;
      st[order[k]] = solve(order[k]);
    }
  };
  std::vector<std::thread> pool;
  try {
    for (int t = 1; t < threads; ++t) pool.emplace_back(worker);
  } catch (...) {
    // fewer threads than asked: the calling thread and those started share the queue
  }
  worker();
  for (auto& th : pool) th.join();
  for (int i = 0; i < count; ++i)
    if (st[i] != IBRD_OK) return st[i];
  return IBRD_OK;
}

// ---------------------------------------------------------------- autotuner
// Shapes tuned in this process, by device, element size, kernel and grid.
struct TuneKey {
  int dev, elem, kind, nx, ny, nz;
  bool operator<(const TuneKey& o) const {
    return std::tie(dev, elem, kind, nx, ny, nz) < std::tie(o.dev, o.elem, o.kind, o.nx, o.ny, o.nz);
  }
};
struct TuneResult {
  SweepShape s;
  double us_default, us_tuned;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneResult> g_tune_cache;

// Average duration (us) of `reps` back-to-back sweeps with the handle's current
// shape for (elem, kind, d); the best of two timed runs after one warm-up.
// Consecutive sweeps alternate between two sets of fields (x in, x out, b),
// so that on levels larger than half the L2 each launch streams from DRAM as
// it does inside a V-cycle, while small levels stay L2-resident as they are
// there too.
template <typename T>
double time_sweep(ibrd_grid g, int kind, Dims d, Stencil st, T* const set[2][3], cudaEvent_t e0, cudaEvent_t e1,
                  int reps) {
  auto one = [&](int i) {
    T* const* f = set[i & 1];
    launch_rb_sweep<T>(f[0], f[1], f[2], nullptr, d, st, kind == TUNE_ZERO, nullptr, 0, g->s);
  };
  one(0);
  one(1);
  double best = 1e30;
  for (int r = 0; r < 2; ++r) {
    IBRD_CUDA(cudaEventRecord(e0, g->s));
    for (int i = 0; i < reps; ++i) one(i);
    IBRD_CUDA(cudaEventRecord(e1, g->s));
    IBRD_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    IBRD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    best = std::min(best, 1e3 * (double)ms / reps);
  }
  return best;
}

// Tunes the sweep kernels of element type T on the levels that run them.
template <typename T>
void autotune_levels(ibrd_grid g, bool retune, std::vector<ibrd_tune_entry>& rep) {
  const int elem = (int)sizeof(T);
  int end = g->small_from;
  if (elem == 4 && g->exact32 >= 0) end = g->exact32;
  end = std::min(end, (int)g->levels.size() - 1);
  if (end <= 0) return;
  const size_t n = g->d.n();
  // two sets of (x in, x out, b), each field n values (256-byte aligned)
  const size_t ld = (n + 63) / 64 * 64;
  T* buf = dalloc<T>(6 * ld);
  T* const set[2][3] = {{buf, buf + ld, buf + 2 * ld}, {buf + 3 * ld, buf + 4 * ld, buf + 5 * ld}};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto cleanup = [&]() {
    cudaFree(buf);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  try {
    IBRD_CUDA(cudaEventCreate(&e0));
    IBRD_CUDA(cudaEventCreate(&e1));
    IBRD_CUDA(cudaMemsetAsync(buf, 0, sizeof(T) * 6 * ld, g->s));
    for (int l = 0; l < end; ++l) {
      const Dims d = g->levels[l].d;
      const Stencil st = stencil(g->levels[l].h, g->chi, g->alpha > 0.0 ? g->alpha : 1.0);
      const int reps = 2 * (int)std::max(2.0, std::min(100.0, 1e8 / (3.0 * elem * (double)d.n())));
      for (int kind = TUNE_SWEEP; kind <= TUNE_ZERO; ++kind) {
        if (kind == TUNE_SWEEP && !rb_sweep_fused_ok<T>(d)) continue;
        if (kind == TUNE_ZERO && (elem != 4 || d.nx % 4 != 0)) continue;
        const TuneKey key{g->dev, elem, kind, d.nx, d.ny, d.nz};
        TuneResult res{};
        bool cached = false;
        if (!retune) {
          std::lock_guard<std::mutex> lk(g_tune_mu);
          auto it = g_tune_cache.find(key);
          if (it != g_tune_cache.end()) {
            res = it->second;
            cached = true;
          }
        }
        SweepShape* slot = g->tune.find(elem, kind, d);
        if (!slot) {
          g->tune.e.push_back(Tuning::Entry{elem, kind, d, SweepShape{}});
          slot = &g->tune.e.back().s;
        }
        if (!cached) {
          *slot = SweepShape{};
          res.us_default = time_sweep<T>(g, kind, d, st, set, e0, e1, reps);
          res.us_tuned = res.us_default;
          res.s = SweepShape{};
          std::vector<int> txs = {0};
          if (kind == TUNE_SWEEP) {
            txs = {32};
            if (elem == 4 && d.nx % 64 == 0) txs.push_back(64);
            if (elem == 4 && rows_sweep_ok(d)) txs.push_back(d.nx);
          }
          static const int zcs[] = {1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512};
          for (int tx : txs)
            for (int zc : zcs) {
              if (zc > d.nz || (kind == TUNE_SWEEP && zc < 2)) continue;
              *slot = SweepShape{tx, zc};
              const double us = time_sweep<T>(g, kind, d, st, set, e0, e1, reps);
              // a shape replaces the built-in one only when clearly faster
              if (us < res.us_tuned && us < 0.97 * res.us_default) {
                res.us_tuned = us;
                res.s = *slot;
              }
            }
          std::lock_guard<std::mutex> lk(g_tune_mu);
          g_tune_cache[key] = res;
        }
        // re-find: push_back above may have moved the entries
        *g->tune.find(elem, kind, d) = res.s;
        ibrd_tune_entry r{};
        r.nx = d.nx;
        r.ny = d.ny;
        r.nz = d.nz;
        r.elem_bytes = elem;
        r.kind = kind;
        r.tx = res.s.tx;
        r.zc = res.s.zc;
        r.us_default = res.us_default;
        r.us_tuned = res.us_tuned;
        r.cached = cached ? 1 : 0;
        rep.push_back(r);
      }
    }
  } catch (...) {
    cleanup();
    throw;
  }
  cleanup();
}

double now_s() { return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count(); }

// sum over all cells and N-vector reductions for the report
void report(ibrd_grid g, const double* c, const double* lam_or_null, const double* kappa, ibrd_solve_info* info) {
  if (!info) return;
  const size_t nc = g->d.n();
  const int N = g->blobs.n;
  launch_sum<double>(c, nc, g->partial, g->scal + S_TMP, 1.0 / (double)nc, g->s, g->ticket);
  if (lam_or_null) {
    launch_sum<double>(lam_or_null, N, g->partial, g->scal + S_TMP2, 1.0, g->s, g->ticket);
  } else if (N > 0) {
    launch_interp<double>(g->blobs, g->d, c, 1.0, g->nv[2], g->s);
    launch_dot(g->nv[2], kappa, N, g->partial, g->scal + S_TMP2, 1.0, g->s, g->ticket);
  }
  IBRD_CUDA(cudaMemcpyAsync(g->host, g->scal + S_TMP, sizeof(double) * 2, cudaMemcpyDeviceToHost, g->s));
  IBRD_CUDA(cudaStreamSynchronize(g->s));
  info->cbar = g->host[0];
  info->sum_lambda = N > 0 ? g->host[1] : 0.0;
  info->rate_K = (N > 0 && info->cbar != 0.0) ? info->sum_lambda / (N * info->cbar) : 0.0;
  info->a_L = info->rate_K / (4.0 * 3.14159265358979323846 * g->chi);
}

// ---------------------------------------------------------------- solve set-up and report
// Checks and set-up of a reaction-limited solve; returns the preconditioner's
// shift sigma (alpha, or sum(kappa) / V_Omega when alpha = 0, R5).
double reaction_setup(ibrd_grid g, const double* kappa, const double* rhs, double* c, const ibrd_solve_opts& o) {
  const int N = g->blobs.n;
  if (!rhs || !c || (N > 0 && !kappa)) throw ArgError{IBRD_ERR_ARG, "null pointer"};
  g->vcycles = 0;
  g->inner = 0;
  g->reorths = 0;
  g->refinements = 0;
  ensure_nvec(g, o.schur_inner);
  double sigma = g->alpha;
  if (N > 0) {
    IBRD_CUDA(cudaMemsetAsync(g->dflag, 0, sizeof(int), g->s));
    prof_begin(P_SETUP, g->s);
    k_check_rates<<<std::min(1024, (N + 255) / 256), 256, 0, g->s>>>(kappa, N, g->dflag);
    prof_end(P_SETUP, g->s, "check_rates");
    int flag = 0;
    IBRD_CUDA(cudaMemcpyAsync(&flag, g->dflag, sizeof(int), cudaMemcpyDeviceToHost, g->s));
    launch_sum<double>(kappa, N, g->partial, g->scal + S_TMP, 1.0, g->s, g->ticket);
    const double ksum = host_scalar(g, S_TMP);
    if (flag) throw ArgError{IBRD_ERR_NONFINITE, "kappa must be finite and >= 0"};
    if (g->alpha == 0.0) sigma = ksum / ((double)g->d.n() * g->h * g->h * g->h);
  }
  if (!(sigma > 0.0)) throw ArgError{IBRD_ERR_ARG, "steady reaction system needs some kappa > 0"};
  return sigma;
}

void reaction_report(ibrd_grid g, const double* kappa, double* c, SolveResult& R, ibrd_solve_info* info, double t0,
                     const History& hist) {
  if (info) info->history_len = hist.len;
  report(g, c, nullptr, kappa, info);
  if (take_wait_flag(g)) R.st = IBRD_ERR_TIMEOUT;
  fill_info(info, R, g, t0);
  if (info) info->precond = -1;
  if (R.st != IBRD_OK) g->err = std::string("ibrd_solve_reaction: ") + ibrd_status_string(R.st);
}

// Checks and set-up of a saddle-point solve: [g; f] into bs, the guess or the
// warm start into xs, gamma of the diagonal preconditioner. Returns whether
// the solve starts from zero.
bool saddle_setup(ibrd_grid g, const double* rhs, const double* f, double* c, double* lambda,
                  const ibrd_solve_opts& o) {
  const int N = g->blobs.n;
  if (N < 1) throw ArgError{IBRD_ERR_STATE, "saddle solve needs at least one blob"};
  if (!rhs || !c || !lambda) throw ArgError{IBRD_ERR_ARG, "null pointer"};
  g->vcycles = 0;
  g->inner = 0;
  g->reorths = 0;
  g->refinements = 0;
  ensure_nvec(g, o.schur_inner);
  const size_t nc = g->d.n();
  const size_t n = nc + N;
  if (g->xs_cap < n) {
    cudaFree(g->xs);
    cudaFree(g->bs);
    g->xs = g->bs = nullptr;
    g->xs = dalloc<double>(n);
    g->bs = dalloc<double>(n);
    g->xs_cap = n;
  }
  IBRD_CUDA(cudaMemcpyAsync(g->bs, rhs, sizeof(double) * nc, cudaMemcpyDeviceToDevice, g->s));
  if (f)
    IBRD_CUDA(cudaMemcpyAsync(g->bs + nc, f, sizeof(double) * N, cudaMemcpyDeviceToDevice, g->s));
  else
    IBRD_CUDA(cudaMemsetAsync(g->bs + nc, 0, sizeof(double) * N, g->s));
  if (o.use_guess) {
    IBRD_CUDA(cudaMemcpyAsync(g->xs, c, sizeof(double) * nc, cudaMemcpyDeviceToDevice, g->s));
    IBRD_CUDA(cudaMemcpyAsync(g->xs + nc, lambda, sizeof(double) * N, cudaMemcpyDeviceToDevice, g->s));
  }
  const bool warm = !o.use_guess && o.lambda_guess != IBRD_GUESS_NONE;
  if (warm) {
    if (o.lambda_guess == IBRD_GUESS_GIVEN)
      IBRD_CUDA(cudaMemcpyAsync(g->xs + nc, lambda, sizeof(double) * N, cudaMemcpyDeviceToDevice, g->s));
    if (o.lambda_guess == IBRD_GUESS_PENALTY)
      saddle_penalty_start(g, o, g->bs, g->xs);
    else if (o.precision == IBRD_FP64)
      saddle_warm_start<double>(g, o, g->bs, g->xs, o.lambda_guess, o.warm_cycles);
    else
      saddle_warm_start<float>(g, o, g->bs, g->xs, o.lambda_guess, o.warm_cycles);
  }
  if ((o.precond == IBRD_PRECOND_DIAG || o.precond == IBRD_PRECOND_BLOCK) && !g->gamma_valid) {
    // gamma's V-cycles are set-up, not part of this solve's count
    const long v = g->vcycles;
    g->gamma_diag = compute_gamma(g, o);
    g->gamma_valid = true;
    g->vcycles = v;
  }
  if (o.precond == IBRD_PRECOND_BLOCK) ensure_block(g, o);
  return !o.use_guess && !warm;
}

void saddle_report(ibrd_grid g, double* c, double* lambda, SolveResult& R, ibrd_solve_info* info, double t0,
                   const ibrd_solve_opts& o, const History& hist) {
  const size_t nc = g->d.n();
  const int N = g->blobs.n;
  if (info) info->history_len = hist.len;
  IBRD_CUDA(cudaMemcpyAsync(c, g->xs, sizeof(double) * nc, cudaMemcpyDeviceToDevice, g->s));
  IBRD_CUDA(cudaMemcpyAsync(lambda, g->xs + nc, sizeof(double) * N, cudaMemcpyDeviceToDevice, g->s));
  report(g, c, lambda, nullptr, info);
  if (take_wait_flag(g)) R.st = IBRD_ERR_TIMEOUT;
  fill_info(info, R, g, t0);
  if (info) info->precond = o.precond;
  if (R.st != IBRD_OK) g->err = std::string("ibrd_solve_saddle: ") + ibrd_status_string(R.st);
}

// ---------------------------------------------------------------- a batch as one graph
// Refinement-mode solves of many handles (opts.graphs == 2) recorded into ONE
// graph: after each problem's set-up (on the calling thread, in order), one
// capture session forks a capture stream per problem from an origin stream and
// records that problem's whole device-terminated solve on it, so the problems
// are independent branches of one graph, launched once. A batch of a given
// configuration runs its problems' host loops the first time (lazy
// allocations), builds the graph the second time and replays it afterwards.
struct BatchGraph {
  cudaGraphExec_t exec = nullptr;
  std::vector<ibrd_grid_s::SolveGraph> parts;  // launch counts of each problem's part
  std::vector<ibrd_grid> grids;
  int seen = 0;
};
std::mutex g_batch_mu;
std::map<std::string, BatchGraph> g_batch;
cudaStream_t g_batch_origin[64] = {};

void drop_batch_graphs_of(ibrd_grid g) {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  for (auto it = g_batch.begin(); it != g_batch.end();) {
    if (std::find(it->second.grids.begin(), it->second.grids.end(), g) != it->second.grids.end()) {
      if (it->second.exec) cudaGraphExecDestroy(it->second.exec);
      it = g_batch.erase(it);
    } else {
      ++it;
    }
  }
}

struct BatchItem {
  int kind;  // IBRD_SOLVE_REACTION or IBRD_SOLVE_SADDLE
  ibrd_grid g;
  const double* kappa;
  const double* rhs;
  const double* f;
  double* c;
  double* lambda;
  ibrd_solve_info* info;
  // set up by the batch
  ibrd_solve_opts o{};
  double t0 = 0.0;
  bool zero_start = true;
  size_t n = 0;
  const double* b = nullptr;
  double* x = nullptr;
  std::unique_ptr<LinOp<double>> op64;
  std::unique_ptr<LinOp<float>> op32;
  History hist;
  SolveResult R;
};

// Whether every item can run in a batch graph: refinement mode with
// opts.graphs == 2, one device, no per-launch timing.
bool batch_graph_eligible(const std::vector<BatchItem>& items, const ibrd_solve_opts* opts) {
  if (items.empty() || !opts || opts->graphs != 2) return false;
  const int dev = items[0].g->dev;
  for (const auto& it : items) {
    const int prec = opts->precision < 0 ? it.g->precision : opts->precision;
    if (prec != IBRD_MIXED_REFINE || it.g->dev != dev || it.g->prof.timing || opts->restart > 61 ||
        it.g->d.n() > (size_t(1) << 31))
      return false;
  }
  return true;
}

// Set-up of one item (as the single-problem entry points do before solving).
void batch_setup(BatchItem& it, const ibrd_solve_opts* opts) {
  ibrd_grid g = it.g;
  it.t0 = now_s();
  it.o = resolve_opts(g, opts);
  if (it.info) {
    it.hist.buf = it.info->residual_history;
    it.hist.cap = it.info->history_cap;
  }
  if (it.kind == IBRD_SOLVE_REACTION) {
    const double sigma = reaction_setup(g, it.kappa, it.rhs, it.c, it.o);
    it.op64.reset(new ReactionOp<double>(g, it.kappa, sigma, it.o));
    it.op32.reset(new ReactionOp<float>(g, it.kappa, sigma, it.o));
    it.b = it.rhs;
    it.x = it.c;
    it.n = g->d.n();
    it.zero_start = !it.o.use_guess;
  } else {
    it.zero_start = saddle_setup(g, it.rhs, it.f, it.c, it.lambda, it.o);
    it.op64.reset(new SaddleOp<double>(g, it.o, it.o.zeta, it.o.xi));
    it.op32.reset(new SaddleOp<float>(g, it.o, it.o.zeta, it.o.xi));
    it.b = g->bs;
    it.x = g->xs;
    it.n = g->d.n() + g->blobs.n;
  }
  if (g->ir_cap < it.n) {
    // the refinement's residual fields (refine allocates them on first use)
    cudaFree(g->ir_r);
    cudaFree(g->ir_r32);
    cudaFree(g->ir_d32);
    g->ir_r = nullptr;
    g->ir_r32 = g->ir_d32 = nullptr;
    g->ir_r = dalloc<double>(it.n);
    g->ir_r32 = dalloc<float>(it.n);
    g->ir_d32 = dalloc<float>(it.n);
    g->ir_cap = it.n;
  }
  ensure_krylov<float>(g, it.n, std::max(1, it.o.restart));
  ensure_graph_state(g);
}

void batch_report(BatchItem& it) {
  if (it.kind == IBRD_SOLVE_REACTION)
    reaction_report(it.g, it.kappa, it.c, it.R, it.info, it.t0, it.hist);
  else
    saddle_report(it.g, it.c, it.lambda, it.R, it.info, it.t0, it.o, it.hist);
}

// Returns false when the items must run the per-problem path instead (not
// eligible, or a set-up failed: nothing was launched for any item then).
// fn(i) for i in [0, count) on up to `threads` host threads (the calling one included)
template <typename F>
void parallel_for(int count, int threads, F&& fn) {
  if (threads <= 0) threads = 16;
  threads = std::max(1, std::min(std::min(threads, 64), count));
  std::atomic<int> next{0};
  auto worker = [&]() {
    for (;;) {
      const int i = next.fetch_add(1, std::memory_order_relaxed);
      if (i >= count) return;
      fn(i);
    }
  };
  std::vector<std::thread> pool;
  try {
    for (int t = 1; t < threads; ++t) pool.emplace_back(worker);
  } catch (...) {
  }
  worker();
  for (auto& th : pool) th.join();
}

bool batch_graph_solve(std::vector<BatchItem>& items, const ibrd_solve_opts* opts, std::vector<ibrd_status>& st,
                       int threads) {
  if (!batch_graph_eligible(items, opts)) return false;
  const int dev = items[0].g->dev;
  DeviceGuard dg(dev);
  // set-up of every problem (each with its host reads) on the worker threads
  std::atomic<bool> setup_ok{true};
  parallel_for((int)items.size(), threads, [&](int i) {
    BatchItem& it = items[i];
    DeviceGuard dgi(it.g->dev);
    ProfScope ps(&it.g->prof, &it.g->tune);
    try {
      batch_setup(it, opts);
    } catch (...) {
      setup_ok = false;
    }
  });
  if (!setup_ok) return false;
  std::string bkey;
  for (auto& it : items) {
    char hb[48];
    std::snprintf(hb, sizeof hb, "#%p#%d#", (void*)it.g, it.kind);
    bkey += hb + refine_graph_key(it.g, *it.op64, *it.op32, it.b, it.x, it.n, it.o, it.zero_start);
  }
  BatchGraph* B = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    if (g_batch.size() > 16 && !g_batch.count(bkey)) {
      for (auto& kv : g_batch)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
      g_batch.clear();
    }
    B = &g_batch[bkey];
  }
  if (!B->exec && B->seen == 0) {
    // first encounter: the host loops, concurrently on the problems' streams
    B->seen = 1;
    B->grids.clear();
    for (auto& it : items) B->grids.push_back(it.g);
    std::vector<ibrd_grid> gs;
    for (auto& it : items) gs.push_back(it.g);
    run_batch((int)items.size(), gs.data(), threads, [&](int i) {
      BatchItem& it = items[i];
      DeviceGuard dgi(it.g->dev);
      ProfScope ps(&it.g->prof, &it.g->tune);
      try {
        it.R = refine(it.g, *it.op64, *it.op32, it.b, it.x, it.n, it.o, it.zero_start, it.hist);
        batch_report(it);
        st[i] = it.R.st;
      } catch (const ArgError& e) {
        st[i] = fail(it.g, e.code, e.msg);
      } catch (const CudaError& e) {
        cudaGetLastError();
        st[i] = fail(it.g, IBRD_ERR_CUDA, std::string("batch solve: ") + e.what);
      }
      if (it.info) it.info->status = st[i];
      return st[i];
    });
    return true;
  }
  if (!g_batch_origin[dev & 63]) IBRD_CUDA(cudaStreamCreateWithFlags(&g_batch_origin[dev & 63], cudaStreamNonBlocking));
  cudaStream_t origin = g_batch_origin[dev & 63];
  std::vector<cudaEvent_t> evs(items.size() + 1, nullptr);
  auto cleanup_events = [&]() {
    for (auto e : evs)
      if (e) cudaEventDestroy(e);
  };
  for (auto& e : evs) IBRD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  try {
    if (!B->exec) {
      // build: every problem's solve on its own capture stream, forked from the origin
      B->parts.assign(items.size(), ibrd_grid_s::SolveGraph{});
      cudaGraph_t graph = nullptr;
      IBRD_CUDA(cudaStreamBeginCapture(origin, cudaStreamCaptureModeRelaxed));
      try {
        IBRD_CUDA(cudaEventRecord(evs[0], origin));
        for (size_t i = 0; i < items.size(); ++i) {
          BatchItem& it = items[i];
          ProfScope ps(&it.g->prof, &it.g->tune);
          cudaStream_t user = it.g->s;
          it.g->s = it.g->cap_stream;
          try {
            IBRD_CUDA(cudaStreamWaitEvent(it.g->s, evs[0], 0));
            capture_refine(it.g, *it.op64, *it.op32, it.b, it.x, it.n, it.o, it.zero_start, B->parts[i]);
            IBRD_CUDA(cudaEventRecord(evs[i + 1], it.g->s));
            IBRD_CUDA(cudaStreamWaitEvent(origin, evs[i + 1], 0));
          } catch (...) {
            it.g->s = user;
            throw;
          }
          it.g->s = user;
        }
      } catch (...) {
        cudaGraph_t dummy = nullptr;
        cudaStreamEndCapture(origin, &dummy);
        if (dummy) cudaGraphDestroy(dummy);
        throw;
      }
      IBRD_CUDA(cudaStreamEndCapture(origin, &graph));
      const cudaError_t ei = cudaGraphInstantiate(&B->exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ei != cudaSuccess) {
        B->exec = nullptr;
        throw CudaError{ei, "cudaGraphInstantiate (batch graph)"};
      }
    }
    // launch: after every problem's set-up on its stream; each stream then
    // waits for the graph
    for (size_t i = 0; i < items.size(); ++i) {
      BatchItem& it = items[i];
      set_graph_params(it.g, it.o);
      IBRD_CUDA(cudaEventRecord(evs[i + 1], it.g->s));
      IBRD_CUDA(cudaStreamWaitEvent(origin, evs[i + 1], 0));
    }
    IBRD_CUDA(cudaGraphLaunch(B->exec, origin));
    IBRD_CUDA(cudaEventRecord(evs[0], origin));
    for (auto& it : items) IBRD_CUDA(cudaStreamWaitEvent(it.g->s, evs[0], 0));
  } catch (...) {
    cleanup_events();
    throw;
  }
  cleanup_events();
  // each problem's state and report (host reads) on the worker threads
  parallel_for((int)items.size(), threads, [&](int i) {
    BatchItem& it = items[i];
    DeviceGuard dgi(it.g->dev);
    ProfScope ps(&it.g->prof, &it.g->tune);
    try {
      it.R = finish_refine_graph(it.g, B->parts[i], it.x, it.n, it.hist);
      batch_report(it);
      st[i] = it.R.st;
    } catch (const CudaError& e) {
      cudaGetLastError();
      st[i] = fail(it.g, IBRD_ERR_CUDA, std::string("batch solve: ") + e.what);
    }
    if (it.info) it.info->status = st[i];
  });
  return true;
}

bool batch_grids_ok(int count, const ibrd_grid* grids) {
  if (!grids) return false;
  std::vector<ibrd_grid> seen(grids, grids + count);
  std::sort(seen.begin(), seen.end());
  for (int i = 0; i < count; ++i)
    if (!seen[i] || (i > 0 && seen[i] == seen[i - 1])) return false;
  return true;
}

ibrd_status first_failure(const std::vector<ibrd_status>& st) {
  for (auto v : st)
    if (v != IBRD_OK) return v;
  return IBRD_OK;
}

}  // namespace
}  // namespace ibrd

// ================================================================ C ABI
extern "C" {

void ibrd_default_opts(ibrd_solve_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tol = 1e-8;
  o->max_iter = 1000;
  o->restart = 30;
  o->mg_cycles = 1;
  o->schur_inner = 5;
  o->precond = IBRD_PRECOND_AUTO;
  o->zeta = 1.0;
  o->xi = 0.0;
  o->nu1 = 2;
  o->nu2 = 2;
  o->precision = -1;
  o->use_guess = 0;
  o->reorth_eta = 0.70710678118654752;
  o->graphs = 1;
  o->inner_tol = 1e-4;
  o->lambda_guess = IBRD_GUESS_NONE;
  o->warm_cycles = 2;
  o->penalty_kappa = 1000.0;
  o->penalty_tol = 1e-2;
  o->block_cutoff = 0.0;
}

const char* ibrd_status_string(int st) {
  switch (st) {
    case IBRD_OK: return "IBRD_OK";
    case IBRD_ERR_ARG: return "IBRD_ERR_ARG";
    case IBRD_ERR_CUDA: return "IBRD_ERR_CUDA";
    case IBRD_ERR_OOM: return "IBRD_ERR_OOM";
    case IBRD_ERR_NOT_CONVERGED: return "IBRD_ERR_NOT_CONVERGED";
    case IBRD_ERR_BREAKDOWN: return "IBRD_ERR_BREAKDOWN";
    case IBRD_ERR_NONFINITE: return "IBRD_ERR_NONFINITE";
    case IBRD_ERR_TIMEOUT: return "IBRD_ERR_TIMEOUT";
    case IBRD_ERR_STATE: return "IBRD_ERR_STATE";
    default: return "IBRD_UNKNOWN";
  }
}

const char* ibrd_last_error(ibrd_grid g) { return g ? g->err.c_str() : "null handle"; }

void ibrd_grid_destroy(ibrd_grid g) {
  if (!g) return;
  DeviceGuard dg(g->dev);
  auto F = [](void* p) { if (p) cudaFree(p); };
  for (auto p : g->h64.x) F(p);
  for (auto p : g->h64.b) F(p);
  for (auto p : g->h64.y) F(p);
  for (auto p : g->h32.x) F(p);
  for (auto p : g->h32.b) F(p);
  for (auto p : g->h32.y) F(p);
  for (auto& e : g->h64.tables) F(e.second);
  for (auto& e : g->h32.tables) F(e.second);
  for (auto& e : g->h32.hartley) F(e.second);
  BlobSet& b = g->blobs;
  F(b.q); F(b.idx); F(b.w64); F(b.w32); F(b.tile_count); F(b.tile_offset); F(b.tile_cursor); F(b.tile_blobs);
  F(b.active); F(b.d_meta); F(b.cell_count); F(b.cell_offset); F(b.cells); F(b.cell_tile);
  F(g->scal); F(g->partial); F(g->dflag); F(g->ticket); F(g->gst); F(g->ghist);
  if (g->host) cudaFreeHost(g->host);
  F(g->V); F(g->Z); F(g->H); F(g->cs); F(g->sn); F(g->gvec); F(g->yv); F(g->hb2); F(g->vsc); F(g->xs); F(g->bs);
  F(g->ir_r); F(g->ir_r32); F(g->ir_d32);
  for (auto p : g->p64) F(p);
  for (auto p : g->p32) F(p);
  for (auto p : g->nv) F(p);
  F(g->U); F(g->Hs); F(g->scs); F(g->ssn); F(g->sg);
  F(g->blk_idx); F(g->blk_cnt); F(g->blk_val); F(g->blk_pos);
  for (auto e : g->prof.pool) cudaEventDestroy(e);
  drop_batch_graphs_of(g);
  free_graphs(g);
  if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
  for (auto st : g->cap_pool) cudaStreamDestroy(st);
  delete g;
}

ibrd_status ibrd_grid_create(ibrd_grid* out, int nx, int ny, int nz, double h, double chi, double alpha, int kernel,
                             int precision, void* stream) {
  if (!out) return IBRD_ERR_ARG;
  *out = nullptr;
  if (nx < 4 || ny < 4 || nz < 4 || !(h > 0.0) || !(chi > 0.0) || !(alpha >= 0.0) || !std::isfinite(h) ||
      !std::isfinite(chi) || !std::isfinite(alpha) || (kernel != IBRD_PESKIN4 && kernel != IBRD_PESKIN3) ||
      (precision != IBRD_FP64 && precision != IBRD_MIXED_FP32 && precision != IBRD_MIXED_REFINE))
    return IBRD_ERR_ARG;
  if ((double)nx * ny * nz > 4.0e9) return IBRD_ERR_ARG;
  ibrd_grid g = new (std::nothrow) ibrd_grid_s();
  if (!g) return IBRD_ERR_OOM;
  cudaGetDevice(&g->dev);
  g->d = Dims{nx, ny, nz};
  g->h = h;
  g->chi = chi;
  g->alpha = alpha;
  g->kernel = kernel;
  g->precision = precision;
  g->s = (cudaStream_t)stream;
  g->blobs.width = kernel;
  // multigrid levels: halve while every side is even and >= 4
  g->levels.push_back(Level{g->d, h});
  while (true) {
    const Level& l = g->levels.back();
    if (l.d.nx % 2 == 0 && l.d.ny % 2 == 0 && l.d.nz % 2 == 0 && l.d.nx >= 4 && l.d.ny >= 4 && l.d.nz >= 4)
      g->levels.push_back(Level{Dims{l.d.nx / 2, l.d.ny / 2, l.d.nz / 2}, 2.0 * l.h});
    else
      break;
  }
  if (g->levels.back().d.n() > 512 || g->levels.size() > 16) {
    delete g;
    return IBRD_ERR_ARG;
  }
  // single-CTA coarse V-cycle from the first level whose remaining hierarchy
  // (x and b, FP64) fits in 160 KB of shared memory and has at most 12 levels
  {
    const int L = (int)g->levels.size();
    g->small_from = L;
    size_t cells = 0;
    for (int l = L - 1; l >= 0; --l) {
      cells += g->levels[l].d.n();
      if (2 * 8 * cells <= 160 * 1024 && L - l <= kMaxSmallLevels)
        g->small_from = l;
      else
        break;
    }
  }
  // FP32 V-cycles end at the first level of at most 32768 cells with no side
  // above 64, solved exactly (the FP64 V-cycles coarsen to the end)
  for (int l = 0; l < (int)g->levels.size(); ++l)
    if (hartley_ok(g->levels[l].d)) {
      g->exact32 = l;
      break;
    }
  ibrd_status st = guarded(g, "ibrd_grid_create", [&]() {
    g->scal = dalloc<double>(S_COUNT);
    g->partial = dalloc<double>((size_t)kRedBlocks * kDotGroup);
    g->dflag = dalloc<int>(4);
    IBRD_CUDA(cudaMemsetAsync(g->dflag, 0, sizeof(int) * 4, g->s));
    g->ticket = dalloc<unsigned>(1);
    IBRD_CUDA(cudaMemsetAsync(g->ticket, 0, sizeof(unsigned), g->s));
    g->tune.wait_err = reinterpret_cast<int*>(g->scal + S_WAIT);
    IBRD_CUDA(cudaMallocHost(&g->host, sizeof(double) * 64));
    IBRD_CUDA(cudaMemsetAsync(g->scal, 0, sizeof(double) * S_COUNT, g->s));
    blobs_setup(g->blobs, g->d, g->h, nullptr, 0, g->s);
    return IBRD_OK;
  });
  if (st != IBRD_OK) {
    ibrd_grid_destroy(g);
    return st;
  }
  *out = g;
  return IBRD_OK;
}

ibrd_status ibrd_set_blobs(ibrd_grid g, const double* q, int n) {
  return guarded(g, "ibrd_set_blobs", [&]() {
    if (n < 0 || (n > 0 && !q)) throw ArgError{IBRD_ERR_ARG, "bad blob array"};
    IBRD_CUDA(cudaMemsetAsync(g->dflag, 0, sizeof(int), g->s));
    if (n > 0) launch_nonfinite<double>(q, (size_t)3 * n, g->dflag, g->s);
    int flag = 0;
    IBRD_CUDA(cudaMemcpyAsync(&flag, g->dflag, sizeof(int), cudaMemcpyDeviceToHost, g->s));
    IBRD_CUDA(cudaStreamSynchronize(g->s));
    if (flag) throw ArgError{IBRD_ERR_NONFINITE, "non-finite blob position"};
    blobs_setup(g->blobs, g->d, g->h, q, n, g->s);
    g->blob_version++;
    return IBRD_OK;
  });
}

ibrd_status ibrd_apply_L(ibrd_grid g, const double* c, double* y) {
  return guarded(g, "ibrd_apply_L", [&]() {
    if (!c || !y || c == y) throw ArgError{IBRD_ERR_ARG, "null or aliased field"};
    launch_apply_A<double>(c, y, g->d, stencil(g->h, g->chi, g->alpha), g->s);
    return IBRD_OK;
  });
}

double ibrd_periodic_constant(double lx, double ly, double lz) {
  if (!(lx > 0.0 && ly > 0.0 && lz > 0.0) || !std::isfinite(lx * ly * lz)) return std::nan("");
  return periodic_constant(lx, ly, lz);
}

ibrd_status ibrd_residual(ibrd_grid g, const double* rhs, const double* c, double* r) {
  return guarded(g, "ibrd_residual", [&]() {
    if (!rhs || !c || !r || c == r || rhs == r) throw ArgError{IBRD_ERR_ARG, "null or aliased field"};
    launch_residual<double>(c, rhs, r, g->d, stencil(g->h, g->chi, g->alpha), g->scal + S_XMAX, g->s);
    return IBRD_OK;
  });
}

ibrd_status ibrd_vcycle(ibrd_grid g, const double* rhs, double* x, int zero) {
  return guarded(g, "ibrd_vcycle", [&]() {
    if (!rhs || !x || rhs == x) throw ArgError{IBRD_ERR_ARG, "null or aliased field"};
    vcycle<double>(g, rhs, x, zero != 0, g->alpha, 2, 2);
    check_waits_if_not_capturing(g, "V-cycle");
    return IBRD_OK;
  });
}

ibrd_status ibrd_vcycle_f32(ibrd_grid g, const float* rhs, float* x, int zero) {
  return guarded(g, "ibrd_vcycle_f32", [&]() {
    if (!rhs || !x || rhs == x) throw ArgError{IBRD_ERR_ARG, "null or aliased field"};
    vcycle<float>(g, rhs, x, zero != 0, g->alpha, 2, 2);
    check_waits_if_not_capturing(g, "V-cycle");
    return IBRD_OK;
  });
}

ibrd_status ibrd_vcycle_f32_sweeps(ibrd_grid g, const float* rhs, float* x, int zero, int nu1, int nu2) {
  return guarded(g, "ibrd_vcycle_f32_sweeps", [&]() {
    if (!rhs || !x || rhs == x) throw ArgError{IBRD_ERR_ARG, "null or aliased field"};
    if (nu1 < 0 || nu2 < 0 || nu1 > 16 || nu2 > 16) throw ArgError{IBRD_ERR_ARG, "bad sweep counts"};
    vcycle<float>(g, rhs, x, zero != 0, g->alpha, nu1, nu2);
    check_waits_if_not_capturing(g, "V-cycle");
    return IBRD_OK;
  });
}

ibrd_status ibrd_spread(ibrd_grid g, const double* lam, double* out, int accumulate) {
  return guarded(g, "ibrd_spread", [&]() {
    if (!out || (g->blobs.n > 0 && !lam)) throw ArgError{IBRD_ERR_ARG, "null pointer"};
    launch_spread<double>(g->blobs, g->d, lam, nullptr, inv_h3(g), out, accumulate, g->s);
    return IBRD_OK;
  });
}

ibrd_status ibrd_interp(ibrd_grid g, const double* c, double* out) {
  return guarded(g, "ibrd_interp", [&]() {
    if (!c || (g->blobs.n > 0 && !out)) throw ArgError{IBRD_ERR_ARG, "null pointer"};
    launch_interp<double>(g->blobs, g->d, c, 1.0, out, g->s);
    return IBRD_OK;
  });
}

ibrd_status ibrd_solve_reaction(ibrd_grid g, const double* kappa, const double* rhs, double* c,
                                const ibrd_solve_opts* opts, ibrd_solve_info* info) {
  return guarded(g, "ibrd_solve_reaction", [&]() {
    const double t0 = now_s();
    const ibrd_solve_opts o = resolve_opts(g, opts);
    const double sigma = reaction_setup(g, kappa, rhs, c, o);
    SolveResult R;
    History hist;
    if (info) {
      hist.buf = info->residual_history;
      hist.cap = info->history_cap;
    }
    if (o.precision == IBRD_FP64) {
      ReactionOp<double> op(g, kappa, sigma, o);
      R = fgmres<double>(g, op, rhs, c, g->d.n(), o, o.tol, o.max_iter, !o.use_guess, hist);
    } else if (o.precision == IBRD_MIXED_FP32) {
      ReactionOp<float, double> op(g, kappa, sigma, o);
      R = fgmres<double>(g, op, rhs, c, g->d.n(), o, o.tol, o.max_iter, !o.use_guess, hist);
    } else {
      ReactionOp<double> op(g, kappa, sigma, o);
      ReactionOp<float> op32(g, kappa, sigma, o);
      R = run_refine(g, op, op32, rhs, c, g->d.n(), o, !o.use_guess, hist);
    }
    reaction_report(g, kappa, c, R, info, t0, hist);
    return R.st;
  });
}

ibrd_status ibrd_solve_saddle(ibrd_grid g, const double* rhs, const double* f, double* c, double* lambda,
                              const ibrd_solve_opts* opts, ibrd_solve_info* info) {
  return guarded(g, "ibrd_solve_saddle", [&]() {
    const double t0 = now_s();
    const ibrd_solve_opts o = resolve_opts(g, opts);
    const bool zero_start = saddle_setup(g, rhs, f, c, lambda, o);
    const size_t n = g->d.n() + g->blobs.n;
    SolveResult R;
    History hist;
    if (info) {
      hist.buf = info->residual_history;
      hist.cap = info->history_cap;
    }
    if (o.precision == IBRD_FP64) {
      SaddleOp<double> op(g, o, o.zeta, o.xi);
      R = fgmres<double>(g, op, g->bs, g->xs, n, o, o.tol, o.max_iter, zero_start, hist);
    } else if (o.precision == IBRD_MIXED_FP32) {
      SaddleOp<float, double> op(g, o, o.zeta, o.xi);
      R = fgmres<double>(g, op, g->bs, g->xs, n, o, o.tol, o.max_iter, zero_start, hist);
    } else {
      SaddleOp<double> op(g, o, o.zeta, o.xi);
      SaddleOp<float> op32(g, o, o.zeta, o.xi);
      R = run_refine(g, op, op32, g->bs, g->xs, n, o, zero_start, hist);
    }
    saddle_report(g, c, lambda, R, info, t0, o, hist);
    return R.st;
  });
}

ibrd_status ibrd_solve_reaction_batch(int count, const ibrd_grid* grids, const double* const* kappa,
                                      const double* const* rhs, double* const* c, const ibrd_solve_opts* opts,
                                      ibrd_solve_info* infos, int threads) {
  if (count > 0 && (!kappa || !rhs || !c)) return IBRD_ERR_ARG;
  if (opts && opts->graphs == 2 && count > 0 && batch_grids_ok(count, grids)) {
    std::vector<BatchItem> items((size_t)count);
    for (int i = 0; i < count; ++i)
      items[i] = BatchItem{IBRD_SOLVE_REACTION, grids[i], kappa[i], rhs[i], nullptr, c[i], nullptr,
                           infos ? infos + i : nullptr};
    std::vector<ibrd_status> st((size_t)count, IBRD_OK);
    try {
      if (batch_graph_solve(items, opts, st, threads)) return first_failure(st);
    } catch (const CudaError& e) {
      cudaGetLastError();
      return fail(grids[0], IBRD_ERR_CUDA, std::string("ibrd_solve_reaction_batch: ") + e.what);
    }
  }
  return run_batch(count, grids, threads, [&](int i) {
    ibrd_solve_info* info = infos ? infos + i : nullptr;
    const ibrd_status st = ibrd_solve_reaction(grids[i], kappa[i], rhs[i], c[i], opts, info);
    if (info) info->status = st;
    return st;
  });
}

ibrd_status ibrd_solve_saddle_batch(int count, const ibrd_grid* grids, const double* const* rhs,
                                    const double* const* f, double* const* c, double* const* lambda,
                                    const ibrd_solve_opts* opts, ibrd_solve_info* infos, int threads) {
  if (count > 0 && (!rhs || !c || !lambda)) return IBRD_ERR_ARG;
  if (opts && opts->graphs == 2 && count > 0 && batch_grids_ok(count, grids)) {
    std::vector<BatchItem> items((size_t)count);
    for (int i = 0; i < count; ++i)
      items[i] = BatchItem{IBRD_SOLVE_SADDLE, grids[i], nullptr, rhs[i], f ? f[i] : nullptr, c[i], lambda[i],
                           infos ? infos + i : nullptr};
    std::vector<ibrd_status> st((size_t)count, IBRD_OK);
    try {
      if (batch_graph_solve(items, opts, st, threads)) return first_failure(st);
    } catch (const CudaError& e) {
      cudaGetLastError();
      return fail(grids[0], IBRD_ERR_CUDA, std::string("ibrd_solve_saddle_batch: ") + e.what);
    }
  }
  return run_batch(count, grids, threads, [&](int i) {
    ibrd_solve_info* info = infos ? infos + i : nullptr;
    const ibrd_status st = ibrd_solve_saddle(grids[i], rhs[i], f ? f[i] : nullptr, c[i], lambda[i], opts, info);
    if (info) info->status = st;
    return st;
  });
}

ibrd_status ibrd_solve_many(int count, const ibrd_solve_item* items, int threads) {
  if (count < 0 || (count > 0 && !items)) return IBRD_ERR_ARG;
  std::vector<ibrd_grid> grids((size_t)count);
  for (int i = 0; i < count; ++i) {
    if (items[i].kind != IBRD_SOLVE_REACTION && items[i].kind != IBRD_SOLVE_SADDLE) return IBRD_ERR_ARG;
    grids[i] = items[i].grid;
  }
  return run_batch(count, grids.data(), threads, [&](int i) {
    const ibrd_solve_item& it = items[i];
    ibrd_status st = it.q ? ibrd_set_blobs(it.grid, it.q, it.n_blobs) : IBRD_OK;
    if (st == IBRD_OK)
      st = it.kind == IBRD_SOLVE_REACTION
               ? ibrd_solve_reaction(it.grid, it.kappa, it.rhs, it.c, it.opts, it.info)
               : ibrd_solve_saddle(it.grid, it.rhs, it.f, it.c, it.lambda, it.opts, it.info);
    if (st == IBRD_OK && (it.c_host || it.lambda_host)) {
      st = guarded(it.grid, "ibrd_solve_many", [&]() {
        ibrd_grid g = it.grid;
        if (it.c_host)
          IBRD_CUDA(cudaMemcpyAsync(it.c_host, it.c, sizeof(double) * g->d.n(), cudaMemcpyDeviceToHost, g->s));
        if (it.lambda_host && it.kind == IBRD_SOLVE_SADDLE && g->blobs.n > 0)
          IBRD_CUDA(cudaMemcpyAsync(it.lambda_host, it.lambda, sizeof(double) * g->blobs.n,
                                    cudaMemcpyDeviceToHost, g->s));
        IBRD_CUDA(cudaStreamSynchronize(g->s));
        return IBRD_OK;
      });
    }
    if (it.info) it.info->status = st;
    return st;
  });
}

ibrd_status ibrd_autotune(ibrd_grid g, int precision, int retune, ibrd_tune_entry* out, int cap, int* n_out) {
  return guarded(g, "ibrd_autotune", [&]() {
    if (precision != -1 && precision != IBRD_FP64 && precision != IBRD_MIXED_FP32 &&
        precision != IBRD_MIXED_REFINE)
      throw ArgError{IBRD_ERR_ARG, "bad precision"};
    if (cap < 0 || (cap > 0 && !out)) throw ArgError{IBRD_ERR_ARG, "bad report array"};
    std::vector<ibrd_tune_entry> rep;
    free_graphs(g);  // captured launches would keep the old shapes
    if (precision != IBRD_FP64) autotune_levels<float>(g, retune != 0, rep);
    if (precision == IBRD_FP64 || precision == -1) autotune_levels<double>(g, retune != 0, rep);
    IBRD_CUDA(cudaStreamSynchronize(g->s));
    for (int i = 0; i < (int)rep.size() && i < cap; ++i) out[i] = rep[i];
    if (n_out) *n_out = (int)rep.size();
    return IBRD_OK;
  });
}

ibrd_status ibrd_tune_set(ibrd_grid g, int elem_bytes, int kind, int nx, int ny, int nz, int tx, int zc) {
  return guarded(g, "ibrd_tune_set", [&]() {
    const bool rows = elem_bytes == 4 && kind == TUNE_SWEEP && tx == nx && rows_sweep_ok(Dims{nx, ny, nz});
    const bool pro = kind == TUNE_PROLONG;
    if ((elem_bytes != 4 && elem_bytes != 8) || (kind != TUNE_SWEEP && kind != TUNE_ZERO && !pro) || zc < 0 ||
        (!pro && tx != 0 && tx != 32 && tx != 64 && !rows) || (kind == TUNE_ZERO && tx != 0) ||
        (elem_bytes == 8 && tx == 64) || (pro && (elem_bytes != 4 || (tx != 0 && tx != 1) || zc != 0)))
      throw ArgError{IBRD_ERR_ARG, "bad launch shape"};
    bool level = false;
    for (const Level& l : g->levels) level |= (l.d.nx == nx && l.d.ny == ny && l.d.nz == nz);
    if (!level) throw ArgError{IBRD_ERR_ARG, "no multigrid level of that size"};
    const Dims d{nx, ny, nz};
    free_graphs(g);
    SweepShape* slot = g->tune.find(elem_bytes, kind, d);
    if (!slot) {
      g->tune.e.push_back(Tuning::Entry{elem_bytes, kind, d, SweepShape{}});
      slot = &g->tune.e.back().s;
    }
    *slot = SweepShape{tx, zc};
    return IBRD_OK;
  });
}

ibrd_status ibrd_set_wait_limit(ibrd_grid g, unsigned tries) {
  return guarded(g, "ibrd_set_wait_limit", [&]() {
    free_graphs(g);  // captured launches carry the old bound
    g->tune.wait_limit = tries;
    return IBRD_OK;
  });
}

ibrd_status ibrd_tune_clear(ibrd_grid g) {
  return guarded(g, "ibrd_tune_clear", [&]() {
    free_graphs(g);
    g->tune.e.clear();
    return IBRD_OK;
  });
}

static const char* kProfNames[P_NCLASS] = {
    "apply_f64",    "apply_f32",    "rbgs_f64",   "rbgs_f32",   "restrict_f64", "restrict_f32", "prolong_f64",
    "prolong_f32",  "coarse",       "spread_f64", "spread_f32", "interp_f64",   "interp_f32",   "dot",
    "axpy",         "reduce",       "vector",     "small",      "setup"};

const char* ibrd_profile_class_name(int cls) { return (cls >= 0 && cls < P_NCLASS) ? kProfNames[cls] : ""; }

ibrd_status ibrd_profile_enable(ibrd_grid g, unsigned class_mask, double min_bytes) {
  return guarded(g, "ibrd_profile_enable", [&]() {
    g->prof.timing = class_mask != 0;
    g->prof.mask = class_mask;
    g->prof.min_bytes = min_bytes;
    return IBRD_OK;
  });
}

ibrd_status ibrd_profile_read(ibrd_grid g, ibrd_profile* out, int reset) {
  return guarded(g, "ibrd_profile_read", [&]() {
    if (!out) throw ArgError{IBRD_ERR_ARG, "null output"};
    Profiler& p = g->prof;
    IBRD_CUDA(cudaStreamSynchronize(g->s));
    std::memset(out, 0, sizeof(*out));
    out->launches = p.launches;
    out->nclass = P_NCLASS;
    out->overflow = p.overflow ? 1 : 0;
    for (int c = 0; c < P_NCLASS; ++c) {
      out->count[c] = p.count[c];
      out->bytes[c] = p.bytes[c];
      out->max_launch_bytes[c] = p.max_bytes[c];
    }
    for (size_t i = 0; i < p.pending.size(); ++i) {
      const auto& e = p.pending[i];
      float ms = 0.f;
      IBRD_CUDA(cudaEventElapsedTime(&ms, p.pool[e.second], p.pool[e.second + 1]));
      out->ms[e.first] += ms;
      out->timed[e.first] += 1;
      out->timed_bytes[e.first] += p.pending_bytes[i];
    }
    if (reset) {
      p.launches = 0;
      for (auto& c : p.count) c = 0;
      for (auto& b : p.bytes) b = 0.0;
      for (auto& b : p.max_bytes) b = 0.0;
      p.pending.clear();
      p.pending_bytes.clear();
      p.used = 0;
      p.overflow = false;
    }
    return IBRD_OK;
  });
}

}  // extern "C"
