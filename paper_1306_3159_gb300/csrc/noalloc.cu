// ibrd_vcycle_noalloc: the FP64 multigrid V-cycle of ibrd_vcycle for callers
// that cannot allocate device memory.
//
// Some callers must not call cudaMalloc: code that runs while a memory pool
// is locked down (a host allocator that forbids growth after start-up, a
// real-time loop whose memory budget is fixed once), code inside a library
// that may only use memory handed to it, or a process whose device memory is
// already taken by a framework's caching allocator. ibrd_vcycle needs a grid
// handle, and the handle allocates its multigrid workspaces. This entry point
// needs no handle: every workspace of the V-cycle (the coarse levels, the
// smoothing ping-pong field, the coarsest-level Green's table, reduction
// partials and scalars) is carved out of one file-scope device array of fixed
// size, which every GPU that loads the library holds until the process exits.
//
// The computation is the one ibrd_vcycle performs (same kernels, same
// definition); only where the scratch lives differs.
#include <cmath>
#include <mutex>
#include <new>
#include <vector>

#include "internal.h"

namespace ibrd {
namespace {

// Largest scratch this entry point may use: 16 MiB (enough for grids of about
// 1.4 million cells, e.g. 96^3 or 112^3).
constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;

// The scratch itself. In host code this name is only a stand-in for the
// device array; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per
// device (with that device current) on the first call that runs there. With
// CUDA's lazy module loading (the default) that lookup is also what loads
// this file's module on the device and so reserves the array there; the
// address is cached for the process, so a cudaDeviceReset, which unloads the
// module, makes later calls on that device invalid.
cudaError_t scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

struct NaLevel {
  Dims d;
  double h;
};

// The same hierarchy rules as a grid handle: halve while every side is even
// and >= 4; the coarse end runs in one CTA from the first level whose
// remaining levels (x and b, FP64) fit in 160 KB of shared memory.
struct NaPlan {
  std::vector<NaLevel> lv;
  int small_from = 0;
  // scratch layout, in doubles
  size_t partial = 0, scal = 0, table = 0, total = 0;
  std::vector<size_t> x, b, y;
};

bool make_plan(int nx, int ny, int nz, double h, NaPlan& P) {
  P.lv.push_back(NaLevel{Dims{nx, ny, nz}, h});
  while (true) {
    const NaLevel& l = P.lv.back();
    if (l.d.nx % 2 == 0 && l.d.ny % 2 == 0 && l.d.nz % 2 == 0 && l.d.nx >= 4 && l.d.ny >= 4 && l.d.nz >= 4)
      P.lv.push_back(NaLevel{Dims{l.d.nx / 2, l.d.ny / 2, l.d.nz / 2}, 2.0 * l.h});
    else
      break;
  }
  const int L = (int)P.lv.size();
  if (P.lv.back().d.n() > 512 || L > 16) return false;
  P.small_from = L;
  size_t cells = 0;
  for (int l = L - 1; l >= 0; --l) {
    cells += P.lv[l].d.n();
    if (2 * 8 * cells <= 160 * 1024 && L - l <= kMaxSmallLevels)
      P.small_from = l;
    else
      break;
  }
  size_t off = 0;
  auto take = [&](size_t n) {
    const size_t o = off;
    off += (n + 31) & ~size_t(31);  // keep 256-byte alignment
    return o;
  };
  P.partial = take(kRedBlocks);
  P.scal = take(8);
  P.table = take(P.lv.back().d.n());
  P.x.assign(L, 0);
  P.b.assign(L, 0);
  P.y.assign(L, 0);
  for (int l = 0; l < L; ++l) {
    if (l > 0) {
      P.x[l] = take(P.lv[l].d.n());
      P.b[l] = take(P.lv[l].d.n());
    }
    if (l + 1 < L && l < P.small_from) P.y[l] = take(P.lv[l].d.n());
  }
  P.total = off;
  return true;
}

Stencil na_stencil(double h, double chi, double shift) {
  const double off = chi / (h * h);
  return Stencil{shift + 6.0 * off, off};
}

// One V-cycle on level l, as in the handle's driver, with scratch fields.
void na_level(const NaPlan& P, double* S, int l, const double* b, const double* bshift, double* x, bool zero,
              double chi, double shift, cudaStream_t s) {
  const NaLevel& lv = P.lv[l];
  const Stencil st = na_stencil(lv.h, chi, shift);
  const int L = (int)P.lv.size();
  const double* table = S + P.table;
  if (l == L - 1) {
    launch_coarse_solve<double>(table, b, x, lv.d, s);
    return;
  }
  if (l >= P.small_from) {
    CoarseLevels cl{};
    cl.n = L - l;
    int tot = 0;
    for (int i = 0; i < cl.n; ++i) {
      const NaLevel& li = P.lv[l + i];
      const Stencil si = na_stencil(li.h, chi, shift);
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
    launch_vcycle_small<double>(cl, b, x, bshift, table, zero, 2, 2, s);
    return;
  }
  double* cur = x;
  double* oth = S + P.y[l];
  double* bc = S + P.b[l + 1];
  double* xc = S + P.x[l + 1];
  bool first = zero;
  for (int sweep = 0; sweep < 2; ++sweep) {
    if (launch_rb_sweep<double>(cur, oth, b, bshift, lv.d, st, first, nullptr, 0, s) >= 0) std::swap(cur, oth);
    first = false;
  }
  launch_resid_restrict<double>(cur, b, bshift, bc, lv.d, st, s);
  na_level(P, S, l + 1, bc, nullptr, xc, true, chi, shift, s);
  launch_prolong8<double>(xc, cur, lv.d, s);
  for (int sweep = 0; sweep < 2; ++sweep)
    if (launch_rb_sweep<double>(cur, oth, b, bshift, lv.d, st, false, nullptr, 0, s) >= 0) std::swap(cur, oth);
  if (cur != x) IBRD_CUDA(cudaMemcpyAsync(x, cur, sizeof(double) * lv.d.n(), cudaMemcpyDeviceToDevice, s));
}

}  // namespace
}  // namespace ibrd

using namespace ibrd;

namespace {
ibrd_status cuda_status(cudaError_t e) {
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? IBRD_ERR_OOM : IBRD_ERR_CUDA;
}
}  // namespace

extern "C" ibrd_status ibrd_vcycle_noalloc(int nx, int ny, int nz, double h, double chi, double alpha,
                                           const double* rhs, double* x, int zero_initial_guess, void* stream) {
  if (nx < 4 || ny < 4 || nz < 4 || !(h > 0.0) || !(chi > 0.0) || !(alpha >= 0.0) || !std::isfinite(h) ||
      !std::isfinite(chi) || !std::isfinite(alpha))
    return IBRD_ERR_ARG;
  // no exception leaves this function: host-side failures (the plan's small
  // host vectors) and CUDA errors become status codes
  try {
  NaPlan P;
  if (!make_plan(nx, ny, nz, h, P)) return IBRD_ERR_ARG;
  if (P.total * sizeof(double) > kNoAllocScratchBytes) return IBRD_ERR_ARG;  // grid too large for the scratch
  if (!rhs || !x || rhs == x) return IBRD_ERR_ARG;
  void* base = nullptr;
  const cudaError_t ea = scratch_address(&base);
  if (ea != cudaSuccess) return cuda_status(ea);
  double* S = static_cast<double*>(base);
  const cudaStream_t s = (cudaStream_t)stream;
  {
    // Nothing in the scratch is read before this call writes it (the coarse
    // table, the level fields, partials and scalars are all produced here),
    // so no part of it needs clearing.
    const NaLevel& lc = P.lv.back();
    launch_coarse_table<double>(S + P.table, lc.d, na_stencil(lc.h, chi, alpha), alpha == 0.0 ? 1 : 0, s);
    const size_t n = P.lv[0].d.n();
    const double* bshift = nullptr;
    if (alpha == 0.0) {
      launch_sum<double>(rhs, n, S + P.partial, S + P.scal, 1.0 / (double)n, s);
      bshift = S + P.scal;
    }
    na_level(P, S, 0, rhs, bshift, x, zero_initial_guess != 0, chi, alpha, s);
    if (alpha == 0.0) {
      launch_sum<double>(x, n, S + P.partial, S + P.scal + 1, 1.0 / (double)n, s);
      launch_sub_scalar<double>(x, n, S + P.scal + 1, s);
    }
  }
  } catch (const CudaError& e) {
    return cuda_status(e.code);
  } catch (const std::bad_alloc&) {
    return IBRD_ERR_OOM;
  } catch (...) {
    return IBRD_ERR_CUDA;
  }
  return IBRD_OK;
}
