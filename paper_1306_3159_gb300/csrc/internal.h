// Internal declarations shared by the CUDA translation units of libibrd.
// Not part of the public ABI (include/ibrd.h is).
#pragma once

#include <cuda_runtime.h>
#include <atomic>
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/ibrd.h"

namespace ibrd {

// ---------------------------------------------------------------- errors
struct CudaError {
  cudaError_t code;
  const char* what;
};

#define IBRD_CUDA(call)                                         \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) throw ::ibrd::CudaError{e_, #call};  \
  } while (0)

// Check the last launch (asynchronous errors surface at the next sync).
inline void check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw CudaError{e, what};
}

// Raises the dynamic shared-memory limit of kernel f to `bytes` on the current
// device, once per device (thread-safe; concurrent first calls both set it).
inline void ensure_smem_attr(const void* f, int bytes, std::atomic<unsigned long long>& done) {
  int dev = 0;
  IBRD_CUDA(cudaGetDevice(&dev));
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_acquire) & bit) return;
  IBRD_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  done.fetch_or(bit, std::memory_order_release);
}

// 16-byte copies and vector accesses need 16-byte aligned fields; a caller's
// pointer into the middle of an allocation may not be.
inline bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// ---------------------------------------------------------------- profiling
// Kernel classes timed by the launch profiler (names in api.cu).
enum ProfClass {
  P_APPLY64, P_APPLY32, P_RBGS64, P_RBGS32, P_RESTRICT64, P_RESTRICT32, P_PROLONG64, P_PROLONG32,
  P_COARSE, P_SPREAD64, P_SPREAD32, P_INTERP64, P_INTERP32, P_DOT, P_AXPY, P_REDUCE, P_VEC, P_SMALL,
  P_SETUP, P_NCLASS
};
// Every launch in the library is bracketed by prof_begin / prof_end: the
// pair counts the launch, checks it, and (when the calling handle has
// profiling on) records CUDA events around it on stream s.
void prof_begin(int cls, cudaStream_t s);
// `bytes` is the algorithmic traffic of the launch (each input read once, each
// output written once), used for achieved-bandwidth reports.
void prof_end(int cls, cudaStream_t s, const char* what, double bytes = 0.0);
template <typename T>
constexpr int pcls(int c64, int c32) { return sizeof(T) == 4 ? c32 : c64; }

// ---------------------------------------------------------------- geometry
struct Dims {
  int nx, ny, nz;
  size_t n() const { return (size_t)nx * ny * nz; }
};

// The cell-centred trilinear prolongation (weights 3/4 near, 1/4 far per
// axis) in the arithmetic every prolongation kernel shares (the stand-alone
// ones, the single-CTA coarse V-cycle and the sweep with the correction
// fused), so that they agree bit for bit: axes in the order z (parent plane
// first), y (parent row first), x, each as t = 3 near + far in one FMA --
// 4 (3/4 near + 1/4 far), and scaling by 4 commutes with rounding -- so the
// three axes give 64 times the correction, added as x + t / 64 in one FMA.
// Bit for bit the 3/4-1/4 form rounded after every step, away from underflow,
// at one instruction per axis.
#ifdef __CUDACC__
__device__ __forceinline__ float prolong_axis(float nearv, float farv) { return __fmaf_rn(3.f, nearv, farv); }
__device__ __forceinline__ double prolong_axis(double nearv, double farv) { return __fma_rn(3.0, nearv, farv); }
__device__ __forceinline__ float prolong_add(float x, float t64) { return __fmaf_rn(0x1p-6f, t64, x); }
__device__ __forceinline__ double prolong_add(double x, double t64) { return __fma_rn(0x1p-6, t64, x); }
#endif

// Coefficients of A_l = alpha I - chi L_{h_l}: diag = alpha + 6 chi/h^2,
// off = chi/h^2, so (A x)_k = diag x_k - off * sum_{6 neighbours} x.
struct Stencil {
  double diag, off;
};

// ---------------------------------------------------------------- FP64 off the FP64 pipe
// GB300's FP64 pipe does about 1.6 additions, multiplications or FMAs per SM
// per clock (measured), and the double <-> float conversion instructions run
// at a similar rate, against 128 FP32 operations. Streaming FP64 kernels therefore convert with
// integer operations on the bit patterns and do their arithmetic in FP32
// (float-float pairs where FP64 accuracy is needed).
#ifdef __CUDACC__
// double -> float, rounded to nearest even, from the bits (the conversion
// instruction only for values whose float is zero, subnormal or not finite)
__device__ __forceinline__ float d2f_bits(double v) {
  const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
  const int E = (int)((hi >> 20) & 0x7FF) - 896;  // float exponent field
  if (E >= 1 && E <= 254) {
    const unsigned t = ((hi & 0xFFFFF) << 3) | (lo >> 29);  // top 23 fraction bits
    const unsigned rest = lo & 0x1FFFFFFFu;                 // the 29 dropped ones
    const unsigned up = (rest > 0x10000000u) | ((rest == 0x10000000u) & t);
    return __uint_as_float((hi & 0x80000000u) | (((unsigned)E << 23) + t + up));  // a carry moves the exponent
  }
  if (((hi & 0x7FFFFFFFu) | lo) == 0) return __uint_as_float(hi & 0x80000000u);
  return (float)v;
}
// float -> double, exact
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned E = (b >> 23) & 0xFF;
  if (E - 1u < 254u)
    return __hiloint2double((int)((b & 0x80000000u) | ((E + 896u) << 20) | ((b & 0x7FFFFFu) >> 3)),
                            (int)((b & 7u) << 29));
  if ((b & 0x7FFFFFFFu) == 0) return __hiloint2double((int)(b & 0x80000000u), 0);
  return (double)f;
}
#endif

// ---------------------------------------------------------------- reductions
// Deterministic two-stage reductions use a fixed grid of kRedBlocks blocks.
constexpr int kRedBlocks = 608;   // 4 x 152 SMs
constexpr int kRedThreads = 256;

// ---------------------------------------------------------------- grid kernels
// All launchers enqueue on `s` and check the launch.
template <typename T>
void launch_apply_A(const T* x, T* y, Dims d, Stencil st, cudaStream_t s);
// y = b - A x. FP64 with scratch (one device double) on grids with nx % 32 ==
// 0 and ny % 8 == 0 (resid_fx_ok): the Laplacian in 64-bit fixed point (exact
// neighbour sums), then two FMAs, mostly off the FP64 pipe; otherwise, and
// for FP32, the plain stencil.
template <typename T>
void launch_residual(const T* x, const T* b, T* y, Dims d, Stencil st, double* scratch, cudaStream_t s);
bool resid_fx_ok(Dims d, Stencil st);
// One full red-black Gauss-Seidel sweep (red = (i+j+k) even) for A x = b -
// *bshift (bshift nullable). On levels where the fused one-pass kernel
// applies it reads xin and writes xout (xin != xout) and returns the number
// of per-CTA partial sums of the new x written into part (0 when part is
// null or holds fewer than the CTA count); on small levels it updates xin in
// place with two half sweeps and returns -1. zero != 0 treats the incoming x
// as 0.
template <typename T>
int launch_rb_sweep(const T* xin, T* xout, const T* b, const double* bshift, Dims d, Stencil st, bool zero,
                    double* part, int part_cap, cudaStream_t s);
template <typename T>
bool rb_sweep_fused_ok(Dims d);
// Launch shape of a red-black sweep kernel picked by the autotuner: tile width
// tx (cells, fused sweep only: 32 or 64 for the tiled kernel, nx for the
// row-resident kernel on levels it serves) and z-march depth zc (planes per
// CTA); 0 keeps the built-in rule (the row-resident kernel where it applies).
struct SweepShape {
  int tx = 0;
  int zc = 0;
};
// Sweep kernels: the fused sweep and the stencil pass of a sweep from zero;
// TUNE_PROLONG (set by hand only): tx = 1 keeps the prolongation a separate
// kernel on a level where it would be fused into the first post-sweep.
enum { TUNE_SWEEP = 0, TUNE_ZERO = 1, TUNE_PROLONG = 2 };
// The tuned shape for kernel `kind` on elements of `elem` bytes and grid d in
// the handle the calling thread is working for, or null.
const SweepShape* tuned_sweep(int elem, int kind, Dims d);
// Kernels with bounded device waits (the TMA ring of the row sweep) read the
// calling handle's context: the device flag such a kernel sets when a wait
// gives up (null outside a handle's call) and the number of tries a wait makes.
constexpr unsigned kDefaultWaitLimit = 1u << 24;
int* wait_error_flag();
unsigned wait_limit();
// Row-resident FP32 sweep (sweep_rows.cu): rows of 128 or 256 cells, ny a
// multiple of 8, nz even; the same contract as the fused sweep of
// launch_rb_sweep (out of place, per-CTA partial sums of the new x when part
// holds enough entries; returns their count or 0). zc = planes per CTA.
bool rows_sweep_ok(Dims d);
int rows_sweep_default_zc(Dims d);
int launch_rows_sweep(const float* xin, float* xout, const float* b, const double* bshift, Dims d, Stencil st,
                      int zc, double* part, int part_cap, cudaStream_t s);
// The same sweep of xin + P xc (P the trilinear prolongation of the coarse
// field xc, as launch_prolong8 adds it) without writing the corrected field:
// the coarse-grid correction fused into the first post-smoothing sweep.
// zc is made even.
int launch_rows_prolong_sweep(const float* xc, const float* xin, float* xout, const float* b, const double* bshift,
                              Dims d, Stencil st, int zc, double* part, int part_cap, cudaStream_t s);
// The first sweep from zero fused with the residual restriction on the same
// levels as the row-resident sweep: x = sweep(0), bc = mean over 8 children of
// b - shift - A x (bc 8-byte aligned). zc = planes per CTA (made even).
bool zero_restrict_rows_ok(Dims d);
int zero_restrict_rows_default_zc(Dims d);
void launch_zero_restrict_rows(const float* b, const double* bshift, float* x, float* bc, Dims d, Stencil st,
                               int zc, cudaStream_t s);
// Levels handled by the single-CTA coarse V-cycle (shared-memory resident).
constexpr int kMaxSmallLevels = 12;
struct CoarseLevels {
  int n;                          // number of levels
  int total;                      // cells over all levels
  int nx[kMaxSmallLevels], ny[kMaxSmallLevels], nz[kMaxSmallLevels];
  int off[kMaxSmallLevels];       // first cell of each level in the packed arrays
  int lgx[kMaxSmallLevels], lgy[kMaxSmallLevels];  // log2 of nx, ny, or -1 if not a power of 2
  double diag[kMaxSmallLevels], offd[kMaxSmallLevels];
};
// Whole V-cycle over the levels in lv (the last one solved exactly with the
// circulant table) in one CTA: x = V(b - bshift), from zero or from x.
template <typename T>
void launch_vcycle_small(const CoarseLevels& lv, const T* b, T* x, const double* bshift, const T* table, bool zero,
                         int nu1, int nu2, cudaStream_t s);
// bc = mean over 8 children of (b - shift - A x) on the fine grid d.
template <typename T>
void launch_resid_restrict(const T* x, const T* b, const double* bshift, T* bc, Dims d, Stencil st,
                           cudaStream_t s);
// FP32 pre-smoothing of one sweep from x = 0 fused with the residual
// restriction: x = sweep(0), bc = mean over 8 children of (b - shift - A x).
bool zero_restrict_ok(Dims d);
void launch_zero_restrict(const float* b, const double* bshift, float* x, float* bc, Dims d, Stencil st,
                          cudaStream_t s);
// x (fine, dims d) += trilinear cell-centred prolongation of xc (dims d/2).
template <typename T>
void launch_prolong8(const T* xc, T* x, Dims d, cudaStream_t s);
// The prolongation of xc added to xin fused with the red-black sweep that
// follows it, on levels the row-resident FP32 sweep serves: writes the swept
// field to xout (xin is left uncorrected) and returns the partial-sum count
// as launch_rb_sweep does, or -1 without launching when it does not apply
// (the caller then prolongs and sweeps separately).
template <typename T>
int launch_prolong_sweep(const T* xc, const T* xin, T* xout, const T* b, const double* bshift, Dims d, Stencil st,
                         double* part, int part_cap, cudaStream_t s);
// Coarsest exact solve x = G b with the circulant table G (dc.n() entries).
template <typename T>
void launch_coarse_solve(const T* table, const T* b, T* x, Dims dc, cudaStream_t s);
// table(d) = sum_{k} cos(2 pi k.d / n) / (n lambda_k), lambda_k eigenvalues of
// A_c; the k = 0 mode is dropped when singular != 0.
template <typename T>
void launch_coarse_table(T* table, Dims dc, Stencil st, int singular, cudaStream_t s);

// Exact FP32 solve of A x = b - shift on a small periodic level (at most 32768
// cells, no side above 64) by the separable Hartley transform; tab holds
// hartley_table_size(d) floats, the first part written by
// launch_hartley_tables (singular: pseudo-inverse, mean-zero result).
bool hartley_ok(Dims d);
size_t hartley_table_size(Dims d);
void launch_hartley_tables(float* tab, Dims d, Stencil st, int singular, cudaStream_t s);
void launch_hartley_solve(const float* tab, const float* b, const double* bshift, float* x, Dims d, cudaStream_t s);

// ---------------------------------------------------------------- vector kernels
// Reductions below that take a ticket (a per-handle counter, 0 between uses)
// form their result in the last CTA of the partial-sum launch, with the
// arithmetic of launch_finalize, instead of in a separate launch.
//
// Sum of x[0..n) into partials (kRedBlocks doubles); then finalize into *out.
template <typename T>
void launch_sum(const T* x, size_t n, double* partial, double* out, double scale, cudaStream_t s,
                unsigned* ticket = nullptr);
// *out = scale * sum(partial[0..np))
void launch_finalize(const double* partial, int np, double* out, double scale, cudaStream_t s);
// y = (T)x with sums: *out_in = sum(x), *out_out = sum(y), both in FP64
// (partial uses 2 * kRedBlocks doubles).
template <typename X, typename T>
void launch_convert_sum(const X* x, T* y, size_t n, double* partial, double* out_in, double* out_out,
                        cudaStream_t s, unsigned* ticket = nullptr);
// out[i] = a * (in[i] - *shift) + bcoef * f[i]   (shift, f nullable; N-vectors)
template <typename F>
void launch_nvec_affine(const double* in, double* out, int n, double a, const double* shift, const F* f,
                        double bcoef, cudaStream_t s);
// out[0] = scale * sum(x*y)  (FP32 vectors: FP32 products, FP64 sums of runs)
template <typename E>
void launch_dot(const E* x, const E* y, size_t n, double* partial, double* out, double scale, cudaStream_t s,
                unsigned* ticket = nullptr);
// x[i] -= *mean (device scalar)
template <typename T>
void launch_sub_scalar(T* x, size_t n, const double* mean, cudaStream_t s);
// y = (Ty)(a * x + shift), shift from device scalar (nullable)
template <typename Tx, typename Ty>
void launch_convert(const Tx* x, Ty* y, size_t n, double a, const double* shift, cudaStream_t s);
// y = a x + b y (host scalars, applied in E)
template <typename E>
void launch_axpby(double a, const E* x, double b, E* y, size_t n, cudaStream_t s);
// y = x * (num / *den)  (device scalar den, host num)
template <typename E>
void launch_scale_by_inv(const E* x, E* y, size_t n, const double* den, double num, cudaStream_t s);
// y = (float) x * sigma and *out = sum of y^2 (partial: kRedBlocks doubles)
void launch_convert_sq(const double* x, float* y, size_t n, double sigma, double* partial, double* out,
                       cudaStream_t s, unsigned* ticket = nullptr);
// the same with sigma read from device memory
void launch_convert_sq(const double* x, float* y, size_t n, const double* sigma_dev, double* partial, double* out,
                       cudaStream_t s, unsigned* ticket = nullptr);
// x += a * d  (FP32 d added to FP64 x)
void launch_add_scaled(double a, const float* d, double* x, size_t n, cudaStream_t s);
// x += d / *div_dev  (divisor read from device memory)
void launch_add_divided(const double* div_dev, const float* d, double* x, size_t n, cudaStream_t s);
// flag = any non-finite in x (writes 1 into *flag if so; *flag must start 0)
template <typename T>
void launch_nonfinite(const T* x, size_t n, int* flag, cudaStream_t s);

// ---------------------------------------------------------------- blob kernels
constexpr int kTile = 8;  // spreading tile edge (cells)

struct BlobSet {
  int n = 0;
  int cap = 0;
  int width = 4;             // kernel width w (3 or 4)
  double* q = nullptr;       // N x 3 wrapped positions
  int* idx = nullptr;        // N x 3 x 4 wrapped cell indices (axis-major)
  double* w64 = nullptr;     // N x 3 x 4 weights
  float* w32 = nullptr;      // FP32 copy
  // tile binning
  int ntx = 0, nty = 0, ntz = 0, ntiles = 0;
  int* tile_count = nullptr;   // ntiles
  int* tile_offset = nullptr;  // ntiles + 1
  int* tile_cursor = nullptr;  // ntiles
  int* tile_blobs = nullptr;   // pairs (blob index per (tile, blob) pair)
  int pair_cap = 0;
  int* active = nullptr;       // active tile ids (ntiles capacity)
  int n_active = 0;
  int* d_meta = nullptr;       // [0] = pairs, [1] = active tiles, [2] = covered cells
  // cells covered by at least one blob support, in (tile, cell) order
  int* cell_count = nullptr;   // per active tile
  int* cell_offset = nullptr;  // per active tile + 1
  int* cells = nullptr;        // linear cell index
  int* cell_tile = nullptr;    // tile id of each covered cell
  int cell_cap = 0;
  int n_cells = 0;
};

void blobs_setup(BlobSet& b, Dims d, double h, const double* q_in, int n, cudaStream_t s);
// out (+)= scale * sum_b coef_b lam_b phi_b  (coef nullable = 1);
// lam (type L) and coef (FP64) device N-vectors; out field of type T.
template <typename T, typename L = double>
void launch_spread(const BlobSet& b, Dims d, const L* lam, const double* coef, double scale, T* out,
                   int accumulate, cudaStream_t s);
// Spread a constant *cval (device scalar) times scale to all blobs.
template <typename T>
void launch_spread_const(const BlobSet& b, Dims d, const double* cval, double scale, T* out, cudaStream_t s);
// out[b] = scale * (J x)_b  (output N-vector of type O)
template <typename T, typename O = double>
void launch_interp(const BlobSet& b, Dims d, const T* x, double scale, O* out, cudaStream_t s);

// ---------------------------------------------------------------- Krylov kernels
constexpr int kDotGroup = 8;
// Work that the last CTA of a multi-dot or multi-axpy launch to finish does
// after the others (it takes the last ticket of a per-handle counter after a
// fence; no CTA waits for another), so that an FGMRES iteration needs no
// separate single-CTA launches for it. ticket: 0 between uses, reset by that
// CTA. The arithmetic is that of the separate kernels it replaces.
struct DotTail {
  unsigned* ticket = nullptr;
  double* out = nullptr;  // out[g] = the sum of partial row g, times scale[g] for g < nscale
  const double* scale = nullptr;
  int nscale = 0;
  int nb = 0;  // > 0: then launch_gs_norm_estimate's work on out[0..nb]
  double *ww = nullptr, *hhat = nullptr, *hinv = nullptr;
};
struct AxpyTail {
  unsigned* ticket = nullptr;
  double* rho2 = nullptr;  // the sum of the squares partials, then launch_gs_norm_fix's work
  const double* hhat = nullptr;
  double *hsub = nullptr, *vscale = nullptr, *sq = nullptr;
  double* H = nullptr;  // then launch_givens' work on column j
  int ldh = 0, j = 0;
  double *cs = nullptr, *sn = nullptr, *gvec = nullptr, *res = nullptr;
};
// partial[g * kRedBlocks + blk] for g < nvec (nvec <= kDotGroup)
// gate (nullable device scalar): the kernel does nothing when *gate == 0.
void launch_multidot(const double* V, size_t ldv, int nvec, const double* w, size_t n, double* partial,
                     cudaStream_t s, const double* gate = nullptr, const DotTail* tail = nullptr);
// FP32 basis: V and w 16-byte aligned, ldv % 4 == 0.
void launch_multidot(const float* V, size_t ldv, int nvec, const float* w, size_t n, double* partial,
                     cudaStream_t s, const double* gate = nullptr, const DotTail* tail = nullptr);
// out[g] = sum_blk partial[g*kRedBlocks + blk]   (g < nvec), times scale[g]
// for g < nscale when scale is given
void launch_reduce_partials(const double* partial, int nvec, double* out, cudaStream_t s,
                            const double* gate = nullptr, const double* scale = nullptr, int nscale = 0);
// w += sign * sum_g coef[g] cscale[g] V[g] (cscale optional), then w *= *post
// (optional); optional partial sums of squares of the new w.
void launch_multi_axpy(double* w, const double* V, size_t ldv, int nvec, const double* coef, double sign,
                       size_t n, double* partial_sq, cudaStream_t s, const double* gate = nullptr,
                       const double* cscale = nullptr, const double* post = nullptr,
                       const AxpyTail* tail = nullptr);
// FP32 basis: V and w 16-byte aligned, ldv % 4 == 0.
void launch_multi_axpy(float* w, const float* V, size_t ldv, int nvec, const double* coef, double sign, size_t n,
                       double* partial_sq, cudaStream_t s, const double* gate = nullptr,
                       const double* cscale = nullptr, const double* post = nullptr,
                       const AxpyTail* tail = nullptr);
// Gram-Schmidt norm bookkeeping (one-warp kernels): the estimate of the norm
// after one pass from the projections h[0..nb) and h[nb] = ||w||^2 (writes
// ||w||^2, the estimate and its reciprocal); after a pass that stored the
// vector scaled by the estimate's reciprocal, with squared norm *rho2:
// h_{j+1,j}, the stored vector's inverse norm and h_{j+1,j}^2; for a vector
// normalised exactly afterwards: h_{j+1,j} = sqrt(*sq) and scale 1.
void launch_gs_norm_estimate(const double* h, int nb, double* ww, double* hhat, double* hinv, cudaStream_t s);
void launch_gs_norm_fix(const double* rho2, const double* hhat, double* hsub, double* vscale, double* sq,
                        cudaStream_t s);
void launch_gs_norm_unit(const double* sq, double* hsub, double* vscale, cudaStream_t s);
// Givens step j on column H[:, j] (ldh = restart + 1): rotations cs/sn,
// residual vector gvec; writes |gvec[j+1]| to *res.
void launch_givens(double* H, int ldh, int j, double* cs, double* sn, double* gvec, double* res,
                   cudaStream_t s);
// Back substitution y = R^{-1} g for the leading k x k block.
void launch_backsolve(const double* H, int ldh, int k, const double* gvec, double* y, cudaStream_t s);
// Combine two dot results: h[i] += h2[i] for i < n (device).
void launch_vec_add_small(double* h, const double* h2, int n, cudaStream_t s, const double* gate = nullptr);
// *flag = (eta >= 1 || *sq < eta^2 *ww); *count += *flag
void launch_reorth_flag(const double* ww, const double* sq, double eta, double* flag, double* count, cudaStream_t s);
// *dst = sqrt(*src)
void launch_sqrt_scalar(const double* src, double* dst, cudaStream_t s);

// Small-vector (length N) GMRES for the approximate Schur complement: one
// block does the Arnoldi step on U (rows of length n, type S) with small
// Hessenberg Hs (FP64, ldh = m + 1), including Givens rotations.
// Step j: w (= U[j+1]) orthogonalized against U[0..j] by classical
// Gram-Schmidt with a DGKS second pass, normalized.
// If wshift is non-null, *wshift is first subtracted from every entry of w;
// if usum is non-null, *usum = usum_scale * sum(U[j+1]) after normalising.
template <typename S>
void launch_small_arnoldi(S* U, int n, int j, double* Hs, int ldh, double* cs, double* sn, double* gvec,
                          const double* wshift, double* usum, double usum_scale, cudaStream_t s);
// U[0] = r / ||r||, gvec = [||r||, 0, ...]; *usum = usum_scale * sum(U[0]) if
// usum is non-null.
template <typename S>
void launch_small_start(const double* r, S* U0, int n, double* gvec, int m, double* usum, double usum_scale,
                        cudaStream_t s);
// x = U[0..k) y where y = R^{-1} g (solved inside); subtract mean if project.
template <typename S>
void launch_small_finish(const S* U, int n, int k, const double* Hs, int ldh, const double* gvec, double* x,
                         int project_mean, cudaStream_t s);

}  // namespace ibrd
