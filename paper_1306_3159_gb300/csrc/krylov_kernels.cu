// Krylov kernels for flexible GMRES (Sec. III.E: "FGMRES" outer solver) and
// the small inner GMRES of the approximate Schur-complement preconditioner
// (Appendix A, step 2b).
//
// Outer vectors live on the grid (plus the N blob unknowns for the saddle
// point) and are FP64. Orthogonalisation is classical Gram-Schmidt with a
// conditional second pass, done as fused multi-dot / multi-axpy streams over
// up to 8 basis vectors at a time with deterministic two-stage reductions.
// The Hessenberg matrix, Givens rotations and the least-squares update stay on
// the device; the host only reads the residual estimate.
#include <cmath>

#include "internal.h"

namespace ibrd {
namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block sum, result valid in thread 0 of the block. Safe to call repeatedly.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sw[32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sw[wid] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? sw[threadIdx.x] : 0.0;
  if (wid == 0) v = warp_sum(v);
  return v;
}

// Block sum of FP32 per-thread values, result valid in thread 0: each warp
// adds its 32 values in FP32, the block adds the warps' totals in FP64. The
// FP64 pipe of GB300 is about 64 times narrower than the FP32 one, so five
// FP64 shuffle levels over every warp of every block cost microseconds at the
// end of a reduction over a 256^3 field; this keeps them to one warp per block.
__device__ __forceinline__ double block_sum_f(float v) {
  __shared__ double sw[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sw[wid] = (double)v;
  __syncthreads();
  double d = (threadIdx.x < (blockDim.x >> 5)) ? sw[threadIdx.x] : 0.0;
  if (wid == 0) d = warp_sum(d);
  return d;
}

// Givens step j on column H[:, j] (ldh = restart + 1): the earlier rotations
// cs/sn applied, a new one formed and applied to the residual vector gvec;
// |gvec[j+1]| into *res. One thread.
__device__ void givens_step(double* __restrict__ H, int ldh, int j, double* __restrict__ cs,
                            double* __restrict__ sn, double* __restrict__ gvec, double* __restrict__ res) {
  double* h = H + (size_t)j * ldh;
  for (int i = 0; i < j; ++i) {
    const double t = cs[i] * h[i] + sn[i] * h[i + 1];
    h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
    h[i] = t;
  }
  const double a = h[j], b = h[j + 1];
  const double r = hypot(a, b);
  double c = 1.0, s = 0.0;
  if (r > 0.0) {
    c = a / r;
    s = b / r;
  }
  h[j] = r;
  h[j + 1] = 0.0;
  cs[j] = c;
  sn[j] = s;
  const double gj = gvec[j];
  gvec[j + 1] = -s * gj;
  gvec[j] = c * gj;
  *res = fabs(gvec[j + 1]);
}

// The Gram-Schmidt norm estimate (see k_gs_norm_estimate), by one warp.
__device__ void gs_norm_estimate_warp(const double* __restrict__ h, int nb, double* __restrict__ ww,
                                      double* __restrict__ hhat, double* __restrict__ hinv) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int i = lane; i < nb; i += 32) s = fma(h[i], h[i], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane != 0) return;
  const double w2 = h[nb];
  const double e = fmax(w2 - s, 1e-8 * w2);
  const double r = e > 0.0 ? sqrt(e) : 0.0;
  *ww = w2;
  *hhat = r;
  *hinv = r > 0.0 ? 1.0 / r : 0.0;
}

// The Gram-Schmidt norm fix (see k_gs_norm_fix) for rho2 = ||stored||^2. One thread.
__device__ void gs_norm_fix_one(double rho2, const double* __restrict__ hhat, double* __restrict__ hsub,
                                double* __restrict__ vscale, double* __restrict__ sq) {
  const double r = sqrt(fmax(rho2, 0.0));
  const double hs = *hhat * r;
  *hsub = hs;
  *vscale = r > 0.0 ? 1.0 / r : 0.0;
  *sq = hs * hs;
}

// Whether this CTA is the last of the grid to finish; thread 0 wrote the
// CTA's partials before the call. A fence orders them before the ticket.
__device__ __forceinline__ bool last_cta(unsigned* ticket) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// Sum of partial row g (kRedBlocks values) in the order of k_reduce_partials;
// valid in thread 0. Read through L2: other CTAs wrote the row.
__device__ __forceinline__ double partial_row_sum(const double* partial, int g) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < kRedBlocks; i += blockDim.x) acc += __ldcg(partial + (size_t)g * kRedBlocks + i);
  return block_sum(acc);
}

// Tail of a multi-dot launch (last CTA): the rows' sums into tail.out, then
// the norm estimate.
__device__ void dot_tail(const double* partial, int nv, const DotTail& tail) {
  for (int g = 0; g < nv; ++g) {
    const double v = partial_row_sum(partial, g);
    if (threadIdx.x == 0) tail.out[g] = (g < tail.nscale) ? v * tail.scale[g] : v;
  }
  __syncthreads();
  if (tail.nb > 0 && threadIdx.x < 32) gs_norm_estimate_warp(tail.out, tail.nb, tail.ww, tail.hhat, tail.hinv);
  if (threadIdx.x == 0) *tail.ticket = 0u;
}

// Tail of a multi-axpy launch (last CTA): the squares' sum, the norm fix and
// the Givens step.
__device__ void axpy_tail(const double* partial_sq, const AxpyTail& tail) {
  const double v = partial_row_sum(partial_sq, 0);
  if (threadIdx.x == 0) {
    *tail.rho2 = v;
    gs_norm_fix_one(v, tail.hhat, tail.hsub, tail.vscale, tail.sq);
    givens_step(tail.H, tail.ldh, tail.j, tail.cs, tail.sn, tail.gvec, tail.res);
    *tail.ticket = 0u;
  }
}

// FP64 vectors: one FMA per element and vector.// FP64 vectors: one FMA per element and vector.
template <int NV>
__global__ void __launch_bounds__(kRedThreads) k_multidot(const double* __restrict__ V, size_t ldv,
                                                          const double* __restrict__ w, size_t n,
                                                          double* __restrict__ partial, const double* __restrict__ gate,
                                                          DotTail tail) {
  if (gate && *gate == 0.0) return;
  double acc[NV];
#pragma unroll
  for (int g = 0; g < NV; ++g) acc[g] = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double wi = w[i];
#pragma unroll
    for (int g = 0; g < NV; ++g) acc[g] = fma(V[g * ldv + i], wi, acc[g]);
  }
#pragma unroll
  for (int g = 0; g < NV; ++g) {
    const double s = block_sum(acc[g]);
    if (threadIdx.x == 0) partial[g * kRedBlocks + blockIdx.x] = s;
  }
  if (tail.ticket && last_cta(tail.ticket)) dot_tail(partial, NV, tail);
}

// FP32 vectors (16-byte aligned, ldv % 4 == 0): 4-vectors, FP32 products
// summed per thread and across a warp in FP32, across warps and blocks in FP64.
template <int NV>
__global__ void __launch_bounds__(kRedThreads) k_multidot_f32(const float* __restrict__ V, size_t ldv,
                                                              const float* __restrict__ w, size_t n,
                                                              double* __restrict__ partial,
                                                              const double* __restrict__ gate, DotTail tail) {
  if (gate && *gate == 0.0) return;
  float acc[NV];
#pragma unroll
  for (int g = 0; g < NV; ++g) acc[g] = 0.f;
  const size_t n4 = n >> 2, stride = (size_t)gridDim.x * blockDim.x;
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  for (size_t i = t; i < n4; i += stride) {
    const float4 wi = reinterpret_cast<const float4*>(w)[i];
#pragma unroll
    for (int g = 0; g < NV; ++g) {
      const float4 v = reinterpret_cast<const float4*>(V + g * ldv)[i];
      acc[g] = fmaf(v.x, wi.x, fmaf(v.y, wi.y, fmaf(v.z, wi.z, fmaf(v.w, wi.w, acc[g]))));
    }
  }
  const size_t i = 4 * n4 + t;  // at most 3 tail elements
  if (i < n) {
    const float wi = w[i];
#pragma unroll
    for (int g = 0; g < NV; ++g) acc[g] = fmaf(V[g * ldv + i], wi, acc[g]);
  }
#pragma unroll
  for (int g = 0; g < NV; ++g) {
    const double s = block_sum_f(acc[g]);
    if (threadIdx.x == 0) partial[g * kRedBlocks + blockIdx.x] = s;
  }
  if (tail.ticket && last_cta(tail.ticket)) dot_tail(partial, NV, tail);
}

__global__ void __launch_bounds__(kRedThreads) k_reduce_partials(const double* __restrict__ partial,
                                                                 double* __restrict__ out,
                                                                 const double* __restrict__ gate,
                                                                 const double* __restrict__ scale, int nscale) {
  if (gate && *gate == 0.0) return;
  // blockIdx.x = vector g
  double acc = 0.0;
  for (int i = threadIdx.x; i < kRedBlocks; i += blockDim.x) acc += partial[blockIdx.x * kRedBlocks + i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) out[blockIdx.x] = ((int)blockIdx.x < nscale) ? acc * scale[blockIdx.x] : acc;
}

template <int NV, bool SQ>
__global__ void __launch_bounds__(kRedThreads) k_multi_axpy(double* __restrict__ w, const double* __restrict__ V,
                                                            size_t ldv, const double* __restrict__ coef,
                                                            double sign, size_t n, double* __restrict__ partial_sq,
                                                            const double* __restrict__ gate,
                                                            const double* __restrict__ cscale,
                                                            const double* __restrict__ post, AxpyTail tail) {
  if (gate && *gate == 0.0) return;
  double c[NV];
#pragma unroll
  for (int g = 0; g < NV; ++g) c[g] = sign * coef[g] * (cscale ? cscale[g] : 1.0);
  const double ps = post ? *post : 1.0;
  double sq = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double wi = w[i];
#pragma unroll
    for (int g = 0; g < NV; ++g) wi = fma(c[g], V[g * ldv + i], wi);
    if (post) wi *= ps;
    w[i] = wi;
    if (SQ) sq = fma(wi, wi, sq);
  }
  if (SQ) {
    sq = block_sum(sq);
    if (threadIdx.x == 0) partial_sq[blockIdx.x] = sq;
    if (tail.ticket && last_cta(tail.ticket)) axpy_tail(partial_sq, tail);
  }
}

// FP32 vectors (16-byte aligned, ldv % 4 == 0), 4-vectors; the sum of squares
// is taken per thread and across a warp in FP32, across warps in FP64.
template <int NV, bool SQ>
__global__ void __launch_bounds__(kRedThreads) k_multi_axpy_f32(float* __restrict__ w, const float* __restrict__ V,
                                                                size_t ldv, const double* __restrict__ coef,
                                                                double sign, size_t n,
                                                                double* __restrict__ partial_sq,
                                                                const double* __restrict__ gate,
                                                                const double* __restrict__ cscale,
                                                                const double* __restrict__ post, AxpyTail tail) {
  if (gate && *gate == 0.0) return;
  float c[NV];
#pragma unroll
  for (int g = 0; g < NV; ++g) c[g] = (float)(sign * coef[g] * (cscale ? cscale[g] : 1.0));
  const bool scaled = post != nullptr;
  const float ps = scaled ? (float)*post : 1.f;
  float sq = 0.f;
  const size_t n4 = n >> 2, stride = (size_t)gridDim.x * blockDim.x;
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  for (size_t i = t; i < n4; i += stride) {
    float4 wi = reinterpret_cast<const float4*>(w)[i];
#pragma unroll
    for (int g = 0; g < NV; ++g) {
      const float4 v = reinterpret_cast<const float4*>(V + g * ldv)[i];
      wi.x = fmaf(c[g], v.x, wi.x);
      wi.y = fmaf(c[g], v.y, wi.y);
      wi.z = fmaf(c[g], v.z, wi.z);
      wi.w = fmaf(c[g], v.w, wi.w);
    }
    if (scaled) wi.x *= ps, wi.y *= ps, wi.z *= ps, wi.w *= ps;
    reinterpret_cast<float4*>(w)[i] = wi;
    if (SQ) sq = fmaf(wi.x, wi.x, fmaf(wi.y, wi.y, fmaf(wi.z, wi.z, fmaf(wi.w, wi.w, sq))));
  }
  const size_t i = 4 * n4 + t;
  if (i < n) {
    float wi = w[i];
#pragma unroll
    for (int g = 0; g < NV; ++g) wi = fmaf(c[g], V[g * ldv + i], wi);
    if (scaled) wi *= ps;
    w[i] = wi;
    if (SQ) sq = fmaf(wi, wi, sq);
  }
  if (SQ) {
    const double b = block_sum_f(sq);
    if (threadIdx.x == 0) partial_sq[blockIdx.x] = b;
    if (tail.ticket && last_cta(tail.ticket)) axpy_tail(partial_sq, tail);
  }
}

__global__ void k_givens(double* __restrict__ H, int ldh, int j, double* __restrict__ cs, double* __restrict__ sn,
                         double* __restrict__ gvec, double* __restrict__ res) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  givens_step(H, ldh, j, cs, sn, gvec, res);
}

__global__ void k_backsolve(const double* __restrict__ H, int ldh, int k, const double* __restrict__ gvec,
                            double* __restrict__ y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    double t = gvec[i];
    for (int l = i + 1; l < k; ++l) t -= H[(size_t)l * ldh + i] * y[l];
    const double d = H[(size_t)i * ldh + i];
    y[i] = d != 0.0 ? t / d : 0.0;
  }
}

__global__ void k_vec_add_small(double* __restrict__ h, const double* __restrict__ h2, int n,
                                const double* __restrict__ gate) {
  if (gate && *gate == 0.0) return;
  const int i = threadIdx.x;
  if (i < n) h[i] += h2[i];
}

// flag = 1 when the Gram-Schmidt second pass is needed: ||w'||^2 < eta^2 ||w||^2
// (or eta >= 1); counts the passes in *count.
__global__ void k_reorth_flag(const double* __restrict__ ww, const double* __restrict__ sq, double eta,
                              double* __restrict__ flag, double* __restrict__ count) {
  if (threadIdx.x != 0) return;
  const double f = (eta >= 1.0 || *sq < eta * eta * *ww) ? 1.0 : 0.0;
  *flag = f;
  *count += f;
}

__global__ void k_sqrt_scalar(const double* __restrict__ src, double* __restrict__ dst) {
  if (threadIdx.x == 0) *dst = sqrt(fmax(*src, 0.0));
}

// The norm of w after one classical Gram-Schmidt pass, estimated before the
// pass from its projections h[0..nb) and h[nb] = ||w||^2: ||w||^2 - sum h_i^2,
// floored at 1e-8 ||w||^2 (where cancellation leaves no digits the floor only
// changes the stored vector's scale, which the exact norm taken in the same
// pass then records). Writes ||w||^2, the estimate and its reciprocal (0 for
// w = 0). One warp.
__global__ void k_gs_norm_estimate(const double* __restrict__ h, int nb, double* __restrict__ ww,
                                   double* __restrict__ hhat, double* __restrict__ hinv) {
  gs_norm_estimate_warp(h, nb, ww, hhat, hinv);
}

// After the pass wrote the new basis vector scaled by 1 / hhat with squared
// norm rho2: the Hessenberg entry h_{j+1,j} = hhat sqrt(rho2) (the norm of the
// unscaled vector), the stored vector's inverse norm, and h_{j+1,j}^2 into sq.
__global__ void k_gs_norm_fix(const double* __restrict__ rho2, const double* __restrict__ hhat,
                              double* __restrict__ hsub, double* __restrict__ vscale, double* __restrict__ sq) {
  if (threadIdx.x == 0) gs_norm_fix_one(*rho2, hhat, hsub, vscale, sq);
}

// h_{j+1,j} = sqrt(sq), for a basis vector that is then normalised exactly
// (stored scale 1).
__global__ void k_gs_norm_unit(const double* __restrict__ sq, double* __restrict__ hsub,
                               double* __restrict__ vscale) {
  if (threadIdx.x != 0) return;
  *hsub = sqrt(fmax(*sq, 0.0));
  *vscale = 1.0;
}

// ---------------------------------------------------------------- small GMRES
// One CTA; vectors and arithmetic of type S (FP32 in the mixed-precision
// solves). On GB300 one SM runs FP64 at about 2 FMA per clock with long
// dependent latencies, so these kernels avoid serial FP64 chains: every
// reduction is a tree over lanes and warps, and with S = float the small
// least-squares problem (Givens rotations, back substitution) runs in FP32
// too; the Hessenberg matrix and residual vector are stored in FP64.
constexpr int kSmallThreads = 1024;
constexpr int kSmallMaxBasis = 64;  // m + 1 <= 61 basis vectors
constexpr int kSmallRegBasis = 8;   // bases up to this size are read with independent loads

template <typename S>
__device__ __forceinline__ S warp_sum_t(S v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sums over the block of per-warp partials red[w][v] (v < cnt): warp v adds
// the 32 partials of value v. Every thread sees out[] afterwards.
template <typename S>
__device__ __forceinline__ void finish_sums(int cnt, S (*red)[kSmallMaxBasis + 1], S* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  for (int v = wid; v < cnt; v += nw) {
    S x = lane < nw ? red[lane][v] : (S)0;
    x = warp_sum_t<S>(x);
    if (lane == 0) out[v] = x;
  }
  __syncthreads();
}

template <typename S>
__global__ void __launch_bounds__(kSmallThreads) k_small_start(const double* __restrict__ r, S* __restrict__ U0, int n,
                                                                double* __restrict__ gvec, int m,
                                                                double* __restrict__ usum, double usum_scale) {
  __shared__ S red[32][kSmallMaxBasis + 1];
  __shared__ S out[2];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
  S ss = 0;
#pragma unroll 4
  for (int i = tid; i < n; i += nt) {
    const S v = (S)r[i];
    ss += v * v;
  }
  ss = warp_sum_t<S>(ss);
  if (lane == 0) red[wid][0] = ss;
  finish_sums<S>(1, red, out);
  const S nrm = sqrt(out[0]);
  const S inv = nrm > (S)0 ? (S)1 / nrm : (S)0;
  S su = 0;
#pragma unroll 4
  for (int i = tid; i < n; i += nt) {
    const S u = (S)r[i] * inv;
    U0[i] = u;
    su += u;
  }
  if (tid <= m) gvec[tid] = (tid == 0) ? (double)nrm : 0.0;
  if (usum) {
    su = warp_sum_t<S>(su);
    if (lane == 0) red[wid][0] = su;
    finish_sums<S>(1, red, out + 1);
    if (tid == 0) *usum = usum_scale * (double)out[1];
  }
}

// Thread 0's part of an Arnoldi step: column j of the Hessenberg matrix from
// the projections hacc[0..j] and the new norm, the earlier rotations applied,
// a new Givens rotation formed and applied to the residual vector.
template <typename S>
__device__ void small_givens(double* __restrict__ Hs, int ldh, int j, double* __restrict__ cs, double* __restrict__ sn,
                             double* __restrict__ gvec, const S* hacc, S nrm) {
  double* h = Hs + (size_t)j * ldh;
  S hc[kSmallMaxBasis + 1];
  for (int i = 0; i <= j; ++i) hc[i] = hacc[i];
  hc[j + 1] = nrm;
  for (int i = 0; i < j; ++i) {
    const S c = (S)cs[i], sg = (S)sn[i];
    const S tt = c * hc[i] + sg * hc[i + 1];
    hc[i + 1] = -sg * hc[i] + c * hc[i + 1];
    hc[i] = tt;
  }
  const S a = hc[j], b = hc[j + 1];
  const S r = hypot(a, b);
  S c = 1, sg = 0;
  if (r > (S)0) {
    c = a / r;
    sg = b / r;
  }
  hc[j] = r;
  hc[j + 1] = 0;
  for (int i = 0; i <= j + 1; ++i) h[i] = (double)hc[i];
  cs[j] = (double)c;
  sn[j] = (double)sg;
  const S gj = (S)gvec[j];
  gvec[j + 1] = (double)(-sg * gj);
  gvec[j] = (double)(c * gj);
}

// Arnoldi step j: w = U[j+1] holds (J A~^-1 S) U[j]. Classical Gram-Schmidt
// against U[0..j] (all projections in one pass and one block reduction),
// repeated once when the norm falls below 1/sqrt(2) of its value before
// (DGKS test); normalise, then one Givens rotation. Up to kSmallRegBasis
// basis vectors are read with independent loads, larger bases in a loop.
template <typename S>
__global__ void __launch_bounds__(kSmallThreads) k_small_arnoldi(S* __restrict__ U, int n, int j,
                                                                  double* __restrict__ Hs, int ldh,
                                                                  double* __restrict__ cs, double* __restrict__ sn,
                                                                  double* __restrict__ gvec,
                                                                  const double* __restrict__ wshift,
                                                                  double* __restrict__ usum, double usum_scale) {
  __shared__ S red[32][kSmallMaxBasis + 1];
  __shared__ S hv[kSmallMaxBasis + 1], hacc[kSmallMaxBasis + 1], nv[2];
  S* w = U + (size_t)(j + 1) * n;
  const int nb = j + 1;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5;
  const bool reg = nb <= kSmallRegBasis - 1;  // the nb projections and <w, w> fit the register path
  const S sh = wshift ? (S)*wshift : (S)0;
  if (wshift)
    for (int t = tid; t < n; t += nt) w[t] -= sh;
  for (int v = tid; v < nb; v += nt) hacc[v] = 0;
  // hv[i] = <U_i, w> for i < nb and, with ww, hv[nb] = <w, w>
  auto dots = [&](bool ww) {
    const int cnt = nb + (ww ? 1 : 0);
    if (reg) {
      S acc[kSmallRegBasis];
#pragma unroll
      for (int v = 0; v < kSmallRegBasis; ++v) acc[v] = 0;
#pragma unroll 4
      for (int t = tid; t < n; t += nt) {
        const S wt = w[t];
        S u[kSmallRegBasis];
#pragma unroll
        for (int v = 0; v < kSmallRegBasis; ++v) u[v] = v < nb ? U[(size_t)v * n + t] : (S)0;
#pragma unroll
        for (int v = 0; v < kSmallRegBasis; ++v) acc[v] += (v < nb ? u[v] : (v == nb ? wt : (S)0)) * wt;
      }
#pragma unroll
      for (int v = 0; v < kSmallRegBasis; ++v) {
        const S sv = warp_sum_t<S>(acc[v]);
        if (lane == 0 && v < cnt) red[wid][v] = sv;
      }
    } else {
      for (int v = 0; v < cnt; ++v) {
        S a = 0;
        const S* u = v < nb ? U + (size_t)v * n : w;
        for (int t = tid; t < n; t += nt) a += u[t] * w[t];
        a = warp_sum_t<S>(a);
        if (lane == 0) red[wid][v] = a;
      }
    }
    finish_sums<S>(cnt, red, hv);
  };
  // w -= sum_i hv[i] U_i; nv[0] = <w, w> after
  auto update = [&]() {
    S sq = 0;
#pragma unroll 4
    for (int t = tid; t < n; t += nt) {
      S x = w[t];
      if (reg) {
        S u[kSmallRegBasis];
#pragma unroll
        for (int v = 0; v < kSmallRegBasis; ++v) u[v] = v < nb ? U[(size_t)v * n + t] : (S)0;
#pragma unroll
        for (int v = 0; v < kSmallRegBasis; ++v)
          if (v < nb) x -= hv[v] * u[v];
      } else {
        for (int v = 0; v < nb; ++v) x -= hv[v] * U[(size_t)v * n + t];
      }
      w[t] = x;
      sq += x * x;
    }
    for (int v = tid; v < nb; v += nt) hacc[v] += hv[v];
    sq = warp_sum_t<S>(sq);
    if (lane == 0) red[wid][0] = sq;
    finish_sums<S>(1, red, nv);
  };
  dots(true);
  const S before = hv[nb];
  update();
  if (nv[0] < (S)0.5 * before) {
    dots(false);
    update();
  }
  const S nrm = sqrt(nv[0]);
  const S inv = nrm > (S)0 ? (S)1 / nrm : (S)0;
  S su = 0;
#pragma unroll 4
  for (int t = tid; t < n; t += nt) {
    const S x = w[t] * inv;
    w[t] = x;
    su += x;
  }
  if (usum) {
    su = warp_sum_t<S>(su);
    if (lane == 0) red[wid][0] = su;
    finish_sums<S>(1, red, nv + 1);
    if (tid == 0) *usum = usum_scale * (double)nv[1];
  }
  if (tid == 0) small_givens<S>(Hs, ldh, j, cs, sn, gvec, hacc, nrm);
}

// Register-resident Arnoldi step for vectors of at most 4 * kSmallThreads
// entries and NB = j + 1 basis vectors (the inner Schur GMRES of a few
// thousand blobs): each thread loads its entries t + kSmallThreads k of w
// and of U[0..NB) once, and the projections, the update, the second pass,
// the normalisation and the sums run on registers; w is stored once. The
// per-entry arithmetic and the reductions are those of k_small_arnoldi, in
// the same order, so the results are the same bit for bit.
template <typename S, int NB>
__global__ void __launch_bounds__(kSmallThreads) k_small_arnoldi_r(S* __restrict__ U, int n, double* __restrict__ Hs,
                                                                    int ldh, double* __restrict__ cs,
                                                                    double* __restrict__ sn, double* __restrict__ gvec,
                                                                    const double* __restrict__ wshift,
                                                                    double* __restrict__ usum, double usum_scale) {
  constexpr int PER = 4, j = NB - 1;
  __shared__ S red[32][kSmallMaxBasis + 1];
  __shared__ S hv[NB + 1], hacc[NB], nv[2];
  S* w = U + (size_t)NB * n;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5;
  const S sh = wshift ? (S)*wshift : (S)0;
  S x[PER], u[NB][PER];
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int t = tid + k * nt;
    const bool in = t < n;
    x[k] = in ? (wshift ? w[t] - sh : w[t]) : (S)0;
#pragma unroll
    for (int v = 0; v < NB; ++v) u[v][k] = in ? U[(size_t)v * n + t] : (S)0;
  }
  if (tid < NB) hacc[tid] = 0;
  // hv[v] = <U_v, w> (v < NB) and, with ww, hv[NB] = <w, w>
  auto dots = [&](bool ww) {
    S acc[NB + 1];
#pragma unroll
    for (int v = 0; v <= NB; ++v) acc[v] = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
#pragma unroll
      for (int v = 0; v < NB; ++v) acc[v] += u[v][k] * x[k];
      acc[NB] += x[k] * x[k];
    }
#pragma unroll
    for (int v = 0; v <= NB; ++v) {
      const S sv = warp_sum_t<S>(acc[v]);
      if (lane == 0 && (v < NB || ww)) red[wid][v] = sv;
    }
    finish_sums<S>(NB + (ww ? 1 : 0), red, hv);
  };
  auto update = [&]() {
    S h[NB];
#pragma unroll
    for (int v = 0; v < NB; ++v) h[v] = hv[v];
    S sq = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
#pragma unroll
      for (int v = 0; v < NB; ++v) x[k] -= h[v] * u[v][k];
      sq += x[k] * x[k];
    }
    if (tid < NB) hacc[tid] += hv[tid];
    sq = warp_sum_t<S>(sq);
    if (lane == 0) red[wid][0] = sq;
    finish_sums<S>(1, red, nv);
  };
  dots(true);
  const S before = hv[NB];
  update();
  if (nv[0] < (S)0.5 * before) {
    dots(false);
    update();
  }
  const S nrm = sqrt(nv[0]);
  const S inv = nrm > (S)0 ? (S)1 / nrm : (S)0;
  S su = 0;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int t = tid + k * nt;
    if (t < n) {
      const S y = x[k] * inv;
      w[t] = y;
      su += y;
    }
  }
  if (usum) {
    su = warp_sum_t<S>(su);
    if (lane == 0) red[wid][0] = su;
    finish_sums<S>(1, red, nv + 1);
    if (tid == 0) *usum = usum_scale * (double)nv[1];
  }
  if (tid == 0) small_givens<S>(Hs, ldh, j, cs, sn, gvec, hacc, nrm);
}

template <typename S>
__global__ void __launch_bounds__(kSmallThreads) k_small_finish(const S* __restrict__ U, int n, int k,
                                                                 const double* __restrict__ Hs, int ldh,
                                                                 const double* __restrict__ gvec,
                                                                 double* __restrict__ x, int project_mean) {
  __shared__ S red[32][kSmallMaxBasis + 1];
  __shared__ S y[kSmallMaxBasis], out[1];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) {
    for (int i = k - 1; i >= 0; --i) {
      S t = (S)gvec[i];
      for (int l = i + 1; l < k; ++l) t -= (S)Hs[(size_t)l * ldh + i] * y[l];
      const S d = (S)Hs[(size_t)i * ldh + i];
      y[i] = d != (S)0 ? t / d : (S)0;
    }
  }
  __syncthreads();
  auto combo = [&](int t) {
    S v = 0;
    if (k <= kSmallRegBasis) {
      S u[kSmallRegBasis];
#pragma unroll
      for (int l = 0; l < kSmallRegBasis; ++l) u[l] = l < k ? U[(size_t)l * n + t] : (S)0;
#pragma unroll
      for (int l = 0; l < kSmallRegBasis; ++l)
        if (l < k) v += y[l] * u[l];
    } else {
      for (int l = 0; l < k; ++l) v += y[l] * U[(size_t)l * n + t];
    }
    return v;
  };
  auto mean_of = [&](S s) {
    s = warp_sum_t<S>(s);
    if (lane == 0) red[wid][0] = s;
    finish_sums<S>(1, red, out);
    return (double)out[0] / n;
  };
  if (n <= 4 * nt) {
    // short vectors (the inner Schur GMRES of a few thousand blobs): the
    // combination stays in registers until the mean is known, x is written once
    S v[4];
    S s = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int t = tid + q * nt;
      v[q] = t < n ? combo(t) : (S)0;
      s += v[q];
    }
    const double mean = project_mean ? mean_of(s) : 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int t = tid + q * nt;
      if (t < n) x[t] = project_mean ? (double)v[q] - mean : (double)v[q];
    }
    return;
  }
  S s = 0;
  for (int t = tid; t < n; t += nt) {
    const S v = combo(t);
    x[t] = (double)v;
    s += v;
  }
  if (project_mean) {
    const double mean = mean_of(s);
    for (int t = tid; t < n; t += nt) x[t] -= mean;
  }
}

}  // namespace

void launch_multidot(const double* V, size_t ldv, int nvec, const double* w, size_t n, double* partial,
                     cudaStream_t s, const double* gate, const DotTail* tail) {
  const DotTail t = tail ? *tail : DotTail{};
  if (nvec < 1 || nvec > kDotGroup) return;
  prof_begin(P_DOT, s);
  switch (nvec) {
#define IBRD_CASE(k) \
  case k: k_multidot<k><<<kRedBlocks, kRedThreads, 0, s>>>(V, ldv, w, n, partial, gate, t); break;
    IBRD_CASE(1) IBRD_CASE(2) IBRD_CASE(3) IBRD_CASE(4) IBRD_CASE(5) IBRD_CASE(6) IBRD_CASE(7) IBRD_CASE(8)
#undef IBRD_CASE
    default: return;
  }
  prof_end(P_DOT, s, "multidot", 8.0 * (nvec + 1) * n);
}

void launch_multidot(const float* V, size_t ldv, int nvec, const float* w, size_t n, double* partial,
                     cudaStream_t s, const double* gate, const DotTail* tail) {
  const DotTail t = tail ? *tail : DotTail{};
  if (nvec < 1 || nvec > kDotGroup) return;
  if (ldv % 4 != 0 || !aligned16(V) || !aligned16(w)) throw CudaError{cudaErrorMisalignedAddress, "multidot_f32"};
  prof_begin(P_DOT, s);
  switch (nvec) {
#define IBRD_CASE(k) \
  case k: k_multidot_f32<k><<<kRedBlocks, kRedThreads, 0, s>>>(V, ldv, w, n, partial, gate, t); break;
    IBRD_CASE(1) IBRD_CASE(2) IBRD_CASE(3) IBRD_CASE(4) IBRD_CASE(5) IBRD_CASE(6) IBRD_CASE(7) IBRD_CASE(8)
#undef IBRD_CASE
    default: return;
  }
  prof_end(P_DOT, s, "multidot_f32", 4.0 * (nvec + 1) * n);
}

void launch_reduce_partials(const double* partial, int nvec, double* out, cudaStream_t s, const double* gate,
                            const double* scale, int nscale) {
  if (nvec <= 0) return;
  prof_begin(P_REDUCE, s);
  k_reduce_partials<<<nvec, kRedThreads, 0, s>>>(partial, out, gate, scale, scale ? nscale : 0);
  prof_end(P_REDUCE, s, "reduce_partials");
}

void launch_gs_norm_estimate(const double* h, int nb, double* ww, double* hhat, double* hinv, cudaStream_t s) {
  prof_begin(P_SMALL, s);
  k_gs_norm_estimate<<<1, 32, 0, s>>>(h, nb, ww, hhat, hinv);
  prof_end(P_SMALL, s, "gs_norm_estimate");
}

void launch_gs_norm_fix(const double* rho2, const double* hhat, double* hsub, double* vscale, double* sq,
                        cudaStream_t s) {
  prof_begin(P_SMALL, s);
  k_gs_norm_fix<<<1, 32, 0, s>>>(rho2, hhat, hsub, vscale, sq);
  prof_end(P_SMALL, s, "gs_norm_fix");
}

void launch_gs_norm_unit(const double* sq, double* hsub, double* vscale, cudaStream_t s) {
  prof_begin(P_SMALL, s);
  k_gs_norm_unit<<<1, 32, 0, s>>>(sq, hsub, vscale);
  prof_end(P_SMALL, s, "gs_norm_unit");
}

void launch_multi_axpy(double* w, const double* V, size_t ldv, int nvec, const double* coef, double sign, size_t n,
                       double* partial_sq, cudaStream_t s, const double* gate, const double* cscale,
                       const double* post, const AxpyTail* tail) {
  const AxpyTail t = (tail && partial_sq) ? *tail : AxpyTail{};
  if (nvec < 1 || nvec > kDotGroup) return;
  prof_begin(P_AXPY, s);
  if (partial_sq) {
    switch (nvec) {
#define IBRD_CASE(k)                                                                                     \
  case k:                                                                                                \
    k_multi_axpy<k, true><<<kRedBlocks, kRedThreads, 0, s>>>(w, V, ldv, coef, sign, n, partial_sq, gate, \
                                                             cscale, post, t);                           \
    break;
      IBRD_CASE(1) IBRD_CASE(2) IBRD_CASE(3) IBRD_CASE(4) IBRD_CASE(5) IBRD_CASE(6) IBRD_CASE(7) IBRD_CASE(8)
#undef IBRD_CASE
      default: return;
    }
  } else {
    switch (nvec) {
#define IBRD_CASE(k)                                                                                      \
  case k:                                                                                                 \
    k_multi_axpy<k, false><<<kRedBlocks, kRedThreads, 0, s>>>(w, V, ldv, coef, sign, n, nullptr, gate,   \
                                                              cscale, post, t);                           \
    break;
      IBRD_CASE(1) IBRD_CASE(2) IBRD_CASE(3) IBRD_CASE(4) IBRD_CASE(5) IBRD_CASE(6) IBRD_CASE(7) IBRD_CASE(8)
#undef IBRD_CASE
      default: return;
    }
  }
  prof_end(P_AXPY, s, "multi_axpy", 8.0 * (nvec + 2) * n);
}

void launch_multi_axpy(float* w, const float* V, size_t ldv, int nvec, const double* coef, double sign, size_t n,
                       double* partial_sq, cudaStream_t s, const double* gate, const double* cscale,
                       const double* post, const AxpyTail* tail) {
  const AxpyTail t = (tail && partial_sq) ? *tail : AxpyTail{};
  if (nvec < 1 || nvec > kDotGroup) return;
  if (ldv % 4 != 0 || !aligned16(V) || !aligned16(w)) throw CudaError{cudaErrorMisalignedAddress, "multi_axpy_f32"};
  prof_begin(P_AXPY, s);
  if (partial_sq) {
    switch (nvec) {
#define IBRD_CASE(k)                                                                                           \
  case k:                                                                                                      \
    k_multi_axpy_f32<k, true><<<kRedBlocks, kRedThreads, 0, s>>>(w, V, ldv, coef, sign, n, partial_sq, gate, \
                                                                 cscale, post, t);                           \
    break;
      IBRD_CASE(1) IBRD_CASE(2) IBRD_CASE(3) IBRD_CASE(4) IBRD_CASE(5) IBRD_CASE(6) IBRD_CASE(7) IBRD_CASE(8)
#undef IBRD_CASE
      default: return;
    }
  } else {
    switch (nvec) {
#define IBRD_CASE(k)                                                                                            \
  case k:                                                                                                       \
    k_multi_axpy_f32<k, false><<<kRedBlocks, kRedThreads, 0, s>>>(w, V, ldv, coef, sign, n, nullptr, gate, \
                                                                  cscale, post, t);                          \
    break;
      IBRD_CASE(1) IBRD_CASE(2) IBRD_CASE(3) IBRD_CASE(4) IBRD_CASE(5) IBRD_CASE(6) IBRD_CASE(7) IBRD_CASE(8)
#undef IBRD_CASE
      default: return;
    }
  }
  prof_end(P_AXPY, s, "multi_axpy_f32", 4.0 * (nvec + 2) * n);
}

void launch_givens(double* H, int ldh, int j, double* cs, double* sn, double* gvec, double* res, cudaStream_t s) {
  prof_begin(P_SMALL, s);
  k_givens<<<1, 32, 0, s>>>(H, ldh, j, cs, sn, gvec, res);
  prof_end(P_SMALL, s, "givens");
}

void launch_backsolve(const double* H, int ldh, int k, const double* gvec, double* y, cudaStream_t s) {
  prof_begin(P_SMALL, s);
  k_backsolve<<<1, 32, 0, s>>>(H, ldh, k, gvec, y);
  prof_end(P_SMALL, s, "backsolve");
}

void launch_vec_add_small(double* h, const double* h2, int n, cudaStream_t s, const double* gate) {
  prof_begin(P_SMALL, s);
  k_vec_add_small<<<1, 64, 0, s>>>(h, h2, n, gate);
  prof_end(P_SMALL, s, "vec_add_small");
}

void launch_reorth_flag(const double* ww, const double* sq, double eta, double* flag, double* count, cudaStream_t s) {
  prof_begin(P_SMALL, s);
  k_reorth_flag<<<1, 32, 0, s>>>(ww, sq, eta, flag, count);
  prof_end(P_SMALL, s, "reorth_flag");
}

void launch_sqrt_scalar(const double* src, double* dst, cudaStream_t s) {
  prof_begin(P_SMALL, s);
  k_sqrt_scalar<<<1, 32, 0, s>>>(src, dst);
  prof_end(P_SMALL, s, "sqrt_scalar");
}

template <typename S>
void launch_small_start(const double* r, S* U0, int n, double* gvec, int m, double* usum, double usum_scale,
                        cudaStream_t s) {
  prof_begin(P_SMALL, s);
  k_small_start<S><<<1, kSmallThreads, 0, s>>>(r, U0, n, gvec, m, usum, usum_scale);
  prof_end(P_SMALL, s, "small_start");
}

template <typename S>
void launch_small_arnoldi(S* U, int n, int j, double* Hs, int ldh, double* cs, double* sn, double* gvec,
                          const double* wshift, double* usum, double usum_scale, cudaStream_t s) {
  if (j + 2 > kSmallMaxBasis) throw CudaError{cudaErrorInvalidValue, "small_arnoldi: basis too large"};
  prof_begin(P_SMALL, s);
  // registers: up to 6 FP32 or 5 FP64 basis vectors of 4 entries per thread
  constexpr int kMaxRegBasis = sizeof(S) == 4 ? 6 : 5;
  if (n <= 4 * kSmallThreads && j + 1 <= kMaxRegBasis) {
    switch (j + 1) {
#define IBRD_CASE(k)                                                                                           \
  case k:                                                                                                      \
    if constexpr (k <= kMaxRegBasis)                                                                           \
      k_small_arnoldi_r<S, k><<<1, kSmallThreads, 0, s>>>(U, n, Hs, ldh, cs, sn, gvec, wshift, usum, usum_scale); \
    break;
      IBRD_CASE(1) IBRD_CASE(2) IBRD_CASE(3) IBRD_CASE(4) IBRD_CASE(5) IBRD_CASE(6)
#undef IBRD_CASE
    }
  } else {
    k_small_arnoldi<S><<<1, kSmallThreads, 0, s>>>(U, n, j, Hs, ldh, cs, sn, gvec, wshift, usum, usum_scale);
  }
  prof_end(P_SMALL, s, "small_arnoldi");
}

template <typename S>
void launch_small_finish(const S* U, int n, int k, const double* Hs, int ldh, const double* gvec, double* x,
                         int project_mean, cudaStream_t s) {
  if (k > kSmallMaxBasis) throw CudaError{cudaErrorInvalidValue, "small_finish: basis too large"};
  prof_begin(P_SMALL, s);
  k_small_finish<S><<<1, kSmallThreads, 0, s>>>(U, n, k, Hs, ldh, gvec, x, project_mean);
  prof_end(P_SMALL, s, "small_finish");
}

#define IBRD_INST(S)                                                                                          \
  template void launch_small_start<S>(const double*, S*, int, double*, int, double*, double, cudaStream_t);   \
  template void launch_small_arnoldi<S>(S*, int, int, double*, int, double*, double*, double*, const double*, \
                                        double*, double, cudaStream_t);                                       \
  template void launch_small_finish<S>(const S*, int, int, const double*, int, const double*, double*, int,   \
                                       cudaStream_t);
IBRD_INST(double)
IBRD_INST(float)
#undef IBRD_INST

}  // namespace ibrd
