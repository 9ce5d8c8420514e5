// Multigrid smoother and transfer kernels (Sec. III.E: geometric multigrid for
// the Helmholtz problem A = alpha I - chi L, used as a preconditioner).
//
// Red-black Gauss-Seidel: red cells have (i + j + k) even. A full sweep
// updates every red cell from the old black values, then every black cell
// from the new red values.
//
// k_rb_sweep does a full sweep in ONE pass over memory. A CTA owns a TX x TY
// column of cells and marches in z through a chunk of ZC planes with a ring of
// four planes in shared memory (tile plus a 2-cell halo). At plane step k it
// updates the red cells of plane k on the tile plus a 1-cell ring (the ring
// values duplicate what the neighbouring CTA computes, bit for bit), then the
// black cells of plane k-1 on the tile, whose red neighbours are now final,
// and writes plane k-1. The sweep is out of place (x_in -> x_out), so every
// CTA reads old values only and no CTA waits on another. HBM traffic per
// sweep: one read of x, one read of b, one write of x.
#include <climits>
#include <cmath>

#include "internal.h"

namespace ibrd {
namespace {

__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Ring depth (planes) of the pipelined sweep, for x and for b.
constexpr int kSweepR = 8;

// 16-byte vectors: V values per vector.
template <typename T>
struct Vec;
template <>
struct Vec<float> {
  using type = float4;
  static constexpr int V = 4;
};
template <>
struct Vec<double> {
  using type = double2;
  static constexpr int V = 2;
};

template <typename T, int TX, int TY>
constexpr size_t sweep_smem() {
  constexpr int V = Vec<T>::V;
  return sizeof(T) * (size_t)kSweepR * ((TY + 4) + (TY + 2)) * (TX + 2 * V);
}

template <typename T>
__device__ __forceinline__ T vget(const typename Vec<T>::type& v, int c);
template <>
__device__ __forceinline__ float vget<float>(const float4& v, int c) {
  return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
}
template <>
__device__ __forceinline__ double vget<double>(const double2& v, int c) {
  return c == 0 ? v.x : v.y;
}
template <typename T>
__device__ __forceinline__ void vset(typename Vec<T>::type& v, int c, T x);
template <>
__device__ __forceinline__ void vset<float>(float4& v, int c, float x) {
  if (c == 0) v.x = x;
  else if (c == 1) v.y = x;
  else if (c == 2) v.z = x;
  else v.w = x;
}
template <>
__device__ __forceinline__ void vset<double>(double2& v, int c, double x) {
  if (c == 0) v.x = x;
  else v.y = x;
}

// Update of one 16-byte group whose active cells (those of the colour being
// updated) are q = A and q = A + 2 (float4) or q = A (double2); the other
// cells keep c. xo is the neighbour beyond the group's end on the side the
// active cells need: the left one when A = 0, the right one when A = 1.
template <int A>
__device__ __forceinline__ float4 rb_group(float4 c, float xo, float4 u, float4 dn, float4 zm, float4 zp, float4 bb,
                                           float sh, float off, float inv) {
  float4 o = c;
  if (A == 0) {
    o.x = ((bb.x - sh) + off * (((xo + c.y) + (u.x + dn.x)) + (zm.x + zp.x))) * inv;
    o.z = ((bb.z - sh) + off * (((c.y + c.w) + (u.z + dn.z)) + (zm.z + zp.z))) * inv;
  } else {
    o.y = ((bb.y - sh) + off * (((c.x + c.z) + (u.y + dn.y)) + (zm.y + zp.y))) * inv;
    o.w = ((bb.w - sh) + off * (((c.z + xo) + (u.w + dn.w)) + (zm.w + zp.w))) * inv;
  }
  return o;
}
template <int A>
__device__ __forceinline__ double2 rb_group(double2 c, double xo, double2 u, double2 dn, double2 zm, double2 zp,
                                            double2 bb, double sh, double off, double inv) {
  double2 o = c;
  if (A == 0)
    o.x = ((bb.x - sh) + off * (((xo + c.y) + (u.x + dn.x)) + (zm.x + zp.x))) * inv;
  else
    o.y = ((bb.y - sh) + off * (((c.x + xo) + (u.y + dn.y)) + (zm.y + zp.y))) * inv;
  return o;
}

// Plane layout in shared memory: x planes hold rows y0-2 .. y0+TY+1, b planes
// rows y0-1 .. y0+TY; both hold columns x0-V .. x0+TX+V-1 (local column
// lx = x - x0 + V), so every row starts on a 16-byte boundary and every copy,
// including the periodic wrap at the domain edge, is one aligned 16-byte
// cp.async.
//
// Schedule: phase p updates the red cells of plane p (tile + ring) AND the
// black cells of plane p-2 (tile), then stores plane p-2. The two touch
// disjoint cells: red(p) reads planes p-1..p+1 and writes red cells of p;
// black(p-2) reads red cells of planes p-3..p-1, all final by phase p-1, and
// writes black cells of p-2. So one barrier per plane suffices. Warps 0-5
// own the red groups, warps 6-9 the black groups.
//
// Copies: group G_q = {x plane q+1, b plane q} is needed by red(q); it is
// issued right after the barrier of phase q-3 (prefetch distance 3). With
// rings of 8 planes its target slots are not read during that phase.
constexpr int kSweepThreads = 320;

template <typename T, int TX, int TY, bool ZERO>
__global__ void __launch_bounds__(kSweepThreads) k_rb_sweep(const T* __restrict__ xin, T* __restrict__ xout,
                                                            const T* __restrict__ b,
                                                            const double* __restrict__ bshift, int nx, int ny,
                                                            int nz, int zc, T inv_diag, T off,
                                                            double* __restrict__ part) {
  using VT = typename Vec<T>::type;
  constexpr int V = Vec<T>::V;
  constexpr int NT = kSweepThreads;
  constexpr int W = TX + 2 * V;            // row length (values)
  constexpr int NV = W / V;                // vectors per row
  constexpr int XR = TY + 4, BR = TY + 2;  // rows per x / b plane
  constexpr int TV = TX / V;
  constexpr int R = kSweepR;
  constexpr int BLK0 = 192;  // first thread of the black role (warp 6)
  static_assert(XR * NV <= 2 * NT && BR * NV <= NT, "copy roles");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* pxs = reinterpret_cast<T*>(smem_raw);
  T* pbs = pxs + R * XR * W;
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int k0 = blockIdx.z * zc, k1 = min(k0 + zc, nz);
  const size_t plane = (size_t)nx * ny;
  const T sh = bshift ? (T)(*bshift) : (T)0;

  // copy roles: x-plane vectors e = tid and tid + NT, b-plane vector e = tid
  int gx0 = -1, sx0 = 0, gx1 = -1, sx1 = 0, gb = -1, sb = 0;
  {
    int e = tid;
    if (e < XR * NV) {
      const int r = e / NV, v = e - r * NV;
      gx0 = wrap(y0 - 2 + r, ny) * nx + wrap(x0 - V + v * V, nx);
      sx0 = r * W + v * V;
    }
    e = tid + NT;
    if (e < XR * NV) {
      const int r = e / NV, v = e - r * NV;
      gx1 = wrap(y0 - 2 + r, ny) * nx + wrap(x0 - V + v * V, nx);
      sx1 = r * W + v * V;
    }
    if (tid < BR * NV) {
      const int r = tid / NV, v = tid - r * NV;
      gb = wrap(y0 - 1 + r, ny) * nx + wrap(x0 - V + v * V, nx);
      sb = r * W + v * V;
    }
  }
  // update roles. Each warp takes rows of one parity only, so the pattern of
  // active cells in a group is the same for all its lanes: warps 0-2 the red
  // groups of rows 1, 3, .., warps 3-5 those of rows 2, 4, ..; warps 6-7 the
  // black groups of rows 2, 4, .., warps 8-9 those of rows 3, 5, ...
  static_assert(TY % 2 == 0 && (TY + 2) / 2 * NV <= 96 && TY / 2 * TV <= 64, "row-parity roles");
  bool is_red = false, is_black = false;
  int go = 0, gpar = 0;
  bool lo_edge = false, hi_edge = false;
  T* gout = xout;
  if (tid < BLK0) {
    const int h = tid / 96, e = tid - h * 96;
    const int r = 2 * (e / NV) + h, v = e - (e / NV) * NV;
    is_red = e < (TY + 2) / 2 * NV;
    const int ly = 1 + r;
    go = ly * W + v * V;
    gpar = (x0 + y0 + ly) & 1;
    lo_edge = v == 0;
    hi_edge = v == NV - 1;
  } else {
    const int e = tid - BLK0;
    const int h = e / 64, f = e - h * 64;
    const int ty = 2 * (f / TV) + h, v = 1 + (f - (f / TV) * TV);
    is_black = f < TY / 2 * TV;
    go = (2 + ty) * W + v * V;
    gpar = (x0 + y0 + 2 + ty) & 1;
    gout = xout + (size_t)(y0 + ty) * nx + x0 + (v - 1) * V;
  }

  auto slot_x = [&](int k) { return pxs + (k & (R - 1)) * (XR * W); };
  auto slot_b = [&](int k) { return pbs + (k & (R - 1)) * (BR * W); };
  auto copy_x = [&](int k) {
    const T* src = xin + (size_t)wrap(k, nz) * plane;
    T* dst = slot_x(k);
    if (gx0 >= 0) {
      if (ZERO)
        *reinterpret_cast<VT*>(dst + sx0) = VT{};
      else
        cp_async16(dst + sx0, src + gx0);
    }
    if (gx1 >= 0) {
      if (ZERO)
        *reinterpret_cast<VT*>(dst + sx1) = VT{};
      else
        cp_async16(dst + sx1, src + gx1);
    }
  };
  auto copy_b = [&](int k) {
    if (gb >= 0) cp_async16(slot_b(k) + sb, b + (size_t)wrap(k, nz) * plane + gb);
  };
  // Group update for plane k (colour 0 = red). zm, c, zp are this thread's
  // group in planes k-1, k, k+1: a role thread keeps the same (row, group)
  // in every phase, and the cells it needs there (the other colour) do not
  // change between the phase that read them and the phase that uses them,
  // so they rotate through registers and only plane k+1 is read anew.
  VT zm{}, c{}, zp{};
  auto group = [&](int k, int colour, bool first) -> VT {
    const T* P = slot_x(k);
    const T* B = slot_b(k);
    const int o = go;
    if (first) {
      zm = *reinterpret_cast<const VT*>(slot_x(k - 1) + o);
      c = *reinterpret_cast<const VT*>(P + o);
    } else {
      zm = c;
      c = zp;
    }
    zp = *reinterpret_cast<const VT*>(slot_x(k + 1) + o);
    const VT u = *reinterpret_cast<const VT*>(P + o - W);
    const VT dn = *reinterpret_cast<const VT*>(P + o + W);
    const VT bb = *reinterpret_cast<const VT*>(B + o - W);
    // warp-uniform: all lanes of a warp share the row parity
    const int a = (gpar + k + colour) & 1;
    VT r;
    if (a == 0)
      r = rb_group<0>(c, lo_edge ? (T)0 : P[o - 1], u, dn, zm, zp, bb, sh, off, inv_diag);
    else
      r = rb_group<1>(c, hi_edge ? (T)0 : P[o + V], u, dn, zm, zp, bb, sh, off, inv_diag);
    // ring edge groups of the red region hold one active cell each: lx = V-1
    // (last of group 0) and lx = TX+V (first of the last group)
    if (lo_edge) {
      VT t = c;
      vset<T>(t, V - 1, vget<T>(r, V - 1));
      r = t;
    }
    if (hi_edge) {
      VT t = c;
      vset<T>(t, 0, vget<T>(r, 0));
      r = t;
    }
    return r;
  };
  double xsum = 0.0;

  constexpr int D = 3;
  // prologue: x planes k0-2, k0-1 plus G_{k0-1} = {x(k0), b(k0-1)}, then
  // G_{k0} .. G_{k0+D-2}
  copy_x(k0 - 2);
  copy_x(k0 - 1);
  copy_x(k0);
  copy_b(k0 - 1);
  cp_async_commit();
  for (int q = k0; q <= k0 + D - 2; ++q) {
    if (q <= k1) {
      copy_x(q + 1);
      copy_b(q);
    }
    cp_async_commit();
  }
  for (int p = k0 - 1; p <= k1 + 1; ++p) {
    cp_async_wait<D - 1>();
    __syncthreads();
    // G_{p+D} is issued after the barrier: its slots (x plane p+D+1, b plane
    // p+D) are not among the planes any warp reads in phase p (x p-3..p+1,
    // b p-2 and p)
    const int q = p + D;
    if (q <= k1) {
      copy_x(q + 1);
      copy_b(q);
    }
    cp_async_commit();
    if (is_red && p <= k1) {
      const VT r = group(p, 0, p == k0 - 1);
      *reinterpret_cast<VT*>(slot_x(p) + go) = r;
    }
    const int kb = p - 2;
    if (is_black && kb >= k0) {
      const VT r = group(kb, 1, kb == k0);
      *reinterpret_cast<VT*>(slot_x(kb) + go) = r;
      *reinterpret_cast<VT*>(gout + (size_t)kb * plane) = r;
      if (part) {
        T t = vget<T>(r, 0);
#pragma unroll
        for (int qq = 1; qq < V; ++qq) t += vget<T>(r, qq);
        xsum += (double)t;
      }
    }
  }
  if (part) {
    // deterministic CTA sum (fixed shuffle tree, then warp 0)
    __shared__ double ws[NT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) xsum += __shfl_down_sync(0xffffffffu, xsum, o);
    __syncthreads();
    if ((tid & 31) == 0) ws[tid >> 5] = xsum;
    __syncthreads();
    if (tid < 32) {
      double v = tid < NT / 32 ? ws[tid] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (tid == 0) part[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = v;
    }
  }
}

// Half sweep on one colour, in place, for small levels. Reads touch only
// cells of the other colour and writes only cells of this colour, so the
// read and write views of x never share an element.
template <typename T>
__global__ void __launch_bounds__(256) k_rb_half(const T* __restrict__ xr, T* __restrict__ xw,
                                                 const T* __restrict__ b, const double* __restrict__ bshift, int nx,
                                                 int ny, int nz, int zc, T inv_diag, T off, int colour, int zero) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int np = nx >> 1;
  if (p >= np || j >= ny) return;
  const int k0 = blockIdx.z * zc;
  const int k1 = min(k0 + zc, nz);
  const int plane = nx * ny;
  const int rj = j * nx, rjm = wrap(j - 1, ny) * nx, rjp = wrap(j + 1, ny) * nx;
  const T sh = bshift ? (T)(*bshift) : (T)0;
#pragma unroll 4
  for (int k = k0; k < k1; ++k) {
    const int ia = 2 * p + ((colour + j + k) & 1);
    const int base = k * plane;
    if (zero) {
      // first red half sweep from x = 0: red = b/diag, black = 0
      xw[base + rj + ia] = (b[base + rj + ia] - sh) * inv_diag;
      xw[base + rj + (ia ^ 1)] = (T)0;
      continue;
    }
    const T s = ((xr[base + rj + wrap(ia - 1, nx)] + xr[base + rj + wrap(ia + 1, nx)]) +
                 (xr[base + rjm + ia] + xr[base + rjp + ia])) +
                (xr[wrap(k - 1, nz) * plane + rj + ia] + xr[wrap(k + 1, nz) * plane + rj + ia]);
    xw[base + rj + ia] = ((b[base + rj + ia] - sh) + off * s) * inv_diag;
  }
}

// Coarse cell (I, J, K) gets the mean over its 8 children of b - shift - A x.
template <typename T>
__global__ void __launch_bounds__(256) k_resid_restrict(const T* __restrict__ x, const T* __restrict__ b,
                                                        const double* __restrict__ bshift, T* __restrict__ bc,
                                                        int nx, int ny, int nz, T diag, T off) {
  const int nxc = nx >> 1, nyc = ny >> 1, nzc = nz >> 1;
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int K = blockIdx.z * blockDim.z + threadIdx.z;
  if (I >= nxc || J >= nyc || K >= nzc) return;
  const int plane = nx * ny;
  const T sh = bshift ? (T)(*bshift) : (T)0;
  const int i0 = 2 * I, iw = wrap(i0 - 1, nx), ie = wrap(i0 + 2, nx);
  T acc = 0;
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const int k = 2 * K + c;
    const int pk = k * plane, pkm = wrap(k - 1, nz) * plane, pkp = wrap(k + 1, nz) * plane;
#pragma unroll
    for (int bb = 0; bb < 2; ++bb) {
      const int j = 2 * J + bb;
      const int rj = j * nx, rjm = wrap(j - 1, ny) * nx, rjp = wrap(j + 1, ny) * nx;
      const T xw = x[pk + rj + iw], xa = x[pk + rj + i0], xb = x[pk + rj + i0 + 1], xe = x[pk + rj + ie];
      const T ba = b[pk + rj + i0], bb2 = b[pk + rj + i0 + 1];
      const T sa = ((xw + xb) + (x[pk + rjm + i0] + x[pk + rjp + i0])) + (x[pkm + rj + i0] + x[pkp + rj + i0]);
      const T sb = ((xa + xe) + (x[pk + rjm + i0 + 1] + x[pk + rjp + i0 + 1])) +
                   (x[pkm + rj + i0 + 1] + x[pkp + rj + i0 + 1]);
      acc += ((ba - sh) - (diag * xa - off * sa)) + ((bb2 - sh) - (diag * xb - off * sb));
    }
  }
  bc[(K * nyc + J) * nxc + I] = acc * (T)0.125;
}

// The first red-black sweep from x = 0, FP32, as one 7-point stencil on b:
// a red cell gets r = (b - shift) / diag (its neighbours are still 0), a black
// cell ((b - shift) + off * (sum of the r of its 6 red neighbours)) / diag.
// Same arithmetic as the fused sweep; reads b once and writes x once. Four
// cells per thread (16-byte rows; nx % 4 == 0, aligned fields), z-march over
// zc planes with the neighbour planes' r in registers.
__global__ void __launch_bounds__(256) k_rb_zero_f32v(const float* __restrict__ b, float* __restrict__ x,
                                                      const double* __restrict__ bshift, int nx, int ny, int nz,
                                                      int zc, float inv, float off) {
  const int i4 = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i4 >= (nx >> 2) || j >= ny) return;
  const int k0 = blockIdx.z * zc;
  const int k1 = min(k0 + zc, nz);
  if (k0 >= k1) return;
  const float sh = bshift ? (float)(*bshift) : 0.f;
  const int i = 4 * i4;
  const int im = i == 0 ? nx - 1 : i - 1, ip = i + 4 == nx ? 0 : i + 4;
  const size_t plane = (size_t)nx * ny;
  const size_t rj = (size_t)j * nx, rjm = (size_t)(j == 0 ? ny - 1 : j - 1) * nx,
               rjp = (size_t)(j == ny - 1 ? 0 : j + 1) * nx;
  auto ldb = [&](size_t o) { return *reinterpret_cast<const float4*>(b + o); };
  auto red = [&](float4 t) {
    return make_float4((t.x - sh) * inv, (t.y - sh) * inv, (t.z - sh) * inv, (t.w - sh) * inv);
  };
  auto kw = [&](int k) { return (size_t)(k >= nz ? k - nz : k) * plane + rj + i; };
  float4 rm = red(ldb((size_t)(k0 == 0 ? nz - 1 : k0 - 1) * plane + rj + i));
  float4 b0 = ldb(kw(k0));
  float4 r0 = red(b0);
  // the next plane's centre row is loaded one iteration ahead (two rows in flight)
  float4 b1 = ldb(kw(k0 + 1));
  for (int k = k0; k < k1; ++k) {
    const size_t base = (size_t)k * plane;
    const float4 bp = b1;
    if (k + 1 < k1) b1 = ldb(kw(k + 2));
    const float4 rp = red(bp);
    const float4 ys = red(ldb(base + rjm + i)), yn = red(ldb(base + rjp + i));
    const float rl = (b[base + rj + im] - sh) * inv, rr = (b[base + rj + ip] - sh) * inv;
    const float bc[4] = {b0.x, b0.y, b0.z, b0.w}, rc[4] = {r0.x, r0.y, r0.z, r0.w};
    const float us[4] = {ys.x, ys.y, ys.z, ys.w}, un[4] = {yn.x, yn.y, yn.z, yn.w};
    const float zm[4] = {rm.x, rm.y, rm.z, rm.w}, zp[4] = {rp.x, rp.y, rp.z, rp.w};
    float o[4];
    const int par = (j + k) & 1;  // parity of element 0 (i is a multiple of 4)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float L = q == 0 ? rl : rc[q - 1], R = q == 3 ? rr : rc[q + 1];
      const float blk = ((bc[q] - sh) + off * (((L + R) + (us[q] + un[q])) + (zm[q] + zp[q]))) * inv;
      o[q] = ((q + par) & 1) ? blk : rc[q];
    }
    *reinterpret_cast<float4*>(x + base + rj + i) = make_float4(o[0], o[1], o[2], o[3]);
    rm = r0;
    b0 = bp;
    r0 = rp;
  }
}

// One pre-smoothing sweep from x = 0 followed by the residual restriction,
// FP32, in one pass: x = first red-black sweep of A x = b - shift (the
// stencil of k_rb_zero_f32v) and bc = mean over the 8 children of
// b - shift - A x. A CTA of 8 x TX4 threads owns a tile of 8 rows x 4 TX4
// cells (one 4-vector per thread) and marches in z over zc planes (zc even,
// chunks start on even planes). b planes (the tile with a halo of 2 vectors
// in x and 2 rows in y) arrive in a ring of 8 by 16-byte cp.async, kZR_D
// planes ahead of use; x (tile with a halo of 1 vector and 1 row) is formed in
// a ring of 4. Phase p forms x on plane p+1 and, in the same phase, the
// residual on plane p-1 (it reads x planes p-2 .. p, formed in earlier
// phases), so one barrier per plane suffices; it writes x of plane p-1 and,
// when p-1 is odd, the coarse cells of planes (p-2, p-1): x pairs within a
// thread, y pairs across lanes TX4 apart, z pairs in registers.
// Needs nx % (4 TX4) == 0, ny % 8 == 0, nz even.
constexpr int kZR_D = 4;

template <int TX4>
__global__ void __launch_bounds__(TX4 * 8) k_zero_restrict_f32(const float* __restrict__ b,
                                                               const double* __restrict__ bshift,
                                                               float* __restrict__ x, float* __restrict__ bc, int nx,
                                                               int ny, int nz, int zc, float inv, float off,
                                                               float diag) {
  constexpr int TY = 8, NT = TX4 * TY, RB = 8, D = kZR_D;
  constexpr int BW4 = TX4 + 4, BH = TY + 4;  // b tile (4-vectors), halo 2 vectors / 2 rows
  constexpr int XW4 = TX4 + 2, XH = TY + 2;  // x tile, halo 1 vector / 1 row
  constexpr int NB = BH * BW4, NX = XH * XW4;
  constexpr int QB = (NB + NT - 1) / NT, QX = (NX + NT - 1) / NT;
  static_assert(QB <= 3 && QX <= 2 && 32 % TX4 == 0 && D + 3 <= RB, "roles");
  extern __shared__ __align__(16) float4 zr_smem[];
  float4* BSM = zr_smem;           // RB planes of NB raw b values
  float4* XSM = zr_smem + RB * NB;  // 4 planes of NX x values
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX4 + tx;
  const int x0 = blockIdx.x * 4 * TX4, y0 = blockIdx.y * TY;
  const int k0 = blockIdx.z * zc;
  const int k1 = min(k0 + zc, nz);
  if (k0 >= k1) return;
  const float sh = bshift ? (float)(*bshift) : 0.f;
  const size_t plane = (size_t)nx * ny;
  auto wz = [&](int p) { return p < 0 ? p + nz : (p >= nz ? p - nz : p); };
  // x ring slots follow the unwrapped plane index (k0 - 1 <= p <= k1), so
  // consecutive planes never share a slot at the periodic seam
  auto xslot = [](int p) { return p & 3; };
  auto bslot = [&](int p) { return BSM + (p & (RB - 1)) * NB; };
  // this thread's b copies: in-plane offsets (periodic)
  int boff[QB];
  bool bval[QB];
#pragma unroll
  for (int q = 0; q < QB; ++q) {
    const int e = tid + q * NT;
    bval[q] = e < NB;
    const int row = e / BW4, c4 = e - row * BW4;
    boff[q] = bval[q] ? wrap(y0 - 2 + row, ny) * nx + wrap(x0 - 8 + 4 * c4, nx) : 0;
  }
  // this thread's x entries: position in the b tile and parity of element 0
  int xob[QX], xpar[QX];
  bool xval[QX];
#pragma unroll
  for (int q = 0; q < QX; ++q) {
    const int e = tid + q * NT;
    xval[q] = e < NX;
    const int row = e / XW4, c4 = e - row * XW4;
    xob[q] = (row + 1) * BW4 + c4 + 1;
    xpar[q] = ((x0 - 4 + 4 * c4) + (y0 - 1 + row)) & 1;  // the even-period wrap keeps parity
  }
  // b plane p into its ring slot (one commit group per plane)
  auto copy_b = [&](int p) {
    const float* bp = b + (size_t)wz(p) * plane;
    float4* dst = bslot(p);
#pragma unroll
    for (int q = 0; q < QB; ++q)
      if (bval[q]) cp_async16(dst + tid + q * NT, bp + boff[q]);
    cp_async_commit();
  };
  auto el = [](const float4& v, int e) { return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w)); };
  // x on plane p: red cells r = (b - shift) / diag, black cells one update
  // from their red neighbours (same expression as the other sweep kernels)
  auto comp_x = [&](int p) {
    const float4 *Bc = bslot(p), *Bm = bslot(p - 1), *Bp = bslot(p + 1);
    float4* xs = XSM + xslot(p) * NX;
    const int pp = wz(p) & 1;
#pragma unroll
    for (int q = 0; q < QX; ++q) {
      if (!xval[q]) continue;
      const int o = xob[q];
      const float4 c = Bc[o], u = Bc[o - BW4], dn = Bc[o + BW4], zm = Bm[o], zp = Bp[o];
      const float lw = Bc[o - 1].w, rx = Bc[o + 1].x;
      auto r = [&](float v) { return (v - sh) * inv; };
      float out[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float ce = el(c, e) - sh;
        if (((xpar[q] + e + pp) & 1) == 0) {
          out[e] = ce * inv;
        } else {
          const float L = r(e == 0 ? lw : el(c, e - 1)), R = r(e == 3 ? rx : el(c, e + 1));
          const float sum = ((L + R) + (r(el(u, e)) + r(el(dn, e)))) + (r(el(zm, e)) + r(el(zp, e)));
          out[e] = (ce + off * sum) * inv;
        }
      }
      xs[tid + q * NT] = make_float4(out[0], out[1], out[2], out[3]);
    }
  };
  // prologue: b planes k0 - 2 .. k0 + D + 1 in flight; x planes k0 - 1, k0
  for (int p = k0 - 2; p <= k0 + D + 1; ++p) copy_b(p);
  cp_async_wait<D>();  // planes up to k0 + 1 landed
  __syncthreads();
  comp_x(k0 - 1);
  comp_x(k0);
  float acc0 = 0.f, acc1 = 0.f;  // coarse sums over the even plane (threads with even ty)
  const int ox = (ty + 1) * XW4 + tx + 1;  // this thread's tile group in the x ring
  const int ob = (ty + 2) * BW4 + tx + 2;  // and in the b ring
  const int nxc = nx >> 1, nyc = ny >> 1;
  for (int p = k0; p <= k1; ++p) {
    // b plane p + 2 landed; planes p + 3 .. p + D + 1 may still be in flight
    cp_async_wait<D - 1>();
    __syncthreads();
    // plane p + D + 2 takes the slot of plane p + D - 6, last read in phase
    // p - 1 (ring planes in use: p - 1 .. p + D + 2)
    if (p + D + 2 <= k1 + 1)
      copy_b(p + D + 2);
    else
      cp_async_commit();  // keep one group per phase
    if (p + 1 <= k1) comp_x(p + 1);
    const int k = p - 1;
    if (k < k0) continue;
    const float4* xm = XSM + xslot(k - 1) * NX;
    const float4* xc = XSM + xslot(k) * NX;
    const float4* xp = XSM + xslot(k + 1) * NX;
    const float4 c = xc[ox], u = xc[ox - XW4], dn = xc[ox + XW4], zm = xm[ox], zp = xp[ox];
    const float lw = xc[ox - 1].w, rx = xc[ox + 1].x;
    const float4 bb = bslot(k)[ob];
    float res[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float L = e == 0 ? lw : el(c, e - 1), R = e == 3 ? rx : el(c, e + 1);
      const float sum = ((L + R) + (el(u, e) + el(dn, e))) + (el(zm, e) + el(zp, e));
      res[e] = (el(bb, e) - sh) - (diag * el(c, e) - off * sum);
    }
    *reinterpret_cast<float4*>(x + (size_t)k * plane + (size_t)(y0 + ty) * nx + x0 + 4 * tx) = c;
    // x pairs in the thread, y pairs across lanes TX4 apart (same warp)
    float p0 = res[0] + res[1], p1 = res[2] + res[3];
    p0 += __shfl_down_sync(0xffffffffu, p0, TX4);
    p1 += __shfl_down_sync(0xffffffffu, p1, TX4);
    if ((ty & 1) == 0) {
      if ((k & 1) == 0) {
        acc0 = p0;
        acc1 = p1;
      } else {
        float* dst = bc + ((size_t)(k >> 1) * nyc + ((y0 + ty) >> 1)) * nxc + (x0 >> 1) + 2 * tx;
        *reinterpret_cast<float2*>(dst) = make_float2((acc0 + p0) * 0.125f, (acc1 + p1) * 0.125f);
      }
    }
  }
  cp_async_wait<0>();
}

// Thread per coarse cell: adds the trilinear cell-centred interpolation of
// the coarse correction to its 8 fine children (weights 3/4, 1/4 per axis).
template <typename T>
__global__ void __launch_bounds__(256) k_prolong8(const T* __restrict__ xc, T* __restrict__ x, int nx, int ny,
                                                  int nz) {
  const int nxc = nx >> 1, nyc = ny >> 1, nzc = nz >> 1;
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int K = blockIdx.z * blockDim.z + threadIdx.z;
  if (I >= nxc || J >= nyc || K >= nzc) return;
  const int Ix[3] = {wrap(I - 1, nxc), I, wrap(I + 1, nxc)};
  const int Jy[3] = {wrap(J - 1, nyc), J, wrap(J + 1, nyc)};
  const int Kz[3] = {wrap(K - 1, nzc), K, wrap(K + 1, nzc)};
  T c[3][3][3];  // [z][y][x] coarse neighbourhood
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const T* row = xc + (Kz[a] * nyc + Jy[r]) * nxc;
#pragma unroll
      for (int q = 0; q < 3; ++q) c[a][r][q] = row[Ix[q]];
    }
#pragma unroll
  for (int dz = 0; dz < 2; ++dz)
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
      const int k = 2 * K + dz, j = 2 * J + dy, o = dz ? 2 : 0, n = dy ? 2 : 0;
      // z, then y (parent plane / row first), then x, each axis scaled by 4
      T zy[3];
#pragma unroll
      for (int q = 0; q < 3; ++q)
        zy[q] = prolong_axis(prolong_axis(c[1][1][q], c[o][1][q]), prolong_axis(c[1][n][q], c[o][n][q]));
      T* dst = x + ((size_t)k * ny + j) * nx + 2 * I;
      dst[0] = prolong_add(dst[0], prolong_axis(zy[1], zy[0]));
      dst[1] = prolong_add(dst[1], prolong_axis(zy[1], zy[2]));
    }
}

// Two coarse cells (I, I+1) per thread: the fine x range 2I-1 .. 2I+4 of each
// row is one aligned 4-vector plus two scalars. Needs nx % 4 == 0.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 5 : 3) k_resid_restrict2(const T* __restrict__ x, const T* __restrict__ b,
                                                         const double* __restrict__ bshift, T* __restrict__ bc,
                                                         int nx, int ny, int nz, T diag, T off) {
  const int nxc = nx >> 1, nyc = ny >> 1, nzc = nz >> 1;
  const int I2 = blockIdx.x * blockDim.x + threadIdx.x;  // pair index
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int K = blockIdx.z * blockDim.z + threadIdx.z;
  if (2 * I2 >= nxc || J >= nyc || K >= nzc) return;
  const int plane = nx * ny;
  const T sh = bshift ? (T)(*bshift) : (T)0;
  const int i0 = 4 * I2, iw = wrap(i0 - 1, nx), ie = wrap(i0 + 4, nx);
  T acc0 = 0, acc1 = 0;
  auto ld4 = [&](int o, T* v) {
    if constexpr (sizeof(T) == 4) {
      const float4 t = *reinterpret_cast<const float4*>(x + o);
      v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else {
      const double2 t0 = *reinterpret_cast<const double2*>(x + o);
      const double2 t1 = *reinterpret_cast<const double2*>(x + o + 2);
      v[0] = t0.x; v[1] = t0.y; v[2] = t1.x; v[3] = t1.y;
    }
  };
  auto ldb4 = [&](int o, T* v) {
    if constexpr (sizeof(T) == 4) {
      const float4 t = *reinterpret_cast<const float4*>(b + o);
      v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else {
      const double2 t0 = *reinterpret_cast<const double2*>(b + o);
      const double2 t1 = *reinterpret_cast<const double2*>(b + o + 2);
      v[0] = t0.x; v[1] = t0.y; v[2] = t1.x; v[3] = t1.y;
    }
  };
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const int k = 2 * K + c;
    const int pk = k * plane, pkm = wrap(k - 1, nz) * plane, pkp = wrap(k + 1, nz) * plane;
#pragma unroll
    for (int bb = 0; bb < 2; ++bb) {
      const int j = 2 * J + bb;
      const int rj = j * nx, rjm = wrap(j - 1, ny) * nx, rjp = wrap(j + 1, ny) * nx;
      T m[4], yn[4], ys[4], zd[4], zu[4], bv[4];
      ld4(pk + rj + i0, m);
      ld4(pk + rjm + i0, ys);
      ld4(pk + rjp + i0, yn);
      ld4(pkm + rj + i0, zd);
      ld4(pkp + rj + i0, zu);
      ldb4(pk + rj + i0, bv);
      const T xw = x[pk + rj + iw], xe = x[pk + rj + ie];
      T r[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const T l = q == 0 ? xw : m[q - 1];
        const T rr = q == 3 ? xe : m[q + 1];
        const T s = ((l + rr) + (ys[q] + yn[q])) + (zd[q] + zu[q]);
        r[q] = (bv[q] - sh) - (diag * m[q] - off * s);
      }
      acc0 += r[0] + r[1];
      acc1 += r[2] + r[3];
    }
  }
  const int o = (K * nyc + J) * nxc + 2 * I2;
  bc[o] = acc0 * (T)0.125;
  bc[o + 1] = acc1 * (T)0.125;
}

// Two coarse cells (I, I+1) per thread; writes the 4 x 2 x 2 fine children
// with aligned 4-vector read-modify-writes. Needs nx % 4 == 0.
template <typename T>
__global__ void __launch_bounds__(256) k_prolong8x2(const T* __restrict__ xc, T* __restrict__ x, int nx, int ny,
                                                    int nz) {
  const int nxc = nx >> 1, nyc = ny >> 1, nzc = nz >> 1;
  const int I2 = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int K = blockIdx.z * blockDim.z + threadIdx.z;
  if (2 * I2 >= nxc || J >= nyc || K >= nzc) return;
  const int I = 2 * I2;
  const int Ix[4] = {wrap(I - 1, nxc), I, I + 1, wrap(I + 2, nxc)};
  const int Jy[3] = {wrap(J - 1, nyc), J, wrap(J + 1, nyc)};
  const int Kz[3] = {wrap(K - 1, nzc), K, wrap(K + 1, nzc)};
  T c[3][3][4];  // [z][y][x] coarse neighbourhood of the pair
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const T* row = xc + (Kz[a] * nyc + Jy[r]) * nxc;
#pragma unroll
      for (int q = 0; q < 4; ++q) c[a][r][q] = row[Ix[q]];
    }
#pragma unroll
  for (int dz = 0; dz < 2; ++dz)
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
      const int k = 2 * K + dz, j = 2 * J + dy, o = dz ? 2 : 0, n = dy ? 2 : 0;
      T* dst = x + ((size_t)k * ny + j) * nx + 4 * I2;
      // z, then y (parent plane / row first), then x, each axis scaled by 4:
      // fine cells 2I .. 2I+3
      T zy[4], v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        zy[q] = prolong_axis(prolong_axis(c[1][1][q], c[o][1][q]), prolong_axis(c[1][n][q], c[o][n][q]));
      v[0] = prolong_axis(zy[1], zy[0]);
      v[1] = prolong_axis(zy[1], zy[2]);
      v[2] = prolong_axis(zy[2], zy[1]);
      v[3] = prolong_axis(zy[2], zy[3]);
      if constexpr (sizeof(T) == 4) {
        float4 t = *reinterpret_cast<float4*>(dst);
        t.x = prolong_add(t.x, v[0]); t.y = prolong_add(t.y, v[1]);
        t.z = prolong_add(t.z, v[2]); t.w = prolong_add(t.w, v[3]);
        *reinterpret_cast<float4*>(dst) = t;
      } else {
        double2 t0 = *reinterpret_cast<double2*>(dst);
        double2 t1 = *reinterpret_cast<double2*>(dst + 2);
        t0.x = prolong_add(t0.x, v[0]); t0.y = prolong_add(t0.y, v[1]);
        t1.x = prolong_add(t1.x, v[2]); t1.y = prolong_add(t1.y, v[3]);
        *reinterpret_cast<double2*>(dst) = t0;
        *reinterpret_cast<double2*>(dst + 2) = t1;
      }
    }
}

// The coarse end of a V-cycle in ONE CTA: levels lv.first .. lv.n-1 (at most
// a few thousand cells) live in shared memory (smem_raw, 2 lv.total values);
// smoothing, residual restriction, the exact coarsest solve and prolongation
// run with block-wide barriers between phases. Arithmetic matches the
// multi-kernel levels.
template <typename T>
__device__ void vcycle_small_body(const CoarseLevels& lv, const T* __restrict__ bg, T* __restrict__ xg,
                                  const double* __restrict__ bshift, const T* __restrict__ table, int zero, int nu1,
                                  int nu2, unsigned char* smem_raw) {
  T* X = reinterpret_cast<T*>(smem_raw);
  T* B = X + lv.total;
  const int tid = threadIdx.x, nt = blockDim.x;
  const T sh = bshift ? (T)(*bshift) : (T)0;
  {
    const int n0 = lv.nx[0] * lv.ny[0] * lv.nz[0];
    for (int c = tid; c < n0; c += nt) {
      B[c] = bg[c] - sh;
      X[c] = zero ? (T)0 : xg[c];
    }
    for (int c = n0 + tid; c < lv.total; c += nt) X[c] = (T)0;
  }
  __syncthreads();
  // cell index -> (i, j, k); shifts when the level's nx, ny are powers of 2
  auto decode = [&](int l, int c, int& i, int& j, int& k) {
    const int lx = lv.lgx[l], ly = lv.lgy[l];
    if (lx >= 0 && ly >= 0) {
      i = c & (lv.nx[l] - 1);
      j = (c >> lx) & (lv.ny[l] - 1);
      k = c >> (lx + ly);
    } else {
      i = c % lv.nx[l];
      j = (c / lv.nx[l]) % lv.ny[l];
      k = c / (lv.nx[l] * lv.ny[l]);
    }
  };
  // one red-black sweep on level l (all sides even): each half-sweep visits
  // only the cells of its colour, enumerated as (i/2, j, k)
  auto sweep = [&](int l) {
    const int nx = lv.nx[l], ny = lv.ny[l], nz = lv.nz[l];
    const int hx = nx >> 1, nh = hx * ny * nz, plane = nx * ny;
    T* x = X + lv.off[l];
    const T* b = B + lv.off[l];
    const T inv = (T)(1.0 / lv.diag[l]), off = (T)lv.offd[l];
    const int lx = lv.lgx[l], ly = lv.lgy[l];
    const bool pow2 = lx >= 1 && ly >= 0;
    for (int colour = 0; colour < 2; ++colour) {
      for (int p = tid; p < nh; p += nt) {
        int ih, j, k;
        if (pow2) {
          ih = p & (hx - 1);
          j = (p >> (lx - 1)) & (ny - 1);
          k = p >> (lx - 1 + ly);
        } else {
          ih = p % hx;
          j = (p / hx) % ny;
          k = p / (hx * ny);
        }
        const int i = 2 * ih + ((j + k + colour) & 1);
        const int rowc = k * plane + j * nx;
        const int c = rowc + i;
        const int xw = rowc + (i == 0 ? nx - 1 : i - 1), xe = rowc + (i == nx - 1 ? 0 : i + 1);
        const int ys = c + (j == 0 ? plane - nx : -nx), yn = c + (j == ny - 1 ? nx - plane : nx);
        const int zd = c + (k == 0 ? plane * (nz - 1) : -plane), zu = c + (k == nz - 1 ? -plane * (nz - 1) : plane);
        const T sum = ((x[xw] + x[xe]) + (x[ys] + x[yn])) + (x[zd] + x[zu]);
        x[c] = (b[c] + off * sum) * inv;
      }
      __syncthreads();
    }
  };
  const int last = lv.n - 1;
  for (int l = 0; l < last; ++l) {
    for (int sw = 0; sw < nu1; ++sw) sweep(l);
    // residual restriction to level l+1
    const int nx = lv.nx[l], ny = lv.ny[l], nz = lv.nz[l];
    const int nxc = nx >> 1, nyc = ny >> 1, nc = nxc * nyc * (nz >> 1);
    const T* x = X + lv.off[l];
    const T* b = B + lv.off[l];
    T* bc = B + lv.off[l + 1];
    const T diag = (T)lv.diag[l], off = (T)lv.offd[l];
    // one child per thread: entry e = 8 C + (dz, dy, dx) bits, so the 8
    // children of a coarse cell sit in 8 neighbouring lanes and are summed
    // by shuffles (the loop bound is a multiple of 32 so warps stay whole)
    const int nf = 8 * nc, nround = (nf + 31) & ~31;
    for (int e = tid; e < nround; e += nt) {
      T r = 0;
      if (e < nf) {
        int I, J, K;
        decode(l + 1, e >> 3, I, J, K);
        const int i = 2 * I + (e & 1), j = 2 * J + ((e >> 1) & 1), k = 2 * K + (e >> 2 & 1);
        const int c = (k * ny + j) * nx + i;
        const T s = ((x[c - i + wrap(i - 1, nx)] + x[c - i + wrap(i + 1, nx)]) +
                     (x[c + (wrap(j - 1, ny) - j) * nx] + x[c + (wrap(j + 1, ny) - j) * nx])) +
                    (x[c + (wrap(k - 1, nz) - k) * nx * ny] + x[c + (wrap(k + 1, nz) - k) * nx * ny]);
        r = b[c] - (diag * x[c] - off * s);
      }
      r += __shfl_xor_sync(0xffffffffu, r, 1);
      r += __shfl_xor_sync(0xffffffffu, r, 2);
      r += __shfl_xor_sync(0xffffffffu, r, 4);
      if (e < nf && (e & 7) == 0) bc[e >> 3] = r * (T)0.125;
    }
    __syncthreads();
  }
  {
    // exact coarsest solve with the circulant table
    const int nx = lv.nx[last], ny = lv.ny[last], nz = lv.nz[last], n = nx * ny * nz;
    T* x = X + lv.off[last];
    const T* b = B + lv.off[last];
    for (int t = tid; t < n; t += nt) {
      const int ix = t % nx, iy = (t / nx) % ny, iz = t / (nx * ny);
      T acc = 0;
      for (int u = 0; u < n; ++u) {
        const int jx = u % nx, jy = (u / nx) % ny, jz = u / (nx * ny);
        const int dx = ix - jx + (ix < jx ? nx : 0), dy = iy - jy + (iy < jy ? ny : 0), dz = iz - jz + (iz < jz ? nz : 0);
        acc += table[(dz * ny + dy) * nx + dx] * b[u];
      }
      x[t] = acc;
    }
    __syncthreads();
  }
  for (int l = last - 1; l >= 0; --l) {
    const int nx = lv.nx[l], ny = lv.ny[l], nz = lv.nz[l], n = nx * ny * nz;
    const int nxc = nx >> 1, nyc = ny >> 1, nzc = nz >> 1;
    T* x = X + lv.off[l];
    const T* xc = X + lv.off[l + 1];
    for (int c = tid; c < n; c += nt) {
      int i, j, k;
      decode(l, c, i, j, k);
      const int I = i >> 1, J = j >> 1, K = k >> 1;
      const int I2 = (i & 1) ? wrap(I + 1, nxc) : wrap(I - 1, nxc);
      const int J2 = (j & 1) ? wrap(J + 1, nyc) : wrap(J - 1, nyc);
      const int K2 = (k & 1) ? wrap(K + 1, nzc) : wrap(K - 1, nzc);
      auto e = [&](int kk, int jj, int ii) { return xc[(kk * nyc + jj) * nxc + ii]; };
      // z, then y, then x (each axis scaled by 4)
      auto zy = [&](int ii) {
        return prolong_axis(prolong_axis(e(K, J, ii), e(K2, J, ii)), prolong_axis(e(K, J2, ii), e(K2, J2, ii)));
      };
      x[c] = prolong_add(x[c], prolong_axis(zy(I), zy(I2)));
    }
    __syncthreads();
    for (int sw = 0; sw < nu2; ++sw) sweep(l);
  }
  const int n0 = lv.nx[0] * lv.ny[0] * lv.nz[0];
  for (int c = tid; c < n0; c += nt) xg[c] = X[c];
}

template <typename T>
__global__ void __launch_bounds__(1024) k_vcycle_small(CoarseLevels lv, const T* __restrict__ bg, T* __restrict__ xg,
                                                       const double* __restrict__ bshift, const T* __restrict__ table,
                                                       int zero, int nu1, int nu2) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  vcycle_small_body<T>(lv, bg, xg, bshift, table, zero, nu1, nu2, smem_raw);
}

}  // namespace

template <typename T>
bool rb_sweep_fused_ok(Dims d) {
  return d.nx % 32 == 0 && d.ny % 8 == 0 && d.nz % 2 == 0 && d.nz >= 4;
}


template <typename T, int TX, bool ZERO>
void sweep_launch(dim3 g, cudaStream_t s, const T* xin, T* xout, const T* b, const double* bshift, Dims d, int zc,
                  T inv, T off, double* part) {
  constexpr size_t sm = sweep_smem<T, TX, 8>();
  static std::atomic<unsigned long long> attr{0};
  ensure_smem_attr((const void*)k_rb_sweep<T, TX, 8, ZERO>, (int)sm, attr);
  k_rb_sweep<T, TX, 8, ZERO><<<g, kSweepThreads, sm, s>>>(xin, xout, b, bshift, d.nx, d.ny, d.nz, zc, inv, off,
                                                           part);
}

template <typename T>
int launch_rb_sweep(const T* xin, T* xout, const T* b, const double* bshift, Dims d, Stencil st, bool zero,
                    double* part, int part_cap, cudaStream_t s) {
  const int c = pcls<T>(P_RBGS64, P_RBGS32);
  const T inv = (T)(1.0 / st.diag), off = (T)st.off;
  if constexpr (sizeof(T) == 4) {
    // from zero: one stencil pass over b (no partial sums are asked of a first sweep)
    if (zero && !part && d.nx % 4 == 0 && aligned16(xout) && aligned16(b)) {
      const int nx4 = d.nx / 4;
      const int tx = nx4 >= 32 ? 32 : nx4, ty = 256 / tx;
      const int bx = (nx4 + tx - 1) / tx, by = (d.ny + ty - 1) / ty;
      int chunks = (152 * 8) / (bx * by);
      chunks = chunks < 1 ? 1 : chunks;
      int zc = (d.nz + chunks - 1) / chunks;
      zc = zc < 2 ? 2 : zc;
      const SweepShape* tn = tuned_sweep(4, TUNE_ZERO, d);
      if (tn && tn->zc >= 1) zc = tn->zc < d.nz ? tn->zc : d.nz;
      dim3 g(bx, by, (d.nz + zc - 1) / zc);
      prof_begin(c, s);
      k_rb_zero_f32v<<<g, dim3(tx, ty), 0, s>>>(b, xout, bshift, d.nx, d.ny, d.nz, zc, inv, off);
      prof_end(c, s, "rb_sweep_zero", 8.0 * d.n());
      return 0;
    }
  }
  if constexpr (sizeof(T) == 4) {
    // rows of 128 or 256 cells: the row-resident kernel unless a tiled shape
    // was chosen for this level
    if (!zero && rows_sweep_ok(d) && aligned16(xin) && aligned16(xout) && aligned16(b) && xin != xout &&
        b != xout && wait_error_flag()) {
      const SweepShape* tn = tuned_sweep(4, TUNE_SWEEP, d);
      if (!tn || tn->tx == 0 || tn->tx == d.nx) {
        const int zc = (tn && tn->zc >= 2) ? tn->zc : rows_sweep_default_zc(d);
        prof_begin(c, s);
        const int r = launch_rows_sweep(xin, xout, b, bshift, d, st, zc, part, part_cap, s);
        prof_end(c, s, "rb_sweep_rows", 3.0 * sizeof(T) * d.n());
        return r;
      }
    }
  }
  if (rb_sweep_fused_ok<T>(d) && aligned16(xin) && aligned16(xout) && aligned16(b)) {
    // 64-wide tiles for FP32 (18 vectors per row), 32-wide for FP64
    const SweepShape* tn = tuned_sweep((int)sizeof(T), TUNE_SWEEP, d);
    const bool wide = (sizeof(T) == 4) && (d.nx % 64 == 0) && !(tn && tn->tx == 32);
    const int TX = wide ? 64 : 32, TY = 8;
    const int cols = (d.nx / TX) * (d.ny / TY);
    // about one wave of resident CTAs: chunks per column = resident slots / columns
    const size_t sm = wide ? sweep_smem<T, (sizeof(T) == 4 ? 64 : 32), 8>() : sweep_smem<T, 32, 8>();
    int per_sm = (int)(200 * 1024 / sm);
    per_sm = per_sm < 1 ? 1 : (per_sm > 8 ? 8 : per_sm);
    const int slots = 152 * per_sm;
    int chunks = slots / cols;
    chunks = chunks < 1 ? 1 : chunks;
    int zc = (d.nz + chunks - 1) / chunks;
    if (zc < 2) zc = 2;
    if (tn && tn->zc >= 2) zc = tn->zc < d.nz ? tn->zc : d.nz;
    dim3 g(d.nx / TX, d.ny / TY, (d.nz + zc - 1) / zc);
    const int nblk = (int)(g.x * g.y * g.z);
    if (nblk > part_cap) part = nullptr;
    prof_begin(c, s);
    if constexpr (sizeof(T) == 4) {
      if (wide) {
        if (zero)
          sweep_launch<T, 64, true>(g, s, xin, xout, b, bshift, d, zc, inv, off, part);
        else
          sweep_launch<T, 64, false>(g, s, xin, xout, b, bshift, d, zc, inv, off, part);
      }
    }
    if (!wide) {
      if (zero)
        sweep_launch<T, 32, true>(g, s, xin, xout, b, bshift, d, zc, inv, off, part);
      else
        sweep_launch<T, 32, false>(g, s, xin, xout, b, bshift, d, zc, inv, off, part);
    }
    // one read of x (skipped from zero), one read of b, one write of x
    prof_end(c, s, "rb_sweep", (zero ? 2.0 : 3.0) * sizeof(T) * d.n());
    return part ? nblk : 0;
  }
  // small levels: two in-place half sweeps
  const int np = d.nx / 2;
  dim3 blk(np >= 32 ? 32 : np, 8, 1);
  const int bx = (np + blk.x - 1) / blk.x, by = (d.ny + blk.y - 1) / blk.y;
  int zc = 1;
  while (zc < 8 && (long)bx * by * (d.nz / (zc * 2)) >= 4 * 152) zc *= 2;
  dim3 g(bx, by, (d.nz + zc - 1) / zc);
  for (int colour = 0; colour < 2; ++colour) {
    prof_begin(c, s);
    k_rb_half<T><<<g, blk, 0, s>>>(xin, const_cast<T*>(xin), b, bshift, d.nx, d.ny, d.nz, zc, inv, off, colour,
                                   (zero && colour == 0) ? 1 : 0);
    prof_end(c, s, "rb_half", 1.5 * sizeof(T) * d.n());
  }
  return -1;
}

template <typename T>
void launch_resid_restrict(const T* x, const T* b, const double* bshift, T* bc, Dims d, Stencil st, cudaStream_t s) {
  const int nxc = d.nx / 2, nyc = d.ny / 2, nzc = d.nz / 2;
  if (d.nx % 4 == 0 && d.nx >= 8 && aligned16(x) && aligned16(b)) {
    const int np = nxc / 2;
    dim3 blk(np >= 32 ? 32 : np, 4, 2);
    dim3 g((np + blk.x - 1) / blk.x, (nyc + blk.y - 1) / blk.y, (nzc + blk.z - 1) / blk.z);
    const int c = pcls<T>(P_RESTRICT64, P_RESTRICT32);
    prof_begin(c, s);
    k_resid_restrict2<T><<<g, blk, 0, s>>>(x, b, bshift, bc, d.nx, d.ny, d.nz, (T)st.diag, (T)st.off);
    prof_end(c, s, "resid_restrict", 2.125 * sizeof(T) * d.n());
    return;
  }
  dim3 blk(nxc >= 32 ? 32 : nxc, 4, 2);
  dim3 g((nxc + blk.x - 1) / blk.x, (nyc + blk.y - 1) / blk.y, (nzc + blk.z - 1) / blk.z);
  const int c = pcls<T>(P_RESTRICT64, P_RESTRICT32);
  prof_begin(c, s);
  k_resid_restrict<T><<<g, blk, 0, s>>>(x, b, bshift, bc, d.nx, d.ny, d.nz, (T)st.diag, (T)st.off);
  prof_end(c, s, "resid_restrict", 2.125 * sizeof(T) * d.n());
}

bool zero_restrict_ok(Dims d) { return d.nx % 32 == 0 && d.ny % 8 == 0 && d.nz % 2 == 0 && d.nz >= 4; }

template <int TX4>
void zero_restrict_launch(const float* b, const double* bshift, float* x, float* bc, Dims d, Stencil st,
                          cudaStream_t s) {
  const int bx = d.nx / (4 * TX4), by = d.ny / 8;
  // about one wave of 5 resident CTAs per SM (shared-memory rings); chunks of
  // an even number of planes
  int chunks = (152 * 5) / (bx * by);
  chunks = chunks < 1 ? 1 : chunks;
  int zc = (d.nz + chunks - 1) / chunks;
  zc += zc & 1;
  zc = zc < 2 ? 2 : zc;
  dim3 g(bx, by, (d.nz + zc - 1) / zc);
  constexpr size_t sm = sizeof(float4) * (8 * (8 + 4) * (TX4 + 4) + 4 * (8 + 2) * (TX4 + 2));
  static std::atomic<unsigned long long> attr{0};
  ensure_smem_attr((const void*)k_zero_restrict_f32<TX4>, (int)sm, attr);
  k_zero_restrict_f32<TX4><<<g, dim3(TX4, 8), sm, s>>>(b, bshift, x, bc, d.nx, d.ny, d.nz, zc, (float)(1.0 / st.diag),
                                                        (float)st.off, (float)st.diag);
}

void launch_zero_restrict(const float* b, const double* bshift, float* x, float* bc, Dims d, Stencil st,
                          cudaStream_t s) {
  prof_begin(P_RBGS32, s);
  if (d.nx % 64 == 0)
    zero_restrict_launch<16>(b, bshift, x, bc, d, st, s);
  else
    zero_restrict_launch<8>(b, bshift, x, bc, d, st, s);
  // one read of b, one write of x and of the coarse right-hand side
  prof_end(P_RBGS32, s, "zero_restrict", 8.0 * d.n() + 0.5 * d.n());
}

template <typename T>
int launch_prolong_sweep(const T* xc, const T* xin, T* xout, const T* b, const double* bshift, Dims d, Stencil st,
                         double* part, int part_cap, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (rows_sweep_ok(d) && aligned16(xin) && aligned16(xout) && aligned16(b) && aligned16(xc) && xin != xout &&
        b != xout && xc != xout && wait_error_flag()) {
      // the row-resident sweep serves this level unless a tiled shape was
      // chosen or the fusion was switched off for it
      const SweepShape* tn = tuned_sweep(4, TUNE_SWEEP, d);
      const SweepShape* tp = tuned_sweep(4, TUNE_PROLONG, d);
      if ((!tn || tn->tx == 0 || tn->tx == d.nx) && !(tp && tp->tx == 1)) {
        const int zc = (tn && tn->zc >= 2) ? tn->zc : rows_sweep_default_zc(d);
        prof_begin(P_RBGS32, s);
        const int r = launch_rows_prolong_sweep(xc, xin, xout, b, bshift, d, st, zc, part, part_cap, s);
        // x, b and the coarse field read once, x written once
        prof_end(P_RBGS32, s, "prolong_sweep_rows", (3.0 + 0.125) * sizeof(T) * d.n());
        return r;
      }
    }
  }
  return -1;
}

template <typename T>
void launch_prolong8(const T* xc, T* x, Dims d, cudaStream_t s) {
  const int nxc = d.nx / 2, nyc = d.ny / 2, nzc = d.nz / 2;
  if (d.nx % 4 == 0 && d.nx >= 8 && aligned16(x)) {
    const int np = nxc / 2;
    dim3 blk(np >= 32 ? 32 : np, 4, 2);
    dim3 g((np + blk.x - 1) / blk.x, (nyc + blk.y - 1) / blk.y, (nzc + blk.z - 1) / blk.z);
    const int c = pcls<T>(P_PROLONG64, P_PROLONG32);
    prof_begin(c, s);
    k_prolong8x2<T><<<g, blk, 0, s>>>(xc, x, d.nx, d.ny, d.nz);
    prof_end(c, s, "prolong8", 2.125 * sizeof(T) * d.n());
    return;
  }
  dim3 blk(nxc >= 32 ? 32 : nxc, 4, 2);
  dim3 g((nxc + blk.x - 1) / blk.x, (nyc + blk.y - 1) / blk.y, (nzc + blk.z - 1) / blk.z);
  const int c = pcls<T>(P_PROLONG64, P_PROLONG32);
  prof_begin(c, s);
  k_prolong8<T><<<g, blk, 0, s>>>(xc, x, d.nx, d.ny, d.nz);
  prof_end(c, s, "prolong8", 2.125 * sizeof(T) * d.n());
}

template <typename T>
void launch_vcycle_small(const CoarseLevels& lv, const T* b, T* x, const double* bshift, const T* table, bool zero,
                         int nu1, int nu2, cudaStream_t s) {
  const size_t sm = 2 * sizeof(T) * (size_t)lv.total;
  static std::atomic<unsigned long long> attr{0};
  ensure_smem_attr((const void*)k_vcycle_small<T>, 200 * 1024, attr);
  const int c = pcls<T>(P_RBGS64, P_RBGS32);
  prof_begin(c, s);
  k_vcycle_small<T><<<1, 1024, sm, s>>>(lv, b, x, bshift, table, zero ? 1 : 0, nu1, nu2);
  prof_end(c, s, "vcycle_small", 2.0 * sizeof(T) * lv.total);
}

#define IBRD_INST(T)                                                                                         \
  template void launch_vcycle_small<T>(const CoarseLevels&, const T*, T*, const double*, const T*, bool, int,  \
                                       int, cudaStream_t);                                                  \
  template int launch_rb_sweep<T>(const T*, T*, const T*, const double*, Dims, Stencil, bool, double*, int,    \
                                  cudaStream_t);                                                            \
  template void launch_resid_restrict<T>(const T*, const T*, const double*, T*, Dims, Stencil, cudaStream_t); \
  template void launch_prolong8<T>(const T*, T*, Dims, cudaStream_t);                                       \
  template int launch_prolong_sweep<T>(const T*, const T*, T*, const T*, const double*, Dims, Stencil, double*,   \
                                       int, cudaStream_t);                                                   \
  template bool rb_sweep_fused_ok<T>(Dims);
IBRD_INST(double)
IBRD_INST(float)
#undef IBRD_INST

}  // namespace ibrd
