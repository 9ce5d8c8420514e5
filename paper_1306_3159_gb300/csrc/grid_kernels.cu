// Grid kernels: 7-point periodic Helmholtz operator (Sec. III.A, Eq. Helmholtz),
// the multigrid pieces of the V-cycle (Sec. III.E: red-black Gauss-Seidel,
// 8-cell-mean restriction, trilinear cell-centred prolongation, exact
// coarsest solve) and streaming vector kernels (reductions, conversions).
//
// Layout: fields are [nz][ny][nx], x fastest, periodic in every direction.
// FP64 arithmetic on GB300 is bound by the FP64 pipe (about 0.6 T FMA/s), so
// the FP64 kernels minimise FP64 instructions per cell; the FP32 kernels are
// bound by HBM and keep one read of each input and one write per output.
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace ibrd {
namespace {

constexpr int BX = 32, BY = 8, ZCH = 16;

__device__ __forceinline__ int wrap_dec(int i, int n) { return i == 0 ? n - 1 : i - 1; }
__device__ __forceinline__ int wrap_inc(int i, int n) { return i == n - 1 ? 0 : i + 1; }

// y = A x (RESID = false) or y = b - A x (RESID = true); 2.5D z-march with the
// z-neighbours kept in registers and x/y neighbours served by L1.
template <typename T, bool RESID>
__global__ void __launch_bounds__(BX* BY) k_apply(const T* __restrict__ x, const T* __restrict__ b,
                                                  T* __restrict__ y, int nx, int ny, int nz, T diag, T off) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  if (i >= nx || j >= ny) return;
  const int k0 = blockIdx.z * ZCH;
  const int k1 = min(k0 + ZCH, nz);
  const int im = wrap_dec(i, nx), ip = wrap_inc(i, nx);
  const size_t plane = (size_t)nx * ny;
  const size_t rj = (size_t)j * nx, rjm = (size_t)wrap_dec(j, ny) * nx, rjp = (size_t)wrap_inc(j, ny) * nx;
  T xm = x[(size_t)wrap_dec(k0, nz) * plane + rj + i];
  T x0 = x[(size_t)k0 * plane + rj + i];
  for (int k = k0; k < k1; ++k) {
    const size_t base = (size_t)k * plane;
    const T xp = x[(size_t)wrap_inc(k, nz) * plane + rj + i];
    const T s = ((x[base + rj + im] + x[base + rj + ip]) + (x[base + rjm + i] + x[base + rjp + i])) + (xm + xp);
    const T v = diag * x0 - off * s;
    if (RESID)
      y[base + rj + i] = b[base + rj + i] - v;
    else
      y[base + rj + i] = v;
    xm = x0;
    x0 = xp;
  }
}

// ---------------------------------------------------------------- FP64 residual, fixed point
// r = b - A x = b - alpha x + off L x with L x = (sum of the 6 neighbours) -
// 6 x. Every x is scaled by 2^S into a 64-bit integer X (S from the field's
// largest |x|, so that |X| < 2^59): L X is then an exact integer sum, where
// the FP64 form diag x - off s rounds terms of size 6 off |x|, far above |r|
// near convergence. r = fma(-alpha, x, fma(off 2^-S, double(L X), b)) then
// rounds once per FMA: within 2^-52 of |r| + off |L x| plus the scaling's
// 2^-56 off max|x|, with one FP64 instruction per cell (two with alpha != 0;
// the integer work runs on the integer pipe; GB300's FP64 pipe does about 1.6
// additions, multiplications or FMAs per SM per clock).

// v 2^S rounded to an integer, for |v| 2^S < 2^59
__device__ __forceinline__ long long to_fixed(double v, int S) {
  const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
  const int e = (hi >> 20) & 0x7FF;
  if (e == 0) return 0;
  const unsigned long long m = ((unsigned long long)((hi & 0xFFFFFu) | 0x100000u) << 32) | lo;
  const int sh = e - 1075 + S;  // v 2^S = m 2^sh, sh <= 6
  unsigned long long X;
  if (sh >= 0)
    X = m << sh;
  else if (sh > -63)
    X = ((m >> (-sh - 1)) + 1) >> 1;  // nearest, ties up
  else
    X = 0;
  return (int)hi < 0 ? -(long long)X : (long long)X;
}
// a 64-bit integer as the nearest double (ties to even), from the bits
__device__ __forceinline__ double ll2d_bits(long long L) {
  if (L == 0) return 0.0;
  const unsigned long long sgn = (unsigned long long)L & 0x8000000000000000ull;
  unsigned long long a = L < 0 ? 0ull - (unsigned long long)L : (unsigned long long)L;
  const int lz = __clzll((long long)a);
  a <<= lz;  // leading one at bit 63
  const unsigned long long mant = (a >> 11) & 0xFFFFFFFFFFFFFull;
  const unsigned rest = (unsigned)a & 0x7FFu;
  const unsigned long long up = (rest > 0x400u) | ((rest == 0x400u) & ((unsigned)mant & 1u));
  return __longlong_as_double((long long)(sgn | ((((unsigned long long)(1086 - lz)) << 52) + mant + up)));
}

// Largest |x| as the bits of a double (monotonic in |x| for the magnitude bits),
// into *out (zeroed before). Bits at or above those of infinity: x not finite.
__global__ void __launch_bounds__(256) k_absmax_bits(const double* __restrict__ x, size_t n, int vec,
                                                     unsigned long long* __restrict__ out) {
  unsigned long long m = 0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  auto take = [&](double v) {
    const unsigned long long a = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
    m = a > m ? a : m;
  };
  if (vec) {  // 16-byte aligned: pairs, then the odd last entry
    for (size_t i = t; i < n / 2; i += stride) {
      const double2 v = reinterpret_cast<const double2*>(x)[i];
      take(v.x);
      take(v.y);
    }
    if ((n & 1) && t == 0) take(x[n - 1]);
  } else {
    for (size_t i = t; i < n; i += stride) take(x[i]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
    m = v > m ? v : m;
  }
  __shared__ unsigned long long wm[8];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = wm[w] > m ? wm[w] : m;
    atomicMax(out, m);
  }
}

// exponent fields of the largest |x| the fixed-point form takes (off 2^-S
// and the scaled values stay far inside the double range)
constexpr int kFxEmin = 1023 - 900, kFxEmax = 1023 + 900;

// y = b - A x. Block: 32 x TY threads; a thread owns CPT consecutive cells of
// a row (tile 32 CPT x TY) and marches zc planes in z with the z-neighbours
// as fixed-point values in registers, loading the next plane's x, b, halo row
// and tile-edge value one plane ahead. A plane's values go through a
// double-buffered shared tile for the y-neighbours (warps 0 and TY - 1 also
// convert the halo rows); x-neighbours come from the thread itself, its
// lanes' neighbours (shuffles), or, at the tile's edges, from the edge value
// every lane loads (lane 0 the left one, lane 31 the right one). Needs
// nx % (32 CPT) == 0 and ny % TY == 0.
template <int TY, int CPT, bool ALPHA>
__global__ void __launch_bounds__(32 * TY) k_resid_fx(const double* __restrict__ x, const double* __restrict__ b,
                                                      double* __restrict__ y, int nx, int ny, int nz, int zc,
                                                      double alpha, double off, double diag,
                                                      const unsigned long long* __restrict__ xmax) {
  constexpr int TW = 32 * CPT;
  __shared__ long long XS[2][TY + 2][TW];
  const int lane = threadIdx.x, ty = threadIdx.y;
  const int i0 = blockIdx.x * TW, ic = i0 + lane * CPT, j0 = blockIdx.y * TY, j = j0 + ty;
  const int k0 = blockIdx.z * zc, k1 = min(k0 + zc, nz);
  const size_t plane = (size_t)nx * ny, rj = (size_t)j * nx;
  auto at = [&](int k, size_t row, int i) { return (size_t)k * plane + row + i; };
  const int emax = (int)(*xmax >> 52);
  if (emax < kFxEmin || emax > kFxEmax) {
    // the largest |x| is outside the fixed-point range (or x is not finite):
    // the FP64 stencil
    const size_t rjm = (size_t)wrap_dec(j, ny) * nx, rjp = (size_t)wrap_inc(j, ny) * nx;
    for (int k = k0; k < k1; ++k) {
      const int km = wrap_dec(k, nz), kp = wrap_inc(k, nz);
#pragma unroll
      for (int q = 0; q < CPT; ++q) {
        const int i = ic + q;
        const double s = ((x[at(k, rj, wrap_dec(i, nx))] + x[at(k, rj, wrap_inc(i, nx))]) +
                          (x[at(k, rjm, i)] + x[at(k, rjp, i)])) + (x[at(km, rj, i)] + x[at(kp, rj, i)]);
        y[at(k, rj, i)] = b[at(k, rj, i)] - (diag * x[at(k, rj, i)] - off * s);
      }
    }
    return;
  }
  const int S = 1081 - emax;  // |x| < 2^(emax - 1022), so |x| 2^S < 2^59
  const double offs = off * __hiloint2double((1023 - S) << 20, 0);  // off 2^-S, exactly
  const bool halo = ty == 0 || ty == TY - 1;
  const int hrow = ty == 0 ? 0 : TY + 1;
  const size_t rh = (size_t)(ty == 0 ? wrap_dec(j0, ny) : wrap_inc(j0 + TY - 1, ny)) * nx;
  const int ie = lane == 0 ? wrap_dec(i0, nx) : wrap_inc(i0 + TW - 1, nx);  // this lane's tile-edge cell
  struct Vals {
    double v[CPT];
  };
  auto load_row = [&](size_t o) {
    Vals r;
    if constexpr (CPT == 2) {
      const double2 t = *reinterpret_cast<const double2*>(x + o);
      r.v[0] = t.x;
      r.v[1] = t.y;
    } else {
#pragma unroll
      for (int q = 0; q < CPT; ++q) r.v[q] = x[o + q];
    }
    return r;
  };
  auto load_b = [&](size_t o) {
    Vals r;
    if constexpr (CPT == 2) {
      const double2 t = *reinterpret_cast<const double2*>(b + o);
      r.v[0] = t.x;
      r.v[1] = t.y;
    } else {
#pragma unroll
      for (int q = 0; q < CPT; ++q) r.v[q] = b[o + q];
    }
    return r;
  };
  long long Xm[CPT], X0[CPT], Xp[CPT];
  Vals xc = load_row(at(k0, rj, ic));       // plane k (the alpha term)
  Vals xn = load_row(at(wrap_inc(k0, nz), rj, ic));  // plane k + 1
  {
    const Vals t = load_row(at(wrap_dec(k0, nz), rj, ic));
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
      Xm[q] = to_fixed(t.v[q], S);
      X0[q] = to_fixed(xc.v[q], S);
    }
  }
  Vals bv = load_b(at(k0, rj, ic));
  Vals hv = halo ? load_row(at(k0, rh, ic)) : Vals{};
  double ev = x[at(k0, rj, ie)];
  for (int k = k0; k < k1; ++k) {
    const int buf = (k - k0) & 1;
    // next plane's loads first (they land while this plane is computed)
    const bool more = k + 1 < k1;
    const int kn = more ? k + 1 : k;
    const Vals xn2 = load_row(at(wrap_inc(kn, nz), rj, ic));
    const Vals bn = load_b(at(kn, rj, ic));
    const Vals hn = halo ? load_row(at(kn, rh, ic)) : Vals{};
    const double en = x[at(kn, rj, ie)];
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
      Xp[q] = to_fixed(xn.v[q], S);
      XS[buf][ty + 1][lane * CPT + q] = X0[q];
    }
    if (halo) {
#pragma unroll
      for (int q = 0; q < CPT; ++q) XS[buf][hrow][lane * CPT + q] = to_fixed(hv.v[q], S);
    }
    const long long Xedge = to_fixed(ev, S);
    long long Xw = __shfl_up_sync(0xffffffffu, X0[CPT - 1], 1), Xe = __shfl_down_sync(0xffffffffu, X0[0], 1);
    if (lane == 0) Xw = Xedge;
    if (lane == 31) Xe = Xedge;
    __syncthreads();
    double r[CPT];
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
      const long long w = q == 0 ? Xw : X0[q - 1], e = q == CPT - 1 ? Xe : X0[q + 1];
      const long long L = ((w + e) + (XS[buf][ty][lane * CPT + q] + XS[buf][ty + 2][lane * CPT + q])) +
                          (Xm[q] + Xp[q]) - 6 * X0[q];
      r[q] = fma(offs, ll2d_bits(L), bv.v[q]);
      if constexpr (ALPHA) r[q] = fma(-alpha, xc.v[q], r[q]);  // a separate instantiation: a predicated
                                                               // DFMA would still take the FP64 pipe
    }
    if constexpr (CPT == 2) {
      *reinterpret_cast<double2*>(y + at(k, rj, ic)) = make_double2(r[0], r[1]);
    } else {
#pragma unroll
      for (int q = 0; q < CPT; ++q) y[at(k, rj, ic + q)] = r[q];
    }
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
      Xm[q] = X0[q];
      X0[q] = Xp[q];
    }
    xc = xn;
    xn = xn2;
    bv = bn;
    hv = hn;
    ev = en;
  }
}

// FP32 y = A x with 4 cells per thread (16-byte rows; nx % 4 == 0, aligned
// fields): z-march over zc planes with the z-neighbour 4-vectors in registers,
// y-neighbour 4-vectors and the two x-edge scalars from L1/L2.
__global__ void __launch_bounds__(256) k_apply_f32v(const float* __restrict__ x, float* __restrict__ y, int nx,
                                                    int ny, int nz, int zc, float diag, float off) {
  const int i4 = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int nx4 = nx >> 2;
  if (i4 >= nx4 || j >= ny) return;
  const int k0 = blockIdx.z * zc;
  const int k1 = min(k0 + zc, nz);
  if (k0 >= k1) return;
  const int i = 4 * i4;
  const int im = wrap_dec(i, nx), ip = wrap_inc(i + 3, nx);
  const size_t plane = (size_t)nx * ny;
  const size_t rj = (size_t)j * nx, rjm = (size_t)wrap_dec(j, ny) * nx, rjp = (size_t)wrap_inc(j, ny) * nx;
  auto ld4 = [&](size_t o) { return *reinterpret_cast<const float4*>(x + o); };
  auto kw = [&](int k) { return (size_t)(k >= nz ? k - nz : k) * plane + rj + i; };
  float4 xm = ld4((size_t)wrap_dec(k0, nz) * plane + rj + i);
  float4 x0 = ld4(kw(k0));
  // the next plane's centre row is loaded one iteration ahead (two rows in flight)
  float4 x1 = ld4(kw(k0 + 1));
  for (int k = k0; k < k1; ++k) {
    const size_t base = (size_t)k * plane;
    const float4 xp = x1;
    if (k + 1 < k1) x1 = ld4(kw(k + 2));
    const float4 ys = ld4(base + rjm + i), yn = ld4(base + rjp + i);
    const float xl = x[base + rj + im], xr = x[base + rj + ip];
    float4 v;
    v.x = diag * x0.x - off * (((xl + x0.y) + (ys.x + yn.x)) + (xm.x + xp.x));
    v.y = diag * x0.y - off * (((x0.x + x0.z) + (ys.y + yn.y)) + (xm.y + xp.y));
    v.z = diag * x0.z - off * (((x0.y + x0.w) + (ys.z + yn.z)) + (xm.z + xp.z));
    v.w = diag * x0.w - off * (((x0.z + xr) + (ys.w + yn.w)) + (xm.w + xp.w));
    *reinterpret_cast<float4*>(y + base + rj + i) = v;
    xm = x0;
    x0 = xp;
  }
}

// Dense circulant solve on the coarsest grid (at most 512 cells, one block).
template <typename T>
__global__ void k_coarse_solve(const T* __restrict__ table, const T* __restrict__ b, T* __restrict__ x, int nx,
                               int ny, int nz) {
  __shared__ T sb[512];
  const int n = nx * ny * nz;
  for (int t = threadIdx.x; t < n; t += blockDim.x) sb[t] = b[t];
  __syncthreads();
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int ix = t % nx, iy = (t / nx) % ny, iz = t / (nx * ny);
    T acc = 0;
    for (int u = 0; u < n; ++u) {
      const int jx = u % nx, jy = (u / nx) % ny, jz = u / (nx * ny);
      const int dx = ix - jx + (ix < jx ? nx : 0);
      const int dy = iy - jy + (iy < jy ? ny : 0);
      const int dz = iz - jz + (iz < jz ? nz : 0);
      acc += table[(dz * ny + dy) * nx + dx] * sb[u];
    }
    x[t] = acc;
  }
}

template <typename T>
__global__ void k_coarse_table(T* __restrict__ table, int nx, int ny, int nz, double diag, double off,
                               int singular) {
  const int n = nx * ny * nz;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int dx = t % nx, dy = (t / nx) % ny, dz = t / (nx * ny);
  const double twopi = 6.283185307179586476925286766559;
  // eigenvalue of diag I - off * (sum of 6 shifts): diag - 2 off sum_d cos(2 pi k_d / n_d)
  double acc = 0.0;
  for (int u = 0; u < n; ++u) {
    if (singular && u == 0) continue;
    const int kx = u % nx, ky = (u / nx) % ny, kz = u / (nx * ny);
    const double lam = diag - 2.0 * off * (cos(twopi * kx / nx) + cos(twopi * ky / ny) + cos(twopi * kz / nz));
    const double ph = twopi * ((double)kx * dx / nx + (double)ky * dy / ny + (double)kz * dz / nz);
    acc += cos(ph) / lam;
  }
  table[t] = (T)(acc / n);
}

// Exact solve on a small periodic level through the separable Hartley
// transform. With cas(t) = cos t + sin t, the matrix H_n[k][j] =
// cas(2 pi k j / n) is symmetric, H_n^2 = n I, and its columns are
// eigenvectors of every symmetric circulant of order n (cos and sin of the
// same frequency share an eigenvalue). So T = H_nz (x) H_ny (x) H_nx is
// symmetric with T^2 = N I and diagonalises A = diag I - off * (sum of the 6
// shifts) with eigenvalues lambda_k = diag - 2 off (cos(2 pi kx / nx) +
// cos(2 pi ky / ny) + cos(2 pi kz / nz)); hence A^-1 = T diag(w) T with
// w_k = 1 / (N lambda_k), and w_0 = 0 when singular (the pseudo-inverse:
// mean-zero in, mean-zero out).
//
// Table layout (FP32): cas_x (nx^2), cas_y (ny^2), cas_z (nz^2), w (N).
__global__ void k_hartley_tables(float* __restrict__ tab, int nx, int ny, int nz, double diag, double off,
                                 int singular) {
  const int n = nx * ny * nz;
  const int ox = 0, oy = nx * nx, oz = oy + ny * ny, ow = oz + nz * nz;
  const double twopi = 6.283185307179586476925286766559;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  auto cas = [&](int k, int j, int m) {
    const double a = twopi * (double)((k * j) % m) / m;
    return (float)(cos(a) + sin(a));
  };
  if (t < nx * nx) tab[ox + t] = cas(t / nx, t % nx, nx);
  if (t < ny * ny) tab[oy + t] = cas(t / ny, t % ny, ny);
  if (t < nz * nz) tab[oz + t] = cas(t / nz, t % nz, nz);
  if (t < n) {
    const int kx = t % nx, ky = (t / nx) % ny, kz = t / (nx * ny);
    const double lam =
        diag - 2.0 * off * (cos(twopi * kx / nx) + cos(twopi * ky / ny) + cos(twopi * kz / nz));
    tab[ow + t] = (singular && t == 0) ? 0.f : (float)(1.0 / ((double)n * lam));
  }
}

// One CTA: loads b - shift, applies T, scales by w, applies T, stores x. In
// shared memory the field is padded (strides 1, nx + 1, (nx + 1)(ny + 1)) and
// the rows of H are padded to m + 1, so that a pass, one thread per output
// (line, k) with consecutive threads on consecutive k, reads H rows and
// writes outputs without bank conflicts and reads each input as a broadcast.
// CUBE = 16 fixes a 16^3 level at compile time: each thread then computes 4
// outputs (k0 .. k0 + 3) of one line, holding the line's 16 inputs in
// registers and reading H (symmetric, unpadded) as 4-vectors, a quarter of
// the shared-memory loads per output. CUBE = 0 takes the sides at run time.
template <int CUBE>
__global__ void __launch_bounds__(1024) k_hartley_solve(const float* __restrict__ tab, const float* __restrict__ b,
                                                        const double* __restrict__ bshift, float* __restrict__ x,
                                                        int nx_, int ny_, int nz_) {
  extern __shared__ __align__(16) float hs[];
  const int nx = CUBE ? CUBE : nx_, ny = CUBE ? CUBE : ny_, nz = CUBE ? CUBE : nz_;
  const int n = nx * ny * nz;
  const int px = nx + 1, pxy = (nx + 1) * (ny + 1), pn = pxy * nz;
  float* Hp[3];
  Hp[0] = hs;
  Hp[1] = Hp[0] + nx * (nx + 1);  // (CUBE = 16: 272 floats, a multiple of 4, so the unpadded tables stay aligned)
  Hp[2] = Hp[1] + ny * (ny + 1);
  float* D0 = Hp[2] + nz * (nz + 1);
  float* D1 = D0 + pn;
  const float* W = tab + nx * nx + ny * ny + nz * nz;  // read from global (once per cell)
  const int len[3] = {nx, ny, nz}, pstr[3] = {1, px, pxy};
  const float* src[3] = {tab, tab + nx * nx, tab + nx * nx + ny * ny};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int m = len[a];
    if constexpr (CUBE == 16)
      for (int i = threadIdx.x; i < m * m; i += blockDim.x) Hp[a][i] = src[a][i];  // unpadded
    else
      for (int i = threadIdx.x; i < m * m; i += blockDim.x) Hp[a][(i / m) * (m + 1) + i % m] = src[a][i];
  }
  const float sh = bshift ? (float)(*bshift) : 0.f;
  auto pidx = [&](int c) {  // padded index of cell c
    const int i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
    return k * pxy + j * px + i;
  };
  for (int c = threadIdx.x; c < n; c += blockDim.x) D0[pidx(c)] = b[c] - sh;
  __syncthreads();
  // out = transform of in along axis a
  auto pass = [&](const float* in, float* out, int a) {
    const int m = len[a], st = pstr[a];
    const float* h = Hp[a];
    const int o1 = a == 0 ? ny : nx;  // the two other coordinates of a line
    if constexpr (CUBE == 16) {
      // blockDim.x == 1024 == 4096 outputs / 4: one item per thread
      const int line = threadIdx.x >> 2, k0 = (threadIdx.x & 3) * 4;
      const int u = line & 15, v = line >> 4;
      const int base = a == 0 ? u * px + v * pxy : (a == 1 ? u + v * pxy : u + v * px);
      float xin[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) xin[j] = in[base + j * st];
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float4 hv = *reinterpret_cast<const float4*>(h + j * 16 + k0);  // H[k0..k0+3][j] (symmetric)
        acc.x = fmaf(hv.x, xin[j], acc.x);
        acc.y = fmaf(hv.y, xin[j], acc.y);
        acc.z = fmaf(hv.z, xin[j], acc.z);
        acc.w = fmaf(hv.w, xin[j], acc.w);
      }
      out[base + (k0 + 0) * st] = acc.x;
      out[base + (k0 + 1) * st] = acc.y;
      out[base + (k0 + 2) * st] = acc.z;
      out[base + (k0 + 3) * st] = acc.w;
    } else {
    for (int it = threadIdx.x; it < n; it += blockDim.x) {
      const int line = it / m, k = it - line * m;
      const int u = line % o1, v = line / o1;
      const int base = a == 0 ? u * px + v * pxy : (a == 1 ? u + v * pxy : u + v * px);
      const float* hk = h + k * (m + 1);
      const float* ip = in + base;
      float acc = 0.f;
      for (int j = 0; j < m; ++j) acc = fmaf(hk[j], ip[j * st], acc);
      out[base + k * st] = acc;
    }
    }
    __syncthreads();
  };
  pass(D0, D1, 0);
  pass(D1, D0, 1);
  pass(D0, D1, 2);
  for (int c = threadIdx.x; c < n; c += blockDim.x) D1[pidx(c)] *= W[c];
  __syncthreads();
  pass(D1, D0, 0);
  pass(D0, D1, 1);
  pass(D1, D0, 2);
  for (int c = threadIdx.x; c < n; c += blockDim.x) x[c] = D0[pidx(c)];
}

// Larger exact levels (4096 < N <= 32768 cells, sides <= 64): the same
// transform T = H_z H_y H_x in three launches through a scratch field:
// planes (H_y H_x per z-plane, one CTA each), columns (H_z, scale by w, H_z,
// one CTA per y-row), planes again (H_y H_x). In shared memory a 2-D slice is
// padded to a row stride of cols + 1, H rows to m + 1 (conflict-free).
//
// Shared-memory size (floats) reserved for one H table of order m: m (m + 1),
// rounded up to a multiple of 4 so that the next table stays 16-byte aligned.
__host__ __device__ __forceinline__ int hartley_hsz(int m) { return (m * (m + 1) + 3) & ~3; }

// Orders whose transforms run register-blocked (hartley_pass_reg).
__device__ __forceinline__ bool hartley_reg(int m) { return m == 16 || m == 32; }

// H of order m into shared memory: unpadded for the register-blocked pass,
// rows padded to m + 1 for the generic one.
__device__ void hartley_stage(float* __restrict__ dst, const float* __restrict__ src, int m) {
  if (hartley_reg(m))
    for (int i = threadIdx.x; i < m * m; i += blockDim.x) dst[i] = src[i];
  else
    for (int i = threadIdx.x; i < m * m; i += blockDim.x) dst[(i / m) * (m + 1) + i % m] = src[i];
}

// Register-blocked pass for lines of M values: a thread holds one line's
// inputs in registers and forms 4 consecutive outputs k0 .. k0 + 3, reading H
// (symmetric: row j holds H[k][j] at column k) as 4-vectors, a quarter of a
// shared-memory load per multiply-add. Each output is the same chain of FMAs
// over j = 0 .. M - 1 as in the generic pass, so the results are identical.
template <int M>
__device__ __forceinline__ void hartley_pass_reg(const float* __restrict__ in, float* __restrict__ out, const float* __restrict__ h,
                                 int lines, int st, int lstride) {
  constexpr int G = M / 4;
  for (int it = threadIdx.x; it < lines * G; it += blockDim.x) {
    const int line = it / G, k0 = 4 * (it - line * G);
    const float* ip = in + line * lstride;
    float xin[M];
#pragma unroll
    for (int j = 0; j < M; ++j) xin[j] = ip[j * st];
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int j = 0; j < M; ++j) {
      const float4 hv = *reinterpret_cast<const float4*>(h + j * M + k0);
      acc.x = fmaf(hv.x, xin[j], acc.x);
      acc.y = fmaf(hv.y, xin[j], acc.y);
      acc.z = fmaf(hv.z, xin[j], acc.z);
      acc.w = fmaf(hv.w, xin[j], acc.w);
    }
    float* op = out + line * lstride;
    op[(k0 + 0) * st] = acc.x;
    op[(k0 + 1) * st] = acc.y;
    op[(k0 + 2) * st] = acc.z;
    op[(k0 + 3) * st] = acc.w;
  }
  __syncthreads();
}

// Transform along one axis of a padded 2-D slice: `lines` lines of m values,
// element j of line l at l * lstride + j * st; h as staged by hartley_stage.
// Generic pass: one thread per output (line, k), consecutive threads on
// consecutive k, so H rows (padded) are read without bank conflicts and each
// input as a broadcast.
__device__ __forceinline__ void hartley_pass2d(const float* __restrict__ in, float* __restrict__ out,
                                               const float* __restrict__ h, int m, int lines, int st, int lstride) {
  if (m == 32) return hartley_pass_reg<32>(in, out, h, lines, st, lstride);
  if (m == 16) return hartley_pass_reg<16>(in, out, h, lines, st, lstride);
  for (int it = threadIdx.x; it < lines * m; it += blockDim.x) {
    const int line = it / m, k = it - line * m;
    const int base = line * lstride;
    const float* hk = h + k * (m + 1);
    float acc = 0.f;
    for (int j = 0; j < m; ++j) acc = fmaf(hk[j], in[base + j * st], acc);
    out[base + k * st] = acc;
  }
  __syncthreads();
}

// H_y H_x on z-plane blockIdx.x of src (minus *bshift when given) into dst.
__global__ void __launch_bounds__(1024) k_hartley_planes(const float* __restrict__ src,
                                                         const double* __restrict__ bshift, float* __restrict__ dst,
                                                         const float* __restrict__ tab, int nx, int ny) {
  extern __shared__ __align__(16) float hs[];
  const int px = nx + 1, pn = px * ny;
  float* hx = hs;
  float* hy = hx + hartley_hsz(nx);
  float* A = hy + hartley_hsz(ny);
  float* Bf = A + pn;
  hartley_stage(hx, tab, nx);
  hartley_stage(hy, tab + nx * nx, ny);
  const float sh = bshift ? (float)(*bshift) : 0.f;
  const float* sp = src + (size_t)blockIdx.x * nx * ny;
  for (int c = threadIdx.x; c < nx * ny; c += blockDim.x) A[(c / nx) * px + c % nx] = sp[c] - sh;
  __syncthreads();
  hartley_pass2d(A, Bf, hx, nx, ny, 1, px);   // along x: ny lines (rows)
  hartley_pass2d(Bf, A, hy, ny, nx, px, 1);   // along y: nx lines (columns)
  float* dp = dst + (size_t)blockIdx.x * nx * ny;
  for (int c = threadIdx.x; c < nx * ny; c += blockDim.x) dp[c] = A[(c / nx) * px + c % nx];
}

// H_z, scale by w, H_z on the (x, z) slice of y-row blockIdx.x, in place.
__global__ void __launch_bounds__(1024) k_hartley_columns(float* __restrict__ f, const float* __restrict__ tab, int nx,
                                                          int ny, int nz) {
  extern __shared__ __align__(16) float hs[];
  const int px = nx + 1, pn = px * nz, j = blockIdx.x;
  float* hz = hs;
  float* A = hz + hartley_hsz(nz);
  float* Bf = A + pn;
  const float* tz = tab + nx * nx + ny * ny;
  const float* W = tz + nz * nz;
  hartley_stage(hz, tz, nz);
  for (int c = threadIdx.x; c < nx * nz; c += blockDim.x) {
    const int i = c % nx, k = c / nx;
    A[k * px + i] = f[((size_t)k * ny + j) * nx + i];
  }
  __syncthreads();
  hartley_pass2d(A, Bf, hz, nz, nx, px, 1);  // along z: nx lines
  for (int c = threadIdx.x; c < nx * nz; c += blockDim.x) {
    const int i = c % nx, k = c / nx;
    Bf[k * px + i] *= W[((size_t)k * ny + j) * nx + i];
  }
  __syncthreads();
  hartley_pass2d(Bf, A, hz, nz, nx, px, 1);
  for (int c = threadIdx.x; c < nx * nz; c += blockDim.x) {
    const int i = c % nx, k = c / nx;
    f[((size_t)k * ny + j) * nx + i] = A[k * px + i];
  }
}

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of v (blockDim.x == kRedThreads); result valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sw[32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sw[wid] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? sw[threadIdx.x] : 0.0;
  if (wid == 0) v = warp_sum(v);
  __syncthreads();
  return v;
}

// Block sum of FP32 per-thread values (blockDim.x == kRedThreads), result
// valid in thread 0: the warps add in FP32, the block adds the warps' totals
// in FP64 (one warp of FP64 shuffles per block instead of all of them: the
// FP64 pipe is about 64 times narrower than the FP32 one).
__device__ __forceinline__ double block_sum_f(float v) {
  __shared__ double sw[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sw[wid] = (double)v;
  __syncthreads();
  double d = (threadIdx.x < (blockDim.x >> 5)) ? sw[threadIdx.x] : 0.0;
  if (wid == 0) d = warp_sum(d);
  __syncthreads();
  return d;
}

// Optional tail of a partial-sum kernel: the last CTA of the grid to finish
// (a ticket taken after a fence; no CTA waits) adds the CTAs' partials in the
// order of k_finalize into *out0 (times scale0) and, with out1, the second
// row of partials (partial + gridDim.x) into *out1, then resets the ticket.
struct FinTail {
  unsigned* ticket = nullptr;
  double* out0 = nullptr;
  double scale0 = 1.0;
  double* out1 = nullptr;
  double scale1 = 1.0;
};

__device__ void fin_tail(const double* partial, const FinTail& t) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(t.ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double acc = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) acc += __ldcg(partial + i);
  acc = block_sum(acc);
  if (threadIdx.x == 0) *t.out0 = acc * t.scale0;
  if (t.out1) {
    acc = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) acc += __ldcg(partial + gridDim.x + i);
    acc = block_sum(acc);
    if (threadIdx.x == 0) *t.out1 = acc * t.scale1;
  }
  if (threadIdx.x == 0) *t.ticket = 0u;
}

// Sum of x: each thread folds 8-element runs (FP32 inputs summed in FP32 within
// a run, then in FP64) from a grid-stride loop with 4 independent runs in flight.
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_sum_partial(const T* __restrict__ x, size_t n,
                                                             double* __restrict__ partial, FinTail tail) {
  double acc = 0.0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  size_t i = t;
  for (; i + 3 * stride < n; i += 4 * stride) {
    const T a0 = x[i], a1 = x[i + stride], a2 = x[i + 2 * stride], a3 = x[i + 3 * stride];
    acc += (double)((a0 + a1) + (a2 + a3));
  }
  for (; i < n; i += stride) acc += (double)x[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
  if (tail.ticket) fin_tail(partial, tail);
}

// FP64: one FMA per element, sums in FP64; FP32: products summed per thread
// and across a warp in FP32 (a thread holds a few dozen products of a 256^3
// field), across warps and blocks in FP64.
template <typename E>
__global__ void __launch_bounds__(kRedThreads) k_dot_partial(const E* __restrict__ x, const E* __restrict__ y,
                                                             size_t n, double* __restrict__ partial, int vec,
                                                             FinTail tail) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if constexpr (sizeof(E) == 4) {
    float acc = 0.f;
    if (vec) {
      // 16-byte aligned: 4-vectors
      const size_t n4 = n >> 2, t = i;
      for (size_t v = t; v < n4; v += stride) {
        const float4 a = reinterpret_cast<const float4*>(x)[v], b = reinterpret_cast<const float4*>(y)[v];
        acc = fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, fmaf(a.w, b.w, acc))));
      }
      i = 4 * n4 + t;
    }
    for (; i < n; i += stride) acc = fmaf(x[i], y[i], acc);
    const double s = block_sum_f(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
  } else {
    double acc = 0.0;
    for (; i < n; i += stride) acc = fma(x[i], y[i], acc);
    acc = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
  }
  if (tail.ticket) fin_tail(partial, tail);
}

__global__ void __launch_bounds__(kRedThreads) k_finalize(const double* __restrict__ partial, int np,
                                                          double* __restrict__ out, double scale) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc += partial[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) *out = acc * scale;
}

// y = (T) x with the sum of x and the sum of the converted values.
template <typename X, typename T>
__global__ void __launch_bounds__(kRedThreads) k_convert_sum(const X* __restrict__ x, T* __restrict__ y,
                                                             size_t n, double* __restrict__ pin,
                                                             double* __restrict__ pout, FinTail tail) {
  // FP64 input is summed with one FP64 add per value; FP32 values (input or
  // converted) are summed in FP32 over runs of 8 and the runs in FP64
  double si = 0.0, so = 0.0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  while (i < n) {
    T run = 0;
    X run_in = 0;
#pragma unroll 4
    for (int r = 0; r < 8 && i < n; ++r, i += stride) {
      const X v = x[i];
      const T t = (T)v;
      y[i] = t;
      if constexpr (sizeof(X) == 8)
        si += v;
      else
        run_in += v;
      run += t;
    }
    if constexpr (sizeof(X) == 4) si += (double)run_in;
    so += (double)run;
  }
  si = block_sum(si);
  if (threadIdx.x == 0) pin[blockIdx.x] = si;
  so = block_sum(so);
  if (threadIdx.x == 0) pout[blockIdx.x] = so;
  if (tail.ticket) fin_tail(pin, tail);  // pout = pin + gridDim.x
}

template <typename F>
__global__ void k_nvec_affine(const double* __restrict__ in, double* __restrict__ out, int n, double a,
                              const double* __restrict__ shift, const F* __restrict__ f, double bcoef) {
  const double sh = shift ? *shift : 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double v = a * (in[i] - sh);
    if (f) v = fma(bcoef, (double)f[i], v);
    out[i] = v;
  }
}

template <typename T>
__global__ void k_sub_scalar(T* __restrict__ x, size_t n, const double* __restrict__ m) {
  const T v = (T)(*m);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    x[i] -= v;
}

// FP32 to FP32 with 16-byte aligned fields: 4-vectors.
__global__ void k_convert_f32v(const float* __restrict__ x, float* __restrict__ y, size_t n, float a,
                               const double* __restrict__ shift) {
  const float sh = shift ? (float)*shift : 0.f;
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
  const size_t n4 = n >> 2;
  for (size_t i = t; i < n4; i += stride) {
    float4 v = reinterpret_cast<const float4*>(x)[i];
    v.x = a * v.x + sh;
    v.y = a * v.y + sh;
    v.z = a * v.z + sh;
    v.w = a * v.w + sh;
    reinterpret_cast<float4*>(y)[i] = v;
  }
  for (size_t i = 4 * n4 + t; i < n; i += stride) y[i] = a * x[i] + sh;
}

// FP32 copy with sums (both equal to the sum of x), 16-byte aligned fields:
// 4-vectors summed in FP32 over runs of 2 vectors, the runs in FP64.
__global__ void __launch_bounds__(kRedThreads) k_copy_sum_f32v(const float* __restrict__ x, float* __restrict__ y,
                                                               size_t n, double* __restrict__ pin,
                                                               double* __restrict__ pout, FinTail tail) {
  double acc = 0.0;
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
  const size_t n4 = n >> 2;
  size_t i = t;
  for (; i + stride < n4; i += 2 * stride) {
    const float4 a = reinterpret_cast<const float4*>(x)[i];
    const float4 b = reinterpret_cast<const float4*>(x)[i + stride];
    reinterpret_cast<float4*>(y)[i] = a;
    reinterpret_cast<float4*>(y)[i + stride] = b;
    acc += (double)(((a.x + a.y) + (a.z + a.w)) + ((b.x + b.y) + (b.z + b.w)));
  }
  for (; i < n4; i += stride) {
    const float4 a = reinterpret_cast<const float4*>(x)[i];
    reinterpret_cast<float4*>(y)[i] = a;
    acc += (double)((a.x + a.y) + (a.z + a.w));
  }
  for (size_t k = 4 * n4 + t; k < n; k += stride) {
    y[k] = x[k];
    acc += (double)x[k];
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) {
    pin[blockIdx.x] = acc;
    pout[blockIdx.x] = acc;
  }
  if (tail.ticket) fin_tail(pin, tail);  // pout = pin + gridDim.x
}

template <typename Tx, typename Ty>
__global__ void k_convert(const Tx* __restrict__ x, Ty* __restrict__ y, size_t n, double a,
                          const double* __restrict__ shift) {
  const double sh = shift ? *shift : 0.0;
  if (a == 1.0 && sh == 0.0) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
      if constexpr (sizeof(Tx) == 8 && sizeof(Ty) == 4)
        y[i] = d2f_bits(x[i]);
      else if constexpr (sizeof(Tx) == 4 && sizeof(Ty) == 8)
        y[i] = f2d_bits(x[i]);
      else
        y[i] = (Ty)x[i];
    }
  } else if (sizeof(Ty) == 4 && sizeof(Tx) == 4) {
    const float af = (float)a, sf = (float)sh;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
      y[i] = (Ty)(af * (float)x[i] + sf);
  } else {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
      y[i] = (Ty)(a * (double)x[i] + sh);
  }
}

// FP32 fields in 4-vectors when both are 16-byte aligned (vec), the last
// n % 4 entries one by one.
template <typename E>
__global__ void k_axpby(E a, const E* __restrict__ x, E b, E* __restrict__ y, size_t n, int vec) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
  size_t i0 = 0;
  if constexpr (sizeof(E) == 4) {
    if (vec) {
      const size_t n4 = n >> 2;
      for (size_t i = t; i < n4; i += stride) {
        const float4 xv = reinterpret_cast<const float4*>(x)[i];
        float4 yv = b == 0.f ? make_float4(0.f, 0.f, 0.f, 0.f) : reinterpret_cast<const float4*>(y)[i];
        yv.x = b == 0.f ? a * xv.x : fmaf(a, xv.x, b * yv.x);
        yv.y = b == 0.f ? a * xv.y : fmaf(a, xv.y, b * yv.y);
        yv.z = b == 0.f ? a * xv.z : fmaf(a, xv.z, b * yv.z);
        yv.w = b == 0.f ? a * xv.w : fmaf(a, xv.w, b * yv.w);
        reinterpret_cast<float4*>(y)[i] = yv;
      }
      i0 = 4 * n4;
    }
  }
  for (size_t i = i0 + t; i < n; i += stride) y[i] = (b == (E)0) ? a * x[i] : fma(a, x[i], b * y[i]);
}

template <typename E>
__global__ void k_scale_by_inv(const E* __restrict__ x, E* __restrict__ y, size_t n, const double* __restrict__ den,
                               double num, int vec) {
  __shared__ E f;
  if (threadIdx.x == 0) f = (E)(num / *den);
  __syncthreads();
  const E ff = f;
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
  size_t i0 = 0;
  if constexpr (sizeof(E) == 4) {
    if (vec) {
      const size_t n4 = n >> 2;
      for (size_t i = t; i < n4; i += stride) {
        float4 v = reinterpret_cast<const float4*>(x)[i];
        v.x *= ff;
        v.y *= ff;
        v.z *= ff;
        v.w *= ff;
        reinterpret_cast<float4*>(y)[i] = v;
      }
      i0 = 4 * n4;
    }
  }
  for (size_t i = i0 + t; i < n; i += stride) y[i] = x[i] * ff;
}

// y = (float) x * sigma, with the sum of squares of y: per thread and across
// a warp in FP32 (terms of one sign; a thread holds about a hundred of a
// 256^3 field), across warps and blocks in FP64.
__global__ void __launch_bounds__(kRedThreads) k_convert_sq(const double* __restrict__ x, float* __restrict__ y,
                                                            size_t n, float sigma, const double* __restrict__ sigma_dev,
                                                            double* __restrict__ partial, FinTail tail) {
  if (sigma_dev) sigma = (float)*sigma_dev;
  float acc = 0.f;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
#pragma unroll 4
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride) {
    const float v = d2f_bits(x[i]) * sigma;
    y[i] = v;
    acc = fmaf(v, v, acc);
  }
  const double s = block_sum_f(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
  if (tail.ticket) fin_tail(partial, tail);
}

// x += a * (double) d: FP32 correction added to an FP64 field
__global__ void k_add_scaled(double a, const double* __restrict__ div_dev, const float* __restrict__ d,
                             double* __restrict__ x, size_t n) {
  if (div_dev) a = 1.0 / *div_dev;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    x[i] = fma(a, f2d_bits(d[i]), x[i]);
}

template <typename T>
__global__ void k_nonfinite(const T* __restrict__ x, size_t n, int* __restrict__ flag) {
  int bad = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    bad |= !isfinite(x[i]);
  bad = __syncthreads_or(bad);
  if (bad && threadIdx.x == 0) atomicOr(flag, 1);
}

inline int stream_blocks(size_t n, int threads) {
  size_t b = (n + threads - 1) / threads;
  const size_t cap = 152 * 16;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

// ---------------------------------------------------------------- launchers
template <typename T>
void launch_apply_A(const T* x, T* y, Dims d, Stencil st, cudaStream_t s) {
  const int c = pcls<T>(P_APPLY64, P_APPLY32);
  if constexpr (sizeof(T) == 4) {
    if (d.nx % 4 == 0 && aligned16(x) && aligned16(y)) {
      const int nx4 = d.nx / 4;
      const int tx = nx4 >= 32 ? 32 : nx4, ty = 256 / tx;
      const int bx = (nx4 + tx - 1) / tx, by = (d.ny + ty - 1) / ty;
      // about one wave of 8 resident blocks per SM
      int chunks = (152 * 8) / (bx * by);
      chunks = chunks < 1 ? 1 : chunks;
      int zc = (d.nz + chunks - 1) / chunks;
      zc = zc < 2 ? 2 : zc;
      dim3 g(bx, by, (d.nz + zc - 1) / zc);
      prof_begin(c, s);
      k_apply_f32v<<<g, dim3(tx, ty), 0, s>>>(x, y, d.nx, d.ny, d.nz, zc, (float)st.diag, (float)st.off);
      prof_end(c, s, "apply_A", 8.0 * d.n());
      return;
    }
  }
  dim3 g((d.nx + BX - 1) / BX, (d.ny + BY - 1) / BY, (d.nz + ZCH - 1) / ZCH);
  prof_begin(c, s);
  k_apply<T, false><<<g, dim3(BX, BY), 0, s>>>(x, nullptr, y, d.nx, d.ny, d.nz, (T)st.diag, (T)st.off);
  prof_end(c, s, "apply_A", 2.0 * sizeof(T) * d.n());
}

bool resid_fx_ok(Dims d, Stencil st) {
  return d.nx % 32 == 0 && d.ny % 8 == 0 && st.off > 0.0 && std::isfinite(st.diag) && std::isfinite(st.off);
}

template <typename T>
void launch_residual(const T* x, const T* b, T* y, Dims d, Stencil st, double* scratch, cudaStream_t s) {
  const int c = pcls<T>(P_APPLY64, P_APPLY32);
  if constexpr (sizeof(T) == 8) {
    if (scratch && resid_fx_ok(d, st)) {
      // the field's largest |x| (its bits) sets the fixed-point scale
      unsigned long long* xmax = reinterpret_cast<unsigned long long*>(scratch);
      IBRD_CUDA(cudaMemsetAsync(xmax, 0, sizeof(unsigned long long), s));
      prof_begin(P_REDUCE, s);
      k_absmax_bits<<<stream_blocks(d.n() / 2, 256), 256, 0, s>>>(x, d.n(), aligned16(x) ? 1 : 0, xmax);
      prof_end(P_REDUCE, s, "absmax", 8.0 * d.n());
      const double alpha = st.diag - 6.0 * st.off;
      constexpr int TY = 8;
      auto go = [&](auto kern, int cpt) {
        const int cols = (d.nx / (32 * cpt)) * (d.ny / TY);
        int chunks = (152 * 6) / cols;  // about one wave of 6 resident blocks per SM
        chunks = chunks < 1 ? 1 : chunks;
        int zc = (d.nz + chunks - 1) / chunks;
        zc = zc < 1 ? 1 : zc;
        dim3 g(d.nx / (32 * cpt), d.ny / TY, (d.nz + zc - 1) / zc);
        prof_begin(c, s);
        kern<<<g, dim3(32, TY), 0, s>>>(x, b, y, d.nx, d.ny, d.nz, zc, alpha, st.off, st.diag, xmax);
        prof_end(c, s, "residual_fx", 3.0 * sizeof(T) * d.n());
      };
      const bool vec = d.nx % 64 == 0 && aligned16(x) && aligned16(b) && aligned16(y);
      if (alpha != 0.0) {
        if (vec)
          go(k_resid_fx<TY, 2, true>, 2);
        else
          go(k_resid_fx<TY, 1, true>, 1);
      } else {
        if (vec)
          go(k_resid_fx<TY, 2, false>, 2);
        else
          go(k_resid_fx<TY, 1, false>, 1);
      }
      return;
    }
  }
  dim3 g((d.nx + BX - 1) / BX, (d.ny + BY - 1) / BY, (d.nz + ZCH - 1) / ZCH);
  prof_begin(c, s);
  k_apply<T, true><<<g, dim3(BX, BY), 0, s>>>(x, b, y, d.nx, d.ny, d.nz, (T)st.diag, (T)st.off);
  prof_end(c, s, "residual", 3.0 * sizeof(T) * d.n());
}

template <typename T>
void launch_coarse_solve(const T* table, const T* b, T* x, Dims dc, cudaStream_t s) {
  prof_begin(P_COARSE, s);
  k_coarse_solve<T><<<1, 256, 0, s>>>(table, b, x, dc.nx, dc.ny, dc.nz);
  prof_end(P_COARSE, s, "coarse_solve", 3.0 * sizeof(T) * dc.n());
}

template <typename T>
void launch_coarse_table(T* table, Dims dc, Stencil st, int singular, cudaStream_t s) {
  const int n = (int)dc.n();
  prof_begin(P_SETUP, s);
  k_coarse_table<T><<<(n + 127) / 128, 128, 0, s>>>(table, dc.nx, dc.ny, dc.nz, st.diag, st.off, singular);
  prof_end(P_SETUP, s, "coarse_table");
}

// tables, then (levels above 4096 cells) a scratch field of N floats
size_t hartley_table_size(Dims d) {
  const size_t t = (size_t)d.nx * d.nx + (size_t)d.ny * d.ny + (size_t)d.nz * d.nz + d.n();
  return d.n() > 4096 ? t + d.n() : t;
}

bool hartley_ok(Dims d) { return d.n() <= 32768 && d.nx <= 64 && d.ny <= 64 && d.nz <= 64; }

void launch_hartley_tables(float* tab, Dims d, Stencil st, int singular, cudaStream_t s) {
  const int m = (int)std::max<size_t>(d.n(), std::max(d.nx * d.nx, std::max(d.ny * d.ny, d.nz * d.nz)));
  prof_begin(P_SETUP, s);
  k_hartley_tables<<<(m + 127) / 128, 128, 0, s>>>(tab, d.nx, d.ny, d.nz, st.diag, st.off, singular);
  prof_end(P_SETUP, s, "hartley_tables");
}

void launch_hartley_solve(const float* tab, const float* b, const double* bshift, float* x, Dims d, cudaStream_t s) {
  if (d.n() > 4096) {
    // three launches through the scratch field behind the tables
    float* tmp = const_cast<float*>(tab) + ((size_t)d.nx * d.nx + (size_t)d.ny * d.ny + (size_t)d.nz * d.nz + d.n());
    const size_t smp = sizeof(float) * ((size_t)hartley_hsz((int)d.nx) + hartley_hsz((int)d.ny) +
                                        2 * (size_t)(d.nx + 1) * d.ny);
    const size_t smc = sizeof(float) * ((size_t)hartley_hsz((int)d.nz) + 2 * (size_t)(d.nx + 1) * d.nz);
    // sides up to 64 need more than the default 48 KB (at most 67 KB)
    static std::atomic<unsigned long long> attrp{0}, attrc{0};
    ensure_smem_attr((const void*)k_hartley_planes, 200 * 1024, attrp);
    ensure_smem_attr((const void*)k_hartley_columns, 200 * 1024, attrc);
    prof_begin(P_COARSE, s);
    k_hartley_planes<<<d.nz, 1024, smp, s>>>(b, bshift, tmp, tab, d.nx, d.ny);
    prof_end(P_COARSE, s, "hartley_planes", 8.0 * d.n());
    prof_begin(P_COARSE, s);
    k_hartley_columns<<<d.ny, 1024, smc, s>>>(tmp, tab, d.nx, d.ny, d.nz);
    prof_end(P_COARSE, s, "hartley_columns", 12.0 * d.n());
    prof_begin(P_COARSE, s);
    k_hartley_planes<<<d.nz, 1024, smp, s>>>(tmp, nullptr, x, tab, d.nx, d.ny);
    prof_end(P_COARSE, s, "hartley_planes", 8.0 * d.n());
    return;
  }
  const size_t pn = (size_t)(d.nx + 1) * (d.ny + 1) * d.nz;
  const size_t sm = sizeof(float) * ((size_t)d.nx * (d.nx + 1) + (size_t)d.ny * (d.ny + 1) +
                                     (size_t)d.nz * (d.nz + 1) + 2 * pn);
  static std::atomic<unsigned long long> attr0{0}, attr16{0};
  ensure_smem_attr((const void*)k_hartley_solve<0>, 200 * 1024, attr0);
  ensure_smem_attr((const void*)k_hartley_solve<16>, 200 * 1024, attr16);
  prof_begin(P_COARSE, s);
  if (d.nx == 16 && d.ny == 16 && d.nz == 16)
    k_hartley_solve<16><<<1, 1024, sm, s>>>(tab, b, bshift, x, d.nx, d.ny, d.nz);
  else
    k_hartley_solve<0><<<1, 1024, sm, s>>>(tab, b, bshift, x, d.nx, d.ny, d.nz);
  prof_end(P_COARSE, s, "hartley_solve", 8.0 * d.n());
}

template <typename T>
void launch_sum(const T* x, size_t n, double* partial, double* out, double scale, cudaStream_t s, unsigned* ticket) {
  FinTail t;
  if (ticket) t = FinTail{ticket, out, scale, nullptr, 1.0};
  prof_begin(P_DOT, s);
  k_sum_partial<T><<<kRedBlocks, kRedThreads, 0, s>>>(x, n, partial, t);
  prof_end(P_DOT, s, "sum_partial", 1.0 * sizeof(T) * n);
  if (ticket) return;
  prof_begin(P_REDUCE, s);
  k_finalize<<<1, kRedThreads, 0, s>>>(partial, kRedBlocks, out, scale);
  prof_end(P_REDUCE, s, "finalize");
}

void launch_finalize(const double* partial, int np, double* out, double scale, cudaStream_t s) {
  prof_begin(P_REDUCE, s);
  k_finalize<<<1, kRedThreads, 0, s>>>(partial, np, out, scale);
  prof_end(P_REDUCE, s, "finalize");
}

template <typename X, typename T>
void launch_convert_sum(const X* x, T* y, size_t n, double* partial, double* out_in, double* out_out,
                        cudaStream_t s, unsigned* ticket) {
  FinTail t;
  if (ticket) t = FinTail{ticket, out_in, 1.0, out_out, 1.0};
  prof_begin(P_VEC, s);
  if constexpr (sizeof(X) == 4 && sizeof(T) == 4) {
    if (aligned16(x) && aligned16(y))
      k_copy_sum_f32v<<<kRedBlocks, kRedThreads, 0, s>>>(x, y, n, partial, partial + kRedBlocks, t);
    else
      k_convert_sum<X, T><<<kRedBlocks, kRedThreads, 0, s>>>(x, y, n, partial, partial + kRedBlocks, t);
  } else {
    k_convert_sum<X, T><<<kRedBlocks, kRedThreads, 0, s>>>(x, y, n, partial, partial + kRedBlocks, t);
  }
  prof_end(P_VEC, s, "convert_sum", (double)(sizeof(X) + sizeof(T)) * n);
  if (ticket) return;
  launch_finalize(partial, kRedBlocks, out_in, 1.0, s);
  launch_finalize(partial + kRedBlocks, kRedBlocks, out_out, 1.0, s);
}

template <typename F>
void launch_nvec_affine(const double* in, double* out, int n, double a, const double* shift, const F* f,
                        double bcoef, cudaStream_t s) {
  if (n <= 0) return;
  prof_begin(P_VEC, s);
  k_nvec_affine<F><<<std::min(64, (n + 255) / 256), 256, 0, s>>>(in, out, n, a, shift, f, bcoef);
  prof_end(P_VEC, s, "nvec_affine", 24.0 * n);
}

template <typename E>
void launch_dot(const E* x, const E* y, size_t n, double* partial, double* out, double scale, cudaStream_t s,
                unsigned* ticket) {
  FinTail t;
  if (ticket) t = FinTail{ticket, out, scale, nullptr, 1.0};
  prof_begin(P_DOT, s);
  k_dot_partial<E><<<kRedBlocks, kRedThreads, 0, s>>>(x, y, n, partial, aligned16(x) && aligned16(y), t);
  prof_end(P_DOT, s, "dot_partial", 2.0 * sizeof(E) * n);
  if (ticket) return;
  prof_begin(P_REDUCE, s);
  k_finalize<<<1, kRedThreads, 0, s>>>(partial, kRedBlocks, out, scale);
  prof_end(P_REDUCE, s, "finalize");
}

template <typename T>
void launch_sub_scalar(T* x, size_t n, const double* mean, cudaStream_t s) {
  prof_begin(P_VEC, s);
  k_sub_scalar<T><<<stream_blocks(n, 256), 256, 0, s>>>(x, n, mean);
  prof_end(P_VEC, s, "sub_scalar", 2.0 * sizeof(T) * n);
}

template <typename Tx, typename Ty>
void launch_convert(const Tx* x, Ty* y, size_t n, double a, const double* shift, cudaStream_t s) {
  prof_begin(P_VEC, s);
  bool done = false;
  if constexpr (sizeof(Tx) == 4 && sizeof(Ty) == 4) {
    if (aligned16(x) && aligned16(y)) {
      k_convert_f32v<<<stream_blocks(n / 4 + 1, 256), 256, 0, s>>>(x, y, n, (float)a, shift);
      done = true;
    }
  }
  if (!done) k_convert<Tx, Ty><<<stream_blocks(n, 256), 256, 0, s>>>(x, y, n, a, shift);
  prof_end(P_VEC, s, "convert", (double)(sizeof(Tx) + sizeof(Ty)) * n);
}

template <typename E>
void launch_axpby(double a, const E* x, double b, E* y, size_t n, cudaStream_t s) {
  prof_begin(P_VEC, s);
  const int vec = aligned16(x) && aligned16(y);
  k_axpby<E><<<stream_blocks(vec && sizeof(E) == 4 ? n / 4 + 1 : n, 256), 256, 0, s>>>((E)a, x, (E)b, y, n, vec);
  prof_end(P_VEC, s, "axpby", (b == 0.0 ? 2.0 : 3.0) * sizeof(E) * n);
}

template <typename E>
void launch_scale_by_inv(const E* x, E* y, size_t n, const double* den, double num, cudaStream_t s) {
  prof_begin(P_VEC, s);
  const int vec = aligned16(x) && aligned16(y);
  k_scale_by_inv<E><<<stream_blocks(vec && sizeof(E) == 4 ? n / 4 + 1 : n, 256), 256, 0, s>>>(x, y, n, den, num,
                                                                                               vec);
  prof_end(P_VEC, s, "scale_by_inv", 2.0 * sizeof(E) * n);
}

void launch_convert_sq(const double* x, float* y, size_t n, double sigma, double* partial, double* out,
                       cudaStream_t s, unsigned* ticket) {
  FinTail t;
  if (ticket) t = FinTail{ticket, out, 1.0, nullptr, 1.0};
  prof_begin(P_VEC, s);
  k_convert_sq<<<kRedBlocks, kRedThreads, 0, s>>>(x, y, n, (float)sigma, nullptr, partial, t);
  prof_end(P_VEC, s, "convert_sq", 12.0 * n);
  if (ticket) return;
  launch_finalize(partial, kRedBlocks, out, 1.0, s);
}

void launch_convert_sq(const double* x, float* y, size_t n, const double* sigma_dev, double* partial, double* out,
                       cudaStream_t s, unsigned* ticket) {
  FinTail t;
  if (ticket) t = FinTail{ticket, out, 1.0, nullptr, 1.0};
  prof_begin(P_VEC, s);
  k_convert_sq<<<kRedBlocks, kRedThreads, 0, s>>>(x, y, n, 1.f, sigma_dev, partial, t);
  prof_end(P_VEC, s, "convert_sq", 12.0 * n);
  if (ticket) return;
  launch_finalize(partial, kRedBlocks, out, 1.0, s);
}

void launch_add_scaled(double a, const float* d, double* x, size_t n, cudaStream_t s) {
  prof_begin(P_VEC, s);
  k_add_scaled<<<stream_blocks(n, 256), 256, 0, s>>>(a, nullptr, d, x, n);
  prof_end(P_VEC, s, "add_scaled", 20.0 * n);
}

void launch_add_divided(const double* div_dev, const float* d, double* x, size_t n, cudaStream_t s) {
  prof_begin(P_VEC, s);
  k_add_scaled<<<stream_blocks(n, 256), 256, 0, s>>>(0.0, div_dev, d, x, n);
  prof_end(P_VEC, s, "add_scaled", 20.0 * n);
}

template <typename T>
void launch_nonfinite(const T* x, size_t n, int* flag, cudaStream_t s) {
  prof_begin(P_SETUP, s);
  k_nonfinite<T><<<stream_blocks(n, 256), 256, 0, s>>>(x, n, flag);
  prof_end(P_SETUP, s, "nonfinite", 1.0 * sizeof(T) * n);
}

#define IBRD_INST(T)                                                                                   \
  template void launch_apply_A<T>(const T*, T*, Dims, Stencil, cudaStream_t);                         \
  template void launch_residual<T>(const T*, const T*, T*, Dims, Stencil, double*, cudaStream_t);     \
  template void launch_coarse_solve<T>(const T*, const T*, T*, Dims, cudaStream_t);                   \
  template void launch_coarse_table<T>(T*, Dims, Stencil, int, cudaStream_t);                         \
  template void launch_sum<T>(const T*, size_t, double*, double*, double, cudaStream_t, unsigned*);   \
  template void launch_sub_scalar<T>(T*, size_t, const double*, cudaStream_t);                        \
  template void launch_nonfinite<T>(const T*, size_t, int*, cudaStream_t);
IBRD_INST(double)
IBRD_INST(float)
#undef IBRD_INST
template void launch_convert_sum<double, float>(const double*, float*, size_t, double*, double*, double*,
                                                cudaStream_t, unsigned*);
template void launch_convert_sum<double, double>(const double*, double*, size_t, double*, double*, double*,
                                                 cudaStream_t, unsigned*);
template void launch_convert_sum<float, float>(const float*, float*, size_t, double*, double*, double*,
                                               cudaStream_t, unsigned*);
template void launch_nvec_affine<double>(const double*, double*, int, double, const double*, const double*, double,
                                         cudaStream_t);
template void launch_nvec_affine<float>(const double*, double*, int, double, const double*, const float*, double,
                                        cudaStream_t);
template void launch_dot<double>(const double*, const double*, size_t, double*, double*, double, cudaStream_t,
                                 unsigned*);
template void launch_dot<float>(const float*, const float*, size_t, double*, double*, double, cudaStream_t,
                                unsigned*);
template void launch_axpby<double>(double, const double*, double, double*, size_t, cudaStream_t);
template void launch_axpby<float>(double, const float*, double, float*, size_t, cudaStream_t);
template void launch_scale_by_inv<double>(const double*, double*, size_t, const double*, double, cudaStream_t);
template void launch_scale_by_inv<float>(const float*, float*, size_t, const double*, double, cudaStream_t);
template void launch_convert<double, float>(const double*, float*, size_t, double, const double*, cudaStream_t);
template void launch_convert<float, double>(const float*, double*, size_t, double, const double*, cudaStream_t);
template void launch_convert<double, double>(const double*, double*, size_t, double, const double*, cudaStream_t);
template void launch_convert<float, float>(const float*, float*, size_t, double, const double*, cudaStream_t);

}  // namespace ibrd
