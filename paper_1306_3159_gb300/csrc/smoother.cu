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
#include <cmath>

#include "internal.h"

namespace ibrd {
namespace {

__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

template <typename T, int TX, int TY, bool ZERO>
__global__ void __launch_bounds__(TX / 2 * TY) k_rb_sweep(const T* __restrict__ xin, T* __restrict__ xout,
                                                          const T* __restrict__ b, const double* __restrict__ bshift,
                                                          int nx, int ny, int nz, int zc, T inv_diag, T off) {
  constexpr int NT = TX / 2 * TY;
  constexpr int PW = TX + 4, PH = TY + 4;   // x plane with 2-cell halo
  constexpr int BW = TX + 2, BH = TY + 2;   // b plane with 1-cell halo
  constexpr int NPX = (PW * PH + NT - 1) / NT;
  constexpr int NPB = (BW * BH + NT - 1) / NT;
  __shared__ T px[4][PH][PW];
  __shared__ T pb[2][BH][BW];
  const int tid = threadIdx.x + threadIdx.y * (TX / 2);
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int k0 = blockIdx.z * zc, k1 = k0 + zc;
  const size_t plane = (size_t)nx * ny;
  const T sh = bshift ? (T)(*bshift) : (T)0;

  // global offsets (within a plane) of this thread's share of the halo tiles
  int offx[NPX], offb[NPB];
#pragma unroll
  for (int r = 0; r < NPX; ++r) {
    const int e = tid + r * NT;
    const int ly = e / PW, lx = e - ly * PW;
    offx[r] = (e < PW * PH) ? wrap(y0 - 2 + ly, ny) * nx + wrap(x0 - 2 + lx, nx) : -1;
  }
#pragma unroll
  for (int r = 0; r < NPB; ++r) {
    const int e = tid + r * NT;
    const int ly = e / BW, lx = e - ly * BW;
    offb[r] = (e < BW * BH) ? wrap(y0 - 1 + ly, ny) * nx + wrap(x0 - 1 + lx, nx) : -1;
  }
  auto load_x = [&](int k, T* reg) {
    const T* src = xin + (size_t)wrap(k, nz) * plane;
#pragma unroll
    for (int r = 0; r < NPX; ++r) reg[r] = (ZERO || offx[r] < 0) ? (T)0 : src[offx[r]];
  };
  auto store_x = [&](int k, const T* reg) {
    T* dst = &px[k & 3][0][0];
#pragma unroll
    for (int r = 0; r < NPX; ++r)
      if (offx[r] >= 0) dst[tid + r * NT] = reg[r];
  };
  auto load_b = [&](int k, T* reg) {
    const T* src = b + (size_t)wrap(k, nz) * plane;
#pragma unroll
    for (int r = 0; r < NPB; ++r) reg[r] = (offb[r] < 0) ? (T)0 : src[offb[r]] - sh;
  };
  auto store_b = [&](int k, const T* reg) {
    T* dst = &pb[k & 1][0][0];
#pragma unroll
    for (int r = 0; r < NPB; ++r)
      if (offb[r] >= 0) dst[tid + r * NT] = reg[r];
  };
  // red update of plane k on the tile plus a 1-cell ring (local rows/cols 1..TX+2)
  auto red = [&](int k) {
    const int par = (x0 + y0 + k) & 1;  // parity offset of local (lx, ly) -> global
    T(*P)[PW] = px[k & 3];
    T(*Pm)[PW] = px[(k + 3) & 3];
    T(*Pp)[PW] = px[(k + 1) & 3];
    T(*B)[BW] = pb[k & 1];
    constexpr int RW = (TX + 2) / 2;  // red cells per ring row
    for (int e = tid; e < RW * BH; e += NT) {
      const int ly = 1 + e / RW;
      const int q = e - (ly - 1) * RW;
      // local lx in [1, TX+2]; red when (lx - 2 + ly - 2 + par) even
      const int lx = 1 + 2 * q + ((1 + ly + par) & 1);
      const T s = ((P[ly][lx - 1] + P[ly][lx + 1]) + (P[ly - 1][lx] + P[ly + 1][lx])) + (Pm[ly][lx] + Pp[ly][lx]);
      P[ly][lx] = (B[ly - 1][lx - 1] + off * s) * inv_diag;
    }
  };
  // black update of plane k on the tile (local rows/cols 2..TX+1)
  auto black = [&](int k) {
    const int par = (x0 + y0 + k) & 1;
    T(*P)[PW] = px[k & 3];
    T(*Pm)[PW] = px[(k + 3) & 3];
    T(*Pp)[PW] = px[(k + 1) & 3];
    T(*B)[BW] = pb[k & 1];
    const int ly = 2 + threadIdx.y;
    const int lx = 2 + 2 * threadIdx.x + ((ly + par) & 1 ? 0 : 1);
    // black when (lx - 2 + ly - 2 + par) odd
    const T s = ((P[ly][lx - 1] + P[ly][lx + 1]) + (P[ly - 1][lx] + P[ly + 1][lx])) + (Pm[ly][lx] + Pp[ly][lx]);
    P[ly][lx] = (B[ly - 1][lx - 1] + off * s) * inv_diag;
  };
  auto write = [&](int k) {
    T(*P)[PW] = px[k & 3];
    const int ly = 2 + threadIdx.y;
    const int lx = 2 + 2 * threadIdx.x;
    T* dst = xout + (size_t)k * plane + (size_t)(y0 + threadIdx.y) * nx + x0 + 2 * threadIdx.x;
    dst[0] = P[ly][lx];
    dst[1] = P[ly][lx + 1];
  };

  T rx[NPX], rb[NPB];
  // prologue: planes k0-2 .. k0+1 of x, b at k0-1 and k0
  for (int k = k0 - 2; k <= k0 + 1; ++k) {
    load_x(k, rx);
    store_x(k, rx);
  }
  load_b(k0 - 1, rb);
  store_b(k0 - 1, rb);
  load_b(k0, rb);
  store_b(k0, rb);
  __syncthreads();
  red(k0 - 1);
  __syncthreads();
  for (int k = k0; k <= k1; ++k) {
    const bool pre_x = (k + 2 <= k1 + 1), pre_b = (k + 1 <= k1);
    if (pre_x) load_x(k + 2, rx);
    if (pre_b) load_b(k + 1, rb);
    red(k);
    __syncthreads();
    if (k > k0) {
      black(k - 1);
      __syncthreads();
      write(k - 1);
    }
    if (pre_x) store_x(k + 2, rx);
    if (pre_b) store_b(k + 1, rb);
    __syncthreads();
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
  const T w3 = (T)0.75, w1 = (T)0.25;
  const int Ix[3] = {wrap(I - 1, nxc), I, wrap(I + 1, nxc)};
  const int Jy[3] = {wrap(J - 1, nyc), J, wrap(J + 1, nyc)};
  const int Kz[3] = {wrap(K - 1, nzc), K, wrap(K + 1, nzc)};
  // x interpolation on the 3 x 3 coarse rows: west child (uses I-1), east child (uses I+1)
  T ex[3][3][2];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const T* row = xc + (Kz[c] * nyc + Jy[r]) * nxc;
      const T m = row[Ix[1]];
      ex[c][r][0] = w3 * m + w1 * row[Ix[0]];
      ex[c][r][1] = w3 * m + w1 * row[Ix[2]];
    }
#pragma unroll
  for (int dz = 0; dz < 2; ++dz)
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
      const int k = 2 * K + dz, j = 2 * J + dy;
      T* dst = x + ((size_t)k * ny + j) * nx + 2 * I;
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        // y then z interpolation
        const T yA = w3 * ex[1][1][dx] + w1 * ex[1][dy ? 2 : 0][dx];
        const T yB = w3 * ex[dz ? 2 : 0][1][dx] + w1 * ex[dz ? 2 : 0][dy ? 2 : 0][dx];
        dst[dx] += w3 * yA + w1 * yB;
      }
    }
}

inline int pick_zc(Dims d, int tiles_xy, int target_blocks) {
  for (int zc : {32, 16, 8, 4, 2}) {
    if (d.nz % zc == 0 && (long)tiles_xy * (d.nz / zc) >= target_blocks) return zc;
  }
  return (d.nz % 2 == 0) ? 2 : 1;
}

}  // namespace

template <typename T>
bool rb_sweep_fused_ok(Dims d) {
  return d.nx % 32 == 0 && d.ny % 8 == 0 && d.nz % 2 == 0 && d.nz >= 4;
}

template <typename T>
bool launch_rb_sweep(const T* xin, T* xout, const T* b, const double* bshift, Dims d, Stencil st, bool zero,
                     cudaStream_t s) {
  const int c = pcls<T>(P_RBGS64, P_RBGS32);
  const T inv = (T)(1.0 / st.diag), off = (T)st.off;
  if (rb_sweep_fused_ok<T>(d)) {
    const bool wide = (d.nx % 64 == 0);
    const int TX = wide ? 64 : 32, TY = 8;
    const int txy = (d.nx / TX) * (d.ny / TY);
    const int zc = pick_zc(d, txy, 2 * 152 * 4);
    dim3 g(d.nx / TX, d.ny / TY, d.nz / zc);
    prof_begin(c, s);
    if (wide) {
      if (zero)
        k_rb_sweep<T, 64, 8, true><<<g, dim3(32, 8), 0, s>>>(xin, xout, b, bshift, d.nx, d.ny, d.nz, zc, inv, off);
      else
        k_rb_sweep<T, 64, 8, false><<<g, dim3(32, 8), 0, s>>>(xin, xout, b, bshift, d.nx, d.ny, d.nz, zc, inv, off);
    } else {
      if (zero)
        k_rb_sweep<T, 32, 8, true><<<g, dim3(16, 8), 0, s>>>(xin, xout, b, bshift, d.nx, d.ny, d.nz, zc, inv, off);
      else
        k_rb_sweep<T, 32, 8, false><<<g, dim3(16, 8), 0, s>>>(xin, xout, b, bshift, d.nx, d.ny, d.nz, zc, inv, off);
    }
    // one read of x (skipped from zero), one read of b, one write of x
    prof_end(c, s, "rb_sweep", (zero ? 2.0 : 3.0) * sizeof(T) * d.n());
    return true;
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
    prof_end(c, s, "rb_half", (zero && colour == 0 ? 1.5 : 1.5) * sizeof(T) * d.n());
  }
  return false;
}

template <typename T>
void launch_resid_restrict(const T* x, const T* b, const double* bshift, T* bc, Dims d, Stencil st, cudaStream_t s) {
  const int nxc = d.nx / 2, nyc = d.ny / 2, nzc = d.nz / 2;
  dim3 blk(nxc >= 32 ? 32 : nxc, 4, 2);
  dim3 g((nxc + blk.x - 1) / blk.x, (nyc + blk.y - 1) / blk.y, (nzc + blk.z - 1) / blk.z);
  const int c = pcls<T>(P_RESTRICT64, P_RESTRICT32);
  prof_begin(c, s);
  k_resid_restrict<T><<<g, blk, 0, s>>>(x, b, bshift, bc, d.nx, d.ny, d.nz, (T)st.diag, (T)st.off);
  prof_end(c, s, "resid_restrict", 2.125 * sizeof(T) * d.n());
}

template <typename T>
void launch_prolong8(const T* xc, T* x, Dims d, cudaStream_t s) {
  const int nxc = d.nx / 2, nyc = d.ny / 2, nzc = d.nz / 2;
  dim3 blk(nxc >= 32 ? 32 : nxc, 4, 2);
  dim3 g((nxc + blk.x - 1) / blk.x, (nyc + blk.y - 1) / blk.y, (nzc + blk.z - 1) / blk.z);
  const int c = pcls<T>(P_PROLONG64, P_PROLONG32);
  prof_begin(c, s);
  k_prolong8<T><<<g, blk, 0, s>>>(xc, x, d.nx, d.ny, d.nz);
  prof_end(c, s, "prolong8", 2.125 * sizeof(T) * d.n());
}

#define IBRD_INST(T)                                                                                         \
  template bool launch_rb_sweep<T>(const T*, T*, const T*, const double*, Dims, Stencil, bool, cudaStream_t); \
  template void launch_resid_restrict<T>(const T*, const T*, const double*, T*, Dims, Stencil, cudaStream_t); \
  template void launch_prolong8<T>(const T*, T*, Dims, cudaStream_t);                                       \
  template bool rb_sweep_fused_ok<T>(Dims);
IBRD_INST(double)
IBRD_INST(float)
#undef IBRD_INST

}  // namespace ibrd
