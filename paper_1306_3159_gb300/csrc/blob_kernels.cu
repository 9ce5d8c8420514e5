// Blob kernels: per-blob Peskin weights, tile binning, spreading S and
// averaging J (Sec. II.A, Sec. III.A, Eq. tensor_product).
//
// Each blob touches 4 cells per axis (Peskin 4-point kernel; the 3-point
// kernel uses 3 and a zero fourth weight). Spreading never uses global
// atomics on the field: blobs are binned by the 8x8x8 cell tiles their
// support touches, and one CTA per occupied tile gathers, for each of its
// cells, the contributions of the tile's blobs in increasing blob index, so
// the result is deterministic and each field cell is written once.
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace ibrd {
namespace {

// Peskin 4-point kernel phi4(r), r in units of h (Peskin, Acta Numerica 2002).
__device__ __forceinline__ double phi4(double r) {
  r = fabs(r);
  if (r < 1.0) return (3.0 - 2.0 * r + sqrt(1.0 + 4.0 * r - 4.0 * r * r)) * 0.125;
  if (r < 2.0) return (5.0 - 2.0 * r - sqrt(-7.0 + 12.0 * r - 4.0 * r * r)) * 0.125;
  return 0.0;
}

// Peskin 3-point kernel phi3(r) (Roma, Peskin and Berger 1999).
__device__ __forceinline__ double phi3(double r) {
  r = fabs(r);
  if (r <= 0.5) return (1.0 + sqrt(1.0 - 3.0 * r * r)) / 3.0;
  if (r < 1.5) {
    const double t = 1.0 - r;
    return (5.0 - 3.0 * r - sqrt(1.0 - 3.0 * t * t)) / 6.0;
  }
  return 0.0;
}

__device__ __forceinline__ int pmod(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

// Per blob and axis: wrapped position, 4 wrapped cell indices, 4 weights.
__global__ void k_blob_prep(const double* __restrict__ qin, int n, int nx, int ny, int nz, double h, int width,
                            double* __restrict__ q, int* __restrict__ idx, double* __restrict__ w64,
                            float* __restrict__ w32) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  const int dims[3] = {nx, ny, nz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double L = dims[a] * h;
    double p = qin[3 * b + a];
    p -= floor(p / L) * L;
    if (p >= L) p -= L;
    if (p < 0.0) p = 0.0;
    q[3 * b + a] = p;
    const double u = p / h - 0.5;  // position in cell-index units (centres at integers)
    int base;
    if (width == 4)
      base = (int)floor(u) - 1;
    else
      base = (int)floor(u + 0.5) - 1;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const double r = u - (double)(base + s);
      double wt;
      if (width == 4)
        wt = phi4(r);
      else
        wt = (s < 3) ? phi3(r) : 0.0;
      const int o = (b * 3 + a) * 4 + s;
      idx[o] = pmod(base + s, dims[a]);
      w64[o] = wt;
      w32[o] = (float)wt;
    }
  }
}

// Distinct tiles touched along one axis (at most 4).
__device__ __forceinline__ int axis_tiles(const int* __restrict__ ix, int* t) {
  int m = 0;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int v = ix[s] / kTile;
    bool seen = false;
    for (int u = 0; u < m; ++u) seen |= (t[u] == v);
    if (!seen) t[m++] = v;
  }
  return m;
}

template <bool FILL>
__global__ void k_tile_pairs(const int* __restrict__ idx, int n, int ntx, int nty, int* __restrict__ count,
                             const int* __restrict__ offset, int* __restrict__ cursor, int* __restrict__ list) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  int tx[4], ty[4], tz[4];
  const int mx = axis_tiles(idx + (b * 3 + 0) * 4, tx);
  const int my = axis_tiles(idx + (b * 3 + 1) * 4, ty);
  const int mz = axis_tiles(idx + (b * 3 + 2) * 4, tz);
  for (int c = 0; c < mz; ++c)
    for (int bb = 0; bb < my; ++bb)
      for (int a = 0; a < mx; ++a) {
        const int t = tx[a] + ntx * (ty[bb] + nty * tz[c]);
        if (FILL) {
          const int pos = offset[t] + atomicAdd(&cursor[t], 1);
          list[pos] = b;
        } else {
          atomicAdd(&count[t], 1);
        }
      }
}

// Single-block exclusive scan of n counts into offset[0..n] (offset[n] = the
// total, also *total), optionally listing the indices with a nonzero count in
// increasing order into active (their number into *nactive). The counts pass
// through shared memory in segments of 4096, loaded and stored coalesced;
// thread t scans entries 4t .. 4t + 3 of a segment, warps scan their threads'
// sums with shuffles, warp 0 the warps' totals, and a carry joins segments.
constexpr int kScanSeg = 4096;
template <bool ACTIVE>
__global__ void __launch_bounds__(1024) k_scan_counts(const int* __restrict__ count, int n, int* __restrict__ offset,
                                                      int* __restrict__ total, int* __restrict__ active,
                                                      int* __restrict__ nactive) {
  __shared__ int sc[kScanSeg];
  __shared__ int wsum[32], wact[32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  int carry = 0, carry_a = 0;
  for (int base = 0; base < n; base += kScanSeg) {
    const int len = min(kScanSeg, n - base);
    for (int k = t; k < kScanSeg; k += blockDim.x) sc[k] = k < len ? count[base + k] : 0;
    __syncthreads();
    const int v0 = sc[4 * t], v1 = sc[4 * t + 1], v2 = sc[4 * t + 2], v3 = sc[4 * t + 3];
    const int sum = (v0 + v1) + (v2 + v3);
    const int act = ACTIVE ? (v0 > 0) + (v1 > 0) + (v2 > 0) + (v3 > 0) : 0;
    int is = sum, ia = act;  // inclusive scans over the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int us = __shfl_up_sync(0xffffffffu, is, o), ua = __shfl_up_sync(0xffffffffu, ia, o);
      if (lane >= o) is += us, ia += ua;
    }
    if (lane == 31) wsum[w] = is, wact[w] = ia;
    __syncthreads();
    if (w == 0) {
      int ws = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0, wa = lane < (int)(blockDim.x >> 5) ? wact[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int us = __shfl_up_sync(0xffffffffu, ws, o), ua = __shfl_up_sync(0xffffffffu, wa, o);
        if (lane >= o) ws += us, wa += ua;
      }
      wsum[lane] = ws;  // inclusive over warps
      wact[lane] = wa;
    }
    __syncthreads();
    const int before = carry + (w > 0 ? wsum[w - 1] : 0) + is - sum;
    sc[4 * t] = before;
    sc[4 * t + 1] = before + v0;
    sc[4 * t + 2] = before + v0 + v1;
    sc[4 * t + 3] = before + v0 + v1 + v2;
    if (ACTIVE) {
      int ra = carry_a + (w > 0 ? wact[w - 1] : 0) + ia - act;
      const int i0 = base + 4 * t;
      if (v0 > 0) active[ra++] = i0;
      if (v1 > 0) active[ra++] = i0 + 1;
      if (v2 > 0) active[ra++] = i0 + 2;
      if (v3 > 0) active[ra] = i0 + 3;
    }
    carry += wsum[(blockDim.x >> 5) - 1];
    carry_a += wact[(blockDim.x >> 5) - 1];
    __syncthreads();
    for (int k = t; k < len; k += blockDim.x) offset[base + k] = sc[k];
    __syncthreads();
  }
  if (t == 0) {
    offset[n] = carry;
    *total = carry;
    if (ACTIVE) *nactive = carry_a;
  }
}

// Sort the blob list of each occupied tile by blob index (insertion sort).
__global__ void k_tile_sort(const int* __restrict__ active, int na, const int* __restrict__ offset,
                            int* __restrict__ list) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= na) return;
  const int t = active[a];
  const int lo = offset[t], hi = offset[t + 1];
  for (int i = lo + 1; i < hi; ++i) {
    const int v = list[i];
    int j = i - 1;
    while (j >= lo && list[j] > v) {
      list[j + 1] = list[j];
      --j;
    }
    list[j + 1] = v;
  }
}

// Is cell (i, j, k) inside the support of blob b? (offsets from the blob's
// first support cell, per axis, in [0, 4))
__device__ __forceinline__ bool covers(const int* __restrict__ ib, int i, int j, int k, int nx, int ny, int nz,
                                       int& dx, int& dy, int& dz) {
  dx = i - ib[0];
  dy = j - ib[4];
  dz = k - ib[8];
  dx += dx < 0 ? nx : 0;
  dy += dy < 0 ? ny : 0;
  dz += dz < 0 ? nz : 0;
  return (unsigned)dx < 4u && (unsigned)dy < 4u && (unsigned)dz < 4u;
}

// Pass 1 (count) and pass 2 (fill) of the covered-cell list: one CTA per
// occupied tile, one thread per tile cell.
template <bool FILL>
__global__ void __launch_bounds__(512) k_cover(const int* __restrict__ active, const int* __restrict__ offset,
                                               const int* __restrict__ list, const int* __restrict__ idx, int nx,
                                               int ny, int nz, int ntx, int nty, int* __restrict__ count,
                                               const int* __restrict__ coff, int* __restrict__ cells,
                                               int* __restrict__ cell_tile) {
  const int a = blockIdx.x;
  const int tile = active[a];
  const int tx = tile % ntx, ty = (tile / ntx) % nty, tz = tile / (ntx * nty);
  const int i = tx * kTile + threadIdx.x, j = ty * kTile + threadIdx.y, k = tz * kTile + threadIdx.z;
  bool hit = false;
  if (i < nx && j < ny && k < nz) {
    for (int p = offset[tile]; p < offset[tile + 1] && !hit; ++p) {
      int dx, dy, dz;
      hit = covers(idx + list[p] * 12, i, j, k, nx, ny, nz, dx, dy, dz);
    }
  }
  if (!FILL) {
    const int c = __syncthreads_count(hit);
    if (threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0) count[a] = c;
    return;
  }
  // rank of this cell among the block's covered cells, in thread order
  __shared__ int wsum[16];
  const int t = threadIdx.x + kTile * (threadIdx.y + kTile * threadIdx.z);
  const unsigned bal = __ballot_sync(0xffffffffu, hit);
  const int lane = t & 31, w = t >> 5;
  if (lane == 0) wsum[w] = __popc(bal);
  __syncthreads();
  int base = 0;
  for (int u = 0; u < w; ++u) base += wsum[u];
  if (hit) {
    const int r = coff[a] + base + __popc(bal & ((1u << lane) - 1u));
    cells[r] = (k * ny + j) * nx + i;
    cell_tile[r] = tile;
  }
}

// One thread per covered cell: gathers the contributions of its tile's blobs
// in increasing blob index.
template <typename T, typename W, typename L>
__global__ void __launch_bounds__(256) k_spread(const int* __restrict__ cells, const int* __restrict__ cell_tile,
                                                int n_cells, const int* __restrict__ offset,
                                                const int* __restrict__ list, const int* __restrict__ idx,
                                                const W* __restrict__ wt, const L* __restrict__ lam,
                                                const double* __restrict__ cval, const double* __restrict__ coef,
                                                double scale, T* __restrict__ out, int nx, int ny, int nz) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_cells) return;
  const int cell = cells[t], tile = cell_tile[t];
  const int i = cell % nx, j = (cell / nx) % ny, k = cell / (nx * ny);
  W acc = 0;
  for (int p = offset[tile]; p < offset[tile + 1]; ++p) {
    const int b = list[p];
    int dx, dy, dz;
    if (covers(idx + b * 12, i, j, k, nx, ny, nz, dx, dy, dz)) {
      const W* wb = wt + b * 12;
      const double l = lam ? (double)lam[b] : *cval;
      const W amp = (W)(coef ? coef[b] * l : l);
      acc += amp * ((wb[dx] * wb[4 + dy]) * wb[8 + dz]);
    }
  }
  out[cell] += (T)scale * (T)acc;
}

// One warp per blob: lanes cover the 4x4x4 support, two cells each.
template <typename T, typename W, typename O>
__global__ void k_interp(const int* __restrict__ idx, const W* __restrict__ wt, const T* __restrict__ x,
                         double scale, O* __restrict__ out, int n, int nx, int ny) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n) return;
  const int* ib = idx + warp * 12;
  const W* wb = wt + warp * 12;
  W v = 0;
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const int s = lane * 2 + t;
    const int sx = s & 3, sy = (s >> 2) & 3, sz = s >> 4;
    const size_t p = ((size_t)ib[8 + sz] * ny + ib[4 + sy]) * nx + ib[sx];
    v += (wb[sx] * wb[4 + sy]) * wb[8 + sz] * (W)x[p];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) out[warp] = (O)(scale * (double)v);
}

}  // namespace

void blobs_setup(BlobSet& b, Dims d, double h, const double* q_in, int n, cudaStream_t s) {
  b.ntx = (d.nx + kTile - 1) / kTile;
  b.nty = (d.ny + kTile - 1) / kTile;
  b.ntz = (d.nz + kTile - 1) / kTile;
  const int nt = b.ntx * b.nty * b.ntz;
  if (b.ntiles != nt) {
    cudaFree(b.tile_count);
    cudaFree(b.tile_offset);
    cudaFree(b.tile_cursor);
    cudaFree(b.active);
    b.tile_count = b.tile_offset = b.tile_cursor = b.active = nullptr;
    IBRD_CUDA(cudaMalloc(&b.tile_count, sizeof(int) * nt));
    IBRD_CUDA(cudaMalloc(&b.tile_offset, sizeof(int) * (nt + 1)));
    IBRD_CUDA(cudaMalloc(&b.tile_cursor, sizeof(int) * nt));
    IBRD_CUDA(cudaMalloc(&b.active, sizeof(int) * nt));
    cudaFree(b.cell_count);
    cudaFree(b.cell_offset);
    b.cell_count = b.cell_offset = nullptr;
    IBRD_CUDA(cudaMalloc(&b.cell_count, sizeof(int) * (nt + 1)));
    IBRD_CUDA(cudaMalloc(&b.cell_offset, sizeof(int) * (nt + 1)));
    b.ntiles = nt;
  }
  if (!b.d_meta) IBRD_CUDA(cudaMalloc(&b.d_meta, sizeof(int) * 4));
  if (n > b.cap) {
    cudaFree(b.q);
    cudaFree(b.idx);
    cudaFree(b.w64);
    cudaFree(b.w32);
    b.q = nullptr;
    b.idx = nullptr;
    b.w64 = nullptr;
    b.w32 = nullptr;
    IBRD_CUDA(cudaMalloc(&b.q, sizeof(double) * 3 * n));
    IBRD_CUDA(cudaMalloc(&b.idx, sizeof(int) * 12 * n));
    IBRD_CUDA(cudaMalloc(&b.w64, sizeof(double) * 12 * n));
    IBRD_CUDA(cudaMalloc(&b.w32, sizeof(float) * 12 * n));
    b.cap = n;
  }
  b.n = n;
  IBRD_CUDA(cudaMemsetAsync(b.tile_count, 0, sizeof(int) * nt, s));
  IBRD_CUDA(cudaMemsetAsync(b.tile_cursor, 0, sizeof(int) * nt, s));
  if (n > 0) {
    prof_begin(P_SETUP, s);
    k_blob_prep<<<(n + 127) / 128, 128, 0, s>>>(q_in, n, d.nx, d.ny, d.nz, h, b.width, b.q, b.idx, b.w64, b.w32);
    prof_end(P_SETUP, s, "blob_prep");
    prof_begin(P_SETUP, s);
    k_tile_pairs<false><<<(n + 127) / 128, 128, 0, s>>>(b.idx, n, b.ntx, b.nty, b.tile_count, nullptr, nullptr,
                                                         nullptr);
    prof_end(P_SETUP, s, "tile_count");
  }
  prof_begin(P_SETUP, s);
  k_scan_counts<true><<<1, 1024, 0, s>>>(b.tile_count, nt, b.tile_offset, b.d_meta, b.active, b.d_meta + 1);
  prof_end(P_SETUP, s, "scan_tiles");
  int meta[2];
  IBRD_CUDA(cudaMemcpyAsync(meta, b.d_meta, sizeof(meta), cudaMemcpyDeviceToHost, s));
  IBRD_CUDA(cudaStreamSynchronize(s));
  b.n_active = meta[1];
  if (meta[0] > b.pair_cap) {
    cudaFree(b.tile_blobs);
    b.tile_blobs = nullptr;
    IBRD_CUDA(cudaMalloc(&b.tile_blobs, sizeof(int) * meta[0]));
    b.pair_cap = meta[0];
  }
  if (n > 0) {
    prof_begin(P_SETUP, s);
    k_tile_pairs<true><<<(n + 127) / 128, 128, 0, s>>>(b.idx, n, b.ntx, b.nty, nullptr, b.tile_offset,
                                                        b.tile_cursor, b.tile_blobs);
    prof_end(P_SETUP, s, "tile_fill");
    if (b.n_active > 0) {
      prof_begin(P_SETUP, s);
      k_tile_sort<<<(b.n_active + 127) / 128, 128, 0, s>>>(b.active, b.n_active, b.tile_offset, b.tile_blobs);
      prof_end(P_SETUP, s, "tile_sort");
    }
  }
  // covered-cell list (count per occupied tile, scan, ordered fill)
  b.n_cells = 0;
  if (n > 0 && b.n_active > 0) {
    const dim3 tb(kTile, kTile, kTile);
    prof_begin(P_SETUP, s);
    k_cover<false><<<b.n_active, tb, 0, s>>>(b.active, b.tile_offset, b.tile_blobs, b.idx, d.nx, d.ny, d.nz, b.ntx,
                                             b.nty, b.cell_count, nullptr, nullptr, nullptr);
    prof_end(P_SETUP, s, "cover_count");
    prof_begin(P_SETUP, s);
    k_scan_counts<false><<<1, 1024, 0, s>>>(b.cell_count, b.n_active, b.cell_offset, b.d_meta + 2, nullptr,
                                            nullptr);
    prof_end(P_SETUP, s, "cover_scan");
    int nc = 0;
    IBRD_CUDA(cudaMemcpyAsync(&nc, b.d_meta + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
    IBRD_CUDA(cudaStreamSynchronize(s));
    if (nc > b.cell_cap || !b.cells) {
      cudaFree(b.cells);
      cudaFree(b.cell_tile);
      b.cells = b.cell_tile = nullptr;
      const int cap = std::max(nc, 1);
      IBRD_CUDA(cudaMalloc(&b.cells, sizeof(int) * cap));
      IBRD_CUDA(cudaMalloc(&b.cell_tile, sizeof(int) * cap));
      b.cell_cap = cap;
    }
    prof_begin(P_SETUP, s);
    k_cover<true><<<b.n_active, tb, 0, s>>>(b.active, b.tile_offset, b.tile_blobs, b.idx, d.nx, d.ny, d.nz, b.ntx,
                                            b.nty, nullptr, b.cell_offset, b.cells, b.cell_tile);
    prof_end(P_SETUP, s, "cover_fill");
    b.n_cells = nc;
  }
}

template <typename T, typename L>
void launch_spread(const BlobSet& b, Dims d, const L* lam, const double* coef, double scale, T* out,
                   int accumulate, cudaStream_t s) {
  if (!accumulate) IBRD_CUDA(cudaMemsetAsync(out, 0, sizeof(T) * d.n(), s));
  if (b.n == 0 || b.n_cells == 0) return;
  const int c = pcls<T>(P_SPREAD64, P_SPREAD32);
  const int blocks = (b.n_cells + 255) / 256;
  prof_begin(c, s);
  if (sizeof(T) == 8)
    k_spread<T, double, L><<<blocks, 256, 0, s>>>(b.cells, b.cell_tile, b.n_cells, b.tile_offset, b.tile_blobs,
                                                  b.idx, b.w64, lam, nullptr, coef, scale, out, d.nx, d.ny, d.nz);
  else
    k_spread<T, float, L><<<blocks, 256, 0, s>>>(b.cells, b.cell_tile, b.n_cells, b.tile_offset, b.tile_blobs,
                                                 b.idx, b.w32, lam, nullptr, coef, scale, out, d.nx, d.ny, d.nz);
  prof_end(c, s, "spread", (double)b.n_cells * (2.0 * sizeof(T) + 8.0) + (double)b.n * (48.0 + 12.0 * sizeof(T) + 16.0));
}

template <typename T>
void launch_spread_const(const BlobSet& b, Dims d, const double* cval, double scale, T* out, cudaStream_t s) {
  if (b.n == 0 || b.n_cells == 0) return;
  const int c = pcls<T>(P_SPREAD64, P_SPREAD32);
  const int blocks = (b.n_cells + 255) / 256;
  prof_begin(c, s);
  if (sizeof(T) == 8)
    k_spread<T, double, double><<<blocks, 256, 0, s>>>(b.cells, b.cell_tile, b.n_cells, b.tile_offset,
                                                       b.tile_blobs, b.idx, b.w64, nullptr, cval, nullptr, scale,
                                                       out, d.nx, d.ny, d.nz);
  else
    k_spread<T, float, double><<<blocks, 256, 0, s>>>(b.cells, b.cell_tile, b.n_cells, b.tile_offset,
                                                      b.tile_blobs, b.idx, b.w32, nullptr, cval, nullptr, scale,
                                                      out, d.nx, d.ny, d.nz);
  prof_end(c, s, "spread_const", (double)b.n_cells * (2.0 * sizeof(T) + 8.0) + (double)b.n * (48.0 + 12.0 * sizeof(T)));
}

template <typename T, typename O>
void launch_interp(const BlobSet& b, Dims d, const T* x, double scale, O* out, cudaStream_t s) {
  if (b.n == 0) return;
  const int threads = 256;
  const int blocks = (int)(((size_t)b.n * 32 + threads - 1) / threads);
  const int c = pcls<T>(P_INTERP64, P_INTERP32);
  prof_begin(c, s);
  if (sizeof(T) == 8)
    k_interp<T, double, O><<<blocks, threads, 0, s>>>(b.idx, b.w64, x, scale, out, b.n, d.nx, d.ny);
  else
    k_interp<T, float, O><<<blocks, threads, 0, s>>>(b.idx, b.w32, x, scale, out, b.n, d.nx, d.ny);
  prof_end(c, s, "interp", (double)b.n * (64.0 * sizeof(T) + 48.0 + 12.0 * sizeof(T) + 8.0));
}

template void launch_spread<double, double>(const BlobSet&, Dims, const double*, const double*, double, double*,
                                            int, cudaStream_t);
template void launch_spread<float, double>(const BlobSet&, Dims, const double*, const double*, double, float*, int,
                                           cudaStream_t);
template void launch_spread<float, float>(const BlobSet&, Dims, const float*, const double*, double, float*, int,
                                          cudaStream_t);
template void launch_spread_const<double>(const BlobSet&, Dims, const double*, double, double*, cudaStream_t);
template void launch_spread_const<float>(const BlobSet&, Dims, const double*, double, float*, cudaStream_t);
template void launch_interp<double, double>(const BlobSet&, Dims, const double*, double, double*, cudaStream_t);
template void launch_interp<float, double>(const BlobSet&, Dims, const float*, double, double*, cudaStream_t);
template void launch_interp<float, float>(const BlobSet&, Dims, const float*, double, float*, cudaStream_t);

}  // namespace ibrd
