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

// Single-block exclusive scan of tile counts; also lists occupied tiles in
// increasing tile id. meta[0] = number of (tile, blob) pairs, meta[1] = number
// of occupied tiles.
__global__ void __launch_bounds__(1024) k_scan_tiles(const int* __restrict__ count, int nt,
                                                     int* __restrict__ offset, int* __restrict__ active,
                                                     int* __restrict__ meta) {
  __shared__ int s_sum[1024], s_act[1024];
  const int t = threadIdx.x;
  const int chunk = (nt + blockDim.x - 1) / blockDim.x;
  const int lo = min(nt, t * chunk), hi = min(nt, lo + chunk);
  int sum = 0, act = 0;
  for (int i = lo; i < hi; ++i) {
    sum += count[i];
    act += count[i] > 0;
  }
  s_sum[t] = sum;
  s_act[t] = act;
  __syncthreads();
  // Hillis-Steele inclusive scan over 1024 entries.
  for (int o = 1; o < 1024; o <<= 1) {
    int vs = 0, va = 0;
    if (t >= o) {
      vs = s_sum[t - o];
      va = s_act[t - o];
    }
    __syncthreads();
    s_sum[t] += vs;
    s_act[t] += va;
    __syncthreads();
  }
  int run = s_sum[t] - sum, ra = s_act[t] - act;
  for (int i = lo; i < hi; ++i) {
    offset[i] = run;
    run += count[i];
    if (count[i] > 0) active[ra++] = i;
  }
  if (t == blockDim.x - 1) {
    offset[nt] = s_sum[t];
    meta[0] = s_sum[t];
    meta[1] = s_act[t];
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

// Exclusive scan of n ints (single block), total into *total.
__global__ void __launch_bounds__(1024) k_scan_ints(const int* __restrict__ in, int n, int* __restrict__ out,
                                                    int* __restrict__ total) {
  __shared__ int s_sum[1024];
  const int t = threadIdx.x;
  const int chunk = (n + blockDim.x - 1) / blockDim.x;
  const int lo = min(n, t * chunk), hi = min(n, lo + chunk);
  int sum = 0;
  for (int i = lo; i < hi; ++i) sum += in[i];
  s_sum[t] = sum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const int v = t >= o ? s_sum[t - o] : 0;
    __syncthreads();
    s_sum[t] += v;
    __syncthreads();
  }
  int run = s_sum[t] - sum;
  for (int i = lo; i < hi; ++i) {
    out[i] = run;
    run += in[i];
  }
  if (t == blockDim.x - 1) {
    out[n] = s_sum[t];
    *total = s_sum[t];
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
  k_scan_tiles<<<1, 1024, 0, s>>>(b.tile_count, nt, b.tile_offset, b.active, b.d_meta);
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
    k_scan_ints<<<1, 1024, 0, s>>>(b.cell_count, b.n_active, b.cell_offset, b.d_meta + 2);
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
