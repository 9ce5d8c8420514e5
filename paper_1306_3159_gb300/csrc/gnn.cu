// Learned multiplier predictor: a graph network over each blob's neighbours
// that predicts the relative sink strengths lambda_i / <lambda> of the
// diffusion-limited saddle point (Eq. saddle_point), used as the initial
// guess of the multipliers. The paper names a good treatment of the Schur
// complement for many blobs as open (Sec. III.E, Sec. V); this network is
// trained on (configuration, lambda) pairs produced by the saddle solver.
//
// Definition (width H = 64, K = 16 radial bases, L = 3 message-passing
// layers, cutoff R, s = r / R, f_c = (1 - s)^2,
// b_k = f_c exp(-((s - k/(K-1)) / sigma)^2), sigma = 1.5/(K-1)):
//   x_i  = sum_j b(r_ij)
//   h0_i = relu(W0 x_i + c0)
//   layer l: m_i = sum_j f_c(r_ij) relu(E_l b(r_ij) + e_l) * h_{l-1,j}
//            h_{l,i} = h_{l-1,i} + relu(W_l m_i + V_l h_{l-1,i} + c_l)
//   y_i  = o . h_{L,i} + o0,   lambda0_i = T softmax(y)_i
// Loss: <((y - <y>) - (t - <t>))^2>, t = log lambda. Adam updates.
//
// Training (and ibrd_gnn_forward) runs in FP32: one warp per blob (lane l
// owns hidden rows l and l + 32); the neighbour lists are symmetric, so the
// backward pass gathers every edge contribution at its own node (no
// atomics). Inference (ibrd_gnn_predict) runs the dense products on the
// tensor cores with bfloat16 operands and FP32 accumulation (mma.sync
// m16n8k16): the edge filters E_l b as 16-edge x 16-basis x 64 tiles, one
// warp per blob, and the node update [W_l V_l] [m; h] as 16-blob x 128 x 64
// tiles, one warp per 16 blobs, the weights staged in shared memory; biases,
// relus and the residual sums stay FP32, the embedding and output too.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

namespace ibrd {
namespace {

constexpr int H = 64;
constexpr int K = 16;
constexpr int L = 3;
constexpr float kSigmaInv = (K - 1) / 1.5f;
// flat parameter layout (as in the FP64 reference): W0, c0, per layer
// (E, e, W, V, c), o, o0
constexpr int OFF_W0 = 0;
constexpr int OFF_C0 = OFF_W0 + H * K;
constexpr int LSZ = H * K + H + 2 * H * H + H;
__host__ __device__ constexpr int lbase(int l) { return OFF_C0 + H + (l - 1) * LSZ; }  // l = 1 .. L
__host__ __device__ constexpr int offE(int l) { return lbase(l); }
__host__ __device__ constexpr int offEB(int l) { return lbase(l) + H * K; }
__host__ __device__ constexpr int offW(int l) { return lbase(l) + H * K + H; }
__host__ __device__ constexpr int offV(int l) { return lbase(l) + H * K + H + H * H; }
__host__ __device__ constexpr int offC(int l) { return lbase(l) + H * K + H + 2 * H * H; }
constexpr int OFF_O = OFF_C0 + H + L * LSZ;
constexpr int OFF_O0 = OFF_O + H;
constexpr int NPARAM = OFF_O0 + 1;
constexpr int kWarps = 8;  // blobs per CTA
constexpr int kPad = H + 1; // shared-memory row stride of the 64 x 64 matrices
// bfloat16 weights for inference, per layer: E_l (H x K), then [W_l V_l] (H x 2H)
constexpr int BLSZ = H * K + 2 * H * H;

__device__ __forceinline__ float basis_k(float s, int k) {
  const float fc = (1.f - s) * (1.f - s);
  const float t = (s - (float)k / (float)(K - 1)) * kSigmaInv;
  return fc * expf(-t * t);
}

// Minimum-image distance of blobs i and j (FP64, no contraction so that the
// neighbour decision is the reference's bit for bit).
__device__ __forceinline__ double min_image_dist(const double* q, int i, int j, double lx, double ly,
                                                 double lz) {
  double dx = __dsub_rn(q[3 * j + 0], q[3 * i + 0]);
  double dy = __dsub_rn(q[3 * j + 1], q[3 * i + 1]);
  double dz = __dsub_rn(q[3 * j + 2], q[3 * i + 2]);
  dx = __dsub_rn(dx, __dmul_rn(lx, rint(__ddiv_rn(dx, lx))));
  dy = __dsub_rn(dy, __dmul_rn(ly, rint(__ddiv_rn(dy, ly))));
  dz = __dsub_rn(dz, __dmul_rn(lz, rint(__ddiv_rn(dz, lz))));
  return sqrt(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
}

// FP32 copies of the positions (x, y, z, 0) for the neighbour screen, each
// coordinate first brought into the box (about [0, L): the screen takes the
// minimum image anyway), so that its FP32 rounding is a few ulps of L.
__global__ void k_gnn_pos32(const double* __restrict__ q, int n, double lx, double ly, double lz,
                            float4* __restrict__ p) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double x = q[3 * j], y = q[3 * j + 1], z = q[3 * j + 2];
  p[j] = make_float4((float)(x - lx * floor(x * (1.0 / lx))), (float)(y - ly * floor(y * (1.0 / ly))),
                     (float)(z - lz * floor(z * (1.0 / lz))), 0.f);
}

constexpr int kNbTile = 1024;  // positions staged in shared memory per pass

// One candidate pair of the neighbour test: FP32 minimum-image distance
// first; only pairs within a margin of R take the exact FP64 test, so the
// neighbour sets are the FP64 definition's, and a stored distance is the FP32
// one (within a few ulps of the box side) away from the boundary.
struct PairScreen {
  float flx, fly, flz, ilx, ily, ilz, rs2, ri2;
  double lx, ly, lz, R;
  __device__ PairScreen(double lx_, double ly_, double lz_, double R_, float margin)
      : lx(lx_), ly(ly_), lz(lz_), R(R_) {
    flx = (float)lx;
    fly = (float)ly;
    flz = (float)lz;
    ilx = 1.f / flx;
    ily = 1.f / fly;
    ilz = 1.f / flz;
    const float rs = (float)R + margin, ri = (float)R - margin;
    rs2 = rs * rs;
    ri2 = ri > 0.f ? ri * ri : 0.f;
  }
  // the distance of a neighbour pair, -1 for any other
  __device__ __forceinline__ float dist(const double* q, int i, int j, float4 pi, float4 pj) const {
    float dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
    dx -= flx * rintf(dx * ilx);
    dy -= fly * rintf(dy * ily);
    dz -= flz * rintf(dz * ilz);
    const float d2 = dx * dx + dy * dy + dz * dz;
    if (!(d2 < rs2)) return -1.f;
    if (d2 < ri2) return sqrtf(d2);  // clearly inside: the FP32 distance is kept
    const double r = min_image_dist(q, i, j, lx, ly, lz);  // within the margin of R
    return r < R ? (float)r : -1.f;
  }
};

// Neighbours j != i with r_ij < R, in increasing j; count clipped to kmax,
// *overflow set when a list was clipped. All pairs: the CTA's 8 blobs scan
// tiles of FP32 positions staged in shared memory. Used when the box holds
// fewer than 3 cells of side R along an axis.
__global__ void __launch_bounds__(kWarps * 32) k_gnn_neighbours(const double* __restrict__ q,
                                                                const float4* __restrict__ p32, int n, double lx,
                                                                double ly, double lz, double R, float margin,
                                                                int kmax, int* __restrict__ cnt,
                                                                int* __restrict__ nidx, float* __restrict__ nr,
                                                                int* __restrict__ overflow) {
  __shared__ float4 tile[kNbTile];
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * kWarps + (threadIdx.x >> 5);
  const bool active = i < n;
  const float4 pi = active ? p32[i] : make_float4(0.f, 0.f, 0.f, 0.f);
  const PairScreen ps(lx, ly, lz, R, margin);
  int c = 0;
  for (int t0 = 0; t0 < n; t0 += kNbTile) {
    const int tn = min(kNbTile, n - t0);
    __syncthreads();
    for (int t = threadIdx.x; t < tn; t += blockDim.x) tile[t] = p32[t0 + t];
    __syncthreads();
    if (!active) continue;
    for (int j0 = 0; j0 < tn; j0 += 32) {
      const int jl = j0 + lane;
      const int j = t0 + jl;
      const float r = jl < tn && j != i ? ps.dist(q, i, j, pi, tile[jl]) : -1.f;
      const bool in = r >= 0.f;
      const unsigned bal = __ballot_sync(0xffffffffu, in);
      const int slot = c + __popc(bal & ((1u << lane) - 1u));
      if (in && slot < kmax) {
        nidx[(size_t)i * kmax + slot] = j;
        nr[(size_t)i * kmax + slot] = r;
      }
      c += __popc(bal);
    }
  }
  if (active && lane == 0) {
    cnt[i] = c < kmax ? c : kmax;
    if (c > kmax) atomicOr(overflow, 1);
  }
}

// Cell list: the box split into ncx x ncy x ncz cells (3 to 32 per axis,
// each side at least R), every blob in the cell of its wrapped position; a
// pair closer than R then lies in the same or adjacent cells (periodically).
struct Cells {
  int nx, ny, nz;
  double lx, ly, lz;
  __device__ __forceinline__ int axis(double x, double L, int nc) const {
    double f = x / L;
    f -= floor(f);
    const int c = (int)(f * nc);
    return c < 0 ? 0 : (c < nc ? c : nc - 1);
  }
  __device__ __forceinline__ void of(const double* q, int j, int& cx, int& cy, int& cz) const {
    cx = axis(q[3 * j], lx, nx);
    cy = axis(q[3 * j + 1], ly, ny);
    cz = axis(q[3 * j + 2], lz, nz);
  }
};

__global__ void k_gnn_cell_count(const double* __restrict__ q, int n, Cells cl, int* __restrict__ cell_of,
                                 int* __restrict__ cell_cnt) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  int cx, cy, cz;
  cl.of(q, j, cx, cy, cz);
  const int c = (cz * cl.ny + cy) * cl.nx + cx;
  cell_of[j] = c;
  atomicAdd(&cell_cnt[c], 1);
}

// Exclusive scan of the cell counts (one CTA): start[c], start[ncell] = n;
// cursor[c] = start[c] for the fill.
__global__ void __launch_bounds__(1024) k_gnn_cell_scan(const int* __restrict__ cell_cnt, int ncell,
                                                        int* __restrict__ start, int* __restrict__ cursor) {
  __shared__ int part[1024];
  const int per = (ncell + 1023) / 1024;
  const int b = threadIdx.x * per, e = min(ncell, b + per);
  int sum = 0;
  for (int c = b; c < e; ++c) sum += cell_cnt[c];
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const int v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int run = part[threadIdx.x] - sum;
  for (int c = b; c < e; ++c) {
    start[c] = run;
    cursor[c] = run;
    run += cell_cnt[c];
  }
  if (threadIdx.x == 1023) start[ncell] = part[1023];
}

__global__ void k_gnn_cell_fill(int n, const int* __restrict__ cell_of, int* __restrict__ cursor,
                                int* __restrict__ cell_blobs) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) cell_blobs[atomicAdd(&cursor[cell_of[j]], 1)] = j;
}

// Neighbours from the cell list, one CTA per cell: the candidates of its 27
// surrounding cells (distinct, as every axis has at least 3) are staged in
// shared memory, up to kNbTile at a time, as (x, y, z, index), and its blobs
// screen them one warp each. A blob's neighbours are collected in scratch
// lists (tj, tr) in staging order, then placed in increasing j by their rank
// (the j are distinct).
__global__ void __launch_bounds__(kWarps * 32) k_gnn_neighbours_cells(
    const double* __restrict__ q, const float4* __restrict__ p32, Cells cl, double R, float margin,
    const int* __restrict__ start, const int* __restrict__ cell_blobs, int kmax, int* __restrict__ tj,
    float* __restrict__ tr, int* __restrict__ cnt, int* __restrict__ nidx, float* __restrict__ nr,
    int* __restrict__ overflow) {
  __shared__ float4 tile[kNbTile];
  __shared__ int nb_cell[27], pre[28];
  const int cell = blockIdx.x;
  const int cb = start[cell], nown = start[cell + 1] - cb;
  if (nown == 0) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x < 27) {
    const int cx = cell % cl.nx, cy = (cell / cl.nx) % cl.ny, cz = cell / (cl.nx * cl.ny);
    const int t = threadIdx.x;
    int x = cx + t % 3 - 1, y = cy + (t / 3) % 3 - 1, z = cz + t / 9 - 1;
    x = x < 0 ? cl.nx - 1 : (x == cl.nx ? 0 : x);
    y = y < 0 ? cl.ny - 1 : (y == cl.ny ? 0 : y);
    z = z < 0 ? cl.nz - 1 : (z == cl.nz ? 0 : z);
    nb_cell[t] = (z * cl.ny + y) * cl.nx + x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int t = 0; t < 27; ++t) {
      pre[t] = run;
      run += start[nb_cell[t] + 1] - start[nb_cell[t]];
    }
    pre[27] = run;
  }
  __syncthreads();
  const int T = pre[27];
  const PairScreen ps(cl.lx, cl.ly, cl.lz, R, margin);
  for (int g0 = 0; g0 < nown; g0 += kWarps) {
    const int i = g0 + w < nown ? cell_blobs[cb + g0 + w] : -1;
    const float4 pi = i >= 0 ? p32[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    int* li = tj + (size_t)(i >= 0 ? i : 0) * kmax;
    float* lr = tr + (size_t)(i >= 0 ? i : 0) * kmax;
    int c = 0;
    for (int t0 = 0; t0 < T; t0 += kNbTile) {
      const int tn = min(kNbTile, T - t0);
      if (g0 == 0 || T > kNbTile) {
        __syncthreads();
        for (int t = threadIdx.x; t < tn; t += blockDim.x) {
          const int u = t0 + t;
          int k = 0;
          while (pre[k + 1] <= u) ++k;
          const int j = cell_blobs[start[nb_cell[k]] + u - pre[k]];
          const float4 pj = p32[j];
          tile[t] = make_float4(pj.x, pj.y, pj.z, __int_as_float(j));
        }
        __syncthreads();
      }
      if (i < 0) continue;
      for (int j0 = 0; j0 < tn; j0 += 32) {
        const int jl = j0 + lane;
        const float4 pj = jl < tn ? tile[jl] : make_float4(0.f, 0.f, 0.f, __int_as_float(i));
        const int j = __float_as_int(pj.w);
        const float r = j != i ? ps.dist(q, i, j, pi, pj) : -1.f;
        const bool in = r >= 0.f;
        const unsigned bal = __ballot_sync(0xffffffffu, in);
        const int slot = c + __popc(bal & ((1u << lane) - 1u));
        if (in && slot < kmax) {
          li[slot] = j;
          lr[slot] = r;
        }
        c += __popc(bal);
      }
    }
    if (i < 0) continue;
    const int cc = c < kmax ? c : kmax;
    __syncwarp();
    for (int e = lane; e < cc; e += 32) {
      const int je = li[e];
      int rank = 0;
      for (int f = 0; f < cc; ++f) rank += li[f] < je;
      nidx[(size_t)i * kmax + rank] = je;
      nr[(size_t)i * kmax + rank] = lr[e];
    }
    if (lane == 0) {
      cnt[i] = cc;
      if (c > kmax) atomicOr(overflow, 1);
    }
  }
}

// x_i, a0_i = W0 x_i + c0, h0_i = relu(a0_i). The lanes take the edges in
// turn (all K bases of each), then the warp adds its lanes' partial sums.
__global__ void __launch_bounds__(kWarps * 32) k_gnn_layer0(const float* __restrict__ th, int n, float invR,
                                                            int kmax, const int* __restrict__ cnt,
                                                            const float* __restrict__ nr, float* __restrict__ x,
                                                            float* __restrict__ a0, float* __restrict__ h0) {
  __shared__ float sW0[H * (K + 1)];
  for (int t = threadIdx.x; t < H * K; t += blockDim.x) sW0[(t / K) * (K + 1) + t % K] = th[OFF_W0 + t];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (i >= n) return;
  float xk[K];
#pragma unroll
  for (int k = 0; k < K; ++k) xk[k] = 0.f;
  const int c = cnt[i];
  for (int e = lane; e < c; e += 32) {
    const float s = nr[(size_t)i * kmax + e] * invR;
#pragma unroll
    for (int k = 0; k < K; ++k) xk[k] += basis_k(s, k);
  }
#pragma unroll
  for (int k = 0; k < K; ++k)
    for (int o = 16; o > 0; o >>= 1) xk[k] += __shfl_xor_sync(0xffffffffu, xk[k], o);
  if (lane < K) {
    float v = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) v = lane == k ? xk[k] : v;
    x[(size_t)i * K + lane] = v;
  }
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int row = lane + 32 * half;
    float a = th[OFF_C0 + row];
#pragma unroll
    for (int kk = 0; kk < K; ++kk) a = fmaf(sW0[row * (K + 1) + kk], xk[kk], a);
    a0[(size_t)i * H + row] = a;
    h0[(size_t)i * H + row] = fmaxf(a, 0.f);
  }
}

// Loads W_l and V_l into shared memory with a padded row stride.
__device__ __forceinline__ void load_mats(const float* __restrict__ th, int l, float* sW, float* sV) {
  for (int t = threadIdx.x; t < H * H; t += blockDim.x) {
    const int r = t / H, c = t - r * H;
    sW[r * kPad + c] = th[offW(l) + t];
    sV[r * kPad + c] = th[offV(l) + t];
  }
}

// Layer l (FP32): m_i, a_i = W_l m_i + V_l hp_i + c_l, h_i = hp_i + relu(a_i).
__global__ void __launch_bounds__(kWarps * 32) k_gnn_mp(const float* __restrict__ th, int l, int n, float invR,
                                                        int kmax, const int* __restrict__ cnt,
                                                        const int* __restrict__ nidx, const float* __restrict__ nr,
                                                        const float* __restrict__ hp, float* __restrict__ m,
                                                        float* __restrict__ a, float* __restrict__ h) {
  __shared__ float sW[H * kPad], sV[H * kPad];
  load_mats(th, l, sW, sV);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (i >= n) return;
  const int k = lane & (K - 1);
  const float* E = th + offE(l);
  const float* eb = th + offEB(l);
  float m0 = 0.f, m1 = 0.f;
  const int c = cnt[i];
  for (int e = 0; e < c; ++e) {
    const int j = nidx[(size_t)i * kmax + e];
    const float s = nr[(size_t)i * kmax + e] * invR;
    const float bk = basis_k(s, k);
    const float fc = (1.f - s) * (1.f - s);
    float p0 = eb[lane], p1 = eb[lane + 32];
    for (int kk = 0; kk < K; ++kk) {
      const float b = __shfl_sync(0xffffffffu, bk, kk);
      p0 = fmaf(E[lane * K + kk], b, p0);
      p1 = fmaf(E[(lane + 32) * K + kk], b, p1);
    }
    m0 = fmaf(fc * fmaxf(p0, 0.f), hp[(size_t)j * H + lane], m0);
    m1 = fmaf(fc * fmaxf(p1, 0.f), hp[(size_t)j * H + lane + 32], m1);
  }
  const float hi0 = hp[(size_t)i * H + lane], hi1 = hp[(size_t)i * H + lane + 32];
  float s0 = th[offC(l) + lane], s1 = th[offC(l) + lane + 32];
  for (int kk = 0; kk < H; ++kk) {
    const float mk = __shfl_sync(0xffffffffu, kk < 32 ? m0 : m1, kk & 31);
    const float hk = __shfl_sync(0xffffffffu, kk < 32 ? hi0 : hi1, kk & 31);
    s0 = fmaf(sW[lane * kPad + kk], mk, fmaf(sV[lane * kPad + kk], hk, s0));
    s1 = fmaf(sW[(lane + 32) * kPad + kk], mk, fmaf(sV[(lane + 32) * kPad + kk], hk, s1));
  }
  m[(size_t)i * H + lane] = m0;
  m[(size_t)i * H + lane + 32] = m1;
  a[(size_t)i * H + lane] = s0;
  a[(size_t)i * H + lane + 32] = s1;
  h[(size_t)i * H + lane] = hi0 + fmaxf(s0, 0.f);
  h[(size_t)i * H + lane + 32] = hi1 + fmaxf(s1, 0.f);
}

// y_i = o . h_i + o0.
__global__ void __launch_bounds__(kWarps * 32) k_gnn_out(const float* __restrict__ th, int n,
                                                         const float* __restrict__ h, float* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (i >= n) return;
  float v = th[OFF_O + lane] * h[(size_t)i * H + lane] + th[OFF_O + lane + 32] * h[(size_t)i * H + lane + 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) y[i] = v + th[OFF_O0];
}

// Block reduction helper: sum over the block of one double per thread.
__device__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
  __syncthreads();
  if (threadIdx.x == 0) sh[0] = t;
  __syncthreads();
  const double r = sh[0];
  __syncthreads();
  return r;
}

// log v for v > 0 (FP64 in, FP64 out) with one FP32 logarithm: v = f 2^e,
// f in [0.5, 1), log v = log f + e log 2; absolute error about 1e-7, far below
// the spread of the log-multipliers the loss compares.
__device__ __forceinline__ double log_pos(double v) {
  int e;
  const double f = frexp(v, &e);
  return (double)logf((float)f) + (double)e * 0.69314718055994530942;
}

// Loss of one configuration and dL/dy (one CTA): r = (y - <y>) - (t - <t>),
// L = <r^2>, dy = 2 r / n. out[0] = L.
__global__ void __launch_bounds__(1024) k_gnn_loss(const float* __restrict__ y, const double* __restrict__ lam,
                                                   int n, float* __restrict__ dy, double* __restrict__ out) {
  __shared__ double sh[32];
  double sy = 0.0, st = 0.0;
#pragma unroll 4
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    sy += (double)y[i];
    st += log_pos(lam[i]);
  }
  const double inv_n = 1.0 / n;
  const double my = block_sum(sy, sh) * inv_n;
  const double mt = block_sum(st, sh) * inv_n;
  double l2 = 0.0;
#pragma unroll 4
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double r = ((double)y[i] - my) - (log_pos(lam[i]) - mt);
    dy[i] = (float)(2.0 * inv_n * r);
    l2 += r * r;
  }
  const double L = block_sum(l2, sh) * inv_n;
  if (threadIdx.x == 0) out[0] = L;
}

// lambda0_i = total * exp(y_i - max y) / sum_k exp(y_k - max y) (one CTA;
// the exponentials of the FP32 outputs in FP32, their sum in FP64).
__global__ void __launch_bounds__(1024) k_gnn_softmax(const float* __restrict__ y, int n, double total,
                                                      double* __restrict__ lam0) {
  __shared__ double sh[32];
  __shared__ float smax[32];
  float mx = -INFINITY;
#pragma unroll 4
  for (int i = threadIdx.x; i < n; i += blockDim.x) mx = fmaxf(mx, y[i]);
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = smax[0];
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) t = fmaxf(t, smax[k]);
    smax[0] = t;
  }
  __syncthreads();
  const float ymax = smax[0];
  double s = 0.0;
#pragma unroll 4
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += (double)expf(y[i] - ymax);
  const double scale = total / block_sum(s, sh);
#pragma unroll 4
  for (int i = threadIdx.x; i < n; i += blockDim.x) lam0[i] = scale * (double)expf(y[i] - ymax);
}

// Backward through layer l's node update: dh = dh_in (or dy o at the last
// layer), da = dh [a > 0], dm = W_l^T da, dhv = dh + V_l^T da.
__global__ void __launch_bounds__(kWarps * 32) k_gnn_back_node(const float* __restrict__ th, int l, int n,
                                                               const float* __restrict__ dh_in,
                                                               const float* __restrict__ dy,
                                                               const float* __restrict__ a,
                                                               float* __restrict__ da, float* __restrict__ dm,
                                                               float* __restrict__ dhv) {
  __shared__ float sW[H * kPad], sV[H * kPad];
  load_mats(th, l, sW, sV);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (i >= n) return;
  float dh0, dh1;
  if (dh_in) {
    dh0 = dh_in[(size_t)i * H + lane];
    dh1 = dh_in[(size_t)i * H + lane + 32];
  } else {
    const float g = dy[i];
    dh0 = g * th[OFF_O + lane];
    dh1 = g * th[OFF_O + lane + 32];
  }
  const float d0 = a[(size_t)i * H + lane] > 0.f ? dh0 : 0.f;
  const float d1 = a[(size_t)i * H + lane + 32] > 0.f ? dh1 : 0.f;
  float dm0 = 0.f, dm1 = 0.f, dv0 = dh0, dv1 = dh1;
  for (int r = 0; r < H; ++r) {
    const float dr = __shfl_sync(0xffffffffu, r < 32 ? d0 : d1, r & 31);
    dm0 = fmaf(sW[r * kPad + lane], dr, dm0);
    dm1 = fmaf(sW[r * kPad + lane + 32], dr, dm1);
    dv0 = fmaf(sV[r * kPad + lane], dr, dv0);
    dv1 = fmaf(sV[r * kPad + lane + 32], dr, dv1);
  }
  da[(size_t)i * H + lane] = d0;
  da[(size_t)i * H + lane + 32] = d1;
  dm[(size_t)i * H + lane] = dm0;
  dm[(size_t)i * H + lane + 32] = dm1;
  dhv[(size_t)i * H + lane] = dv0;
  dhv[(size_t)i * H + lane + 32] = dv1;
}

// Backward through layer l's messages at blob i, over its own neighbour list
// (symmetric): dh_out_i = dhv_i + sum_j f_c F_ij * dm_j (the messages of the j
// that used hp_i), and the filter gradient dP_ij = f_c dm_i * hp_j * [P_ij > 0]
// gives this CTA's partial sums of dE_l (H x K) and de_l (H). With a0 (the
// first layer) dh_out is the embedding's da0 = dh_0 [a0 > 0].
__global__ void __launch_bounds__(kWarps * 32) k_gnn_back_edges(const float* __restrict__ th, int l, int n,
                                                                float invR, int kmax, const int* __restrict__ cnt,
                                                                const int* __restrict__ nidx,
                                                                const float* __restrict__ nr,
                                                                const float* __restrict__ hp,
                                                                const float* __restrict__ dm,
                                                                const float* __restrict__ dhv,
                                                                const float* __restrict__ a0,
                                                                float* __restrict__ dh_out,
                                                                float* __restrict__ part) {
  __shared__ float sE[kWarps][H * (K + 1)];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i = blockIdx.x * kWarps + w;
  const float* E = th + offE(l);
  const float* eb = th + offEB(l);
  float gE0[K], gE1[K];
#pragma unroll
  for (int kk = 0; kk < K; ++kk) gE0[kk] = gE1[kk] = 0.f;
  float ge0 = 0.f, ge1 = 0.f;
  if (i < n) {
    const int k = lane & (K - 1);
    const float dmi0 = dm[(size_t)i * H + lane], dmi1 = dm[(size_t)i * H + lane + 32];
    float acc0 = dhv[(size_t)i * H + lane], acc1 = dhv[(size_t)i * H + lane + 32];
    const int c = cnt[i];
    for (int e = 0; e < c; ++e) {
      const int j = nidx[(size_t)i * kmax + e];
      const float s = nr[(size_t)i * kmax + e] * invR;
      const float bk = basis_k(s, k);
      const float fc = (1.f - s) * (1.f - s);
      float p0 = eb[lane], p1 = eb[lane + 32];
      float b[K];
#pragma unroll
      for (int kk = 0; kk < K; ++kk) {
        b[kk] = __shfl_sync(0xffffffffu, bk, kk);
        p0 = fmaf(E[lane * K + kk], b[kk], p0);
        p1 = fmaf(E[(lane + 32) * K + kk], b[kk], p1);
      }
      const float F0 = fmaxf(p0, 0.f), F1 = fmaxf(p1, 0.f);
      acc0 = fmaf(fc * F0, dm[(size_t)j * H + lane], acc0);
      acc1 = fmaf(fc * F1, dm[(size_t)j * H + lane + 32], acc1);
      const float q0 = p0 > 0.f ? fc * dmi0 * hp[(size_t)j * H + lane] : 0.f;
      const float q1 = p1 > 0.f ? fc * dmi1 * hp[(size_t)j * H + lane + 32] : 0.f;
      ge0 += q0;
      ge1 += q1;
#pragma unroll
      for (int kk = 0; kk < K; ++kk) {
        gE0[kk] = fmaf(q0, b[kk], gE0[kk]);
        gE1[kk] = fmaf(q1, b[kk], gE1[kk]);
      }
    }
    if (a0) {
      acc0 = a0[(size_t)i * H + lane] > 0.f ? acc0 : 0.f;
      acc1 = a0[(size_t)i * H + lane + 32] > 0.f ? acc1 : 0.f;
    }
    dh_out[(size_t)i * H + lane] = acc0;
    dh_out[(size_t)i * H + lane + 32] = acc1;
  }
  // this CTA's partial sums, warps added in a fixed order
#pragma unroll
  for (int kk = 0; kk < K; ++kk) {
    sE[w][lane * (K + 1) + kk] = gE0[kk];
    sE[w][(lane + 32) * (K + 1) + kk] = gE1[kk];
  }
  sE[w][lane * (K + 1) + K] = ge0;
  sE[w][(lane + 32) * (K + 1) + K] = ge1;
  __syncthreads();
  for (int t = threadIdx.x; t < H * (K + 1); t += blockDim.x) {
    float v = 0.f;
    for (int ww = 0; ww < kWarps; ++ww) v += sE[ww][t];
    part[(size_t)blockIdx.x * H * (K + 1) + t] = v;
  }
}

// Activations and gradients the parameter gradients read.
struct GradArgs {
  int n, nblk;
  const float* x;     // N x K
  const float* da0;   // N x H
  const float* h;     // (L + 1) x N x H: h_0 .. h_L
  const float* m;     // L x N x H
  const float* da;    // L x N x H
  const float* dy;    // N
  const float* part;  // L x nblk x H x (K + 1)
};

// Parameter gradients that are sums over blobs, one thread per parameter,
// blobs added in increasing order: dW0 = sum da0 x^T, dc0 = sum da0, per layer
// dW_l = sum da_l m_l^T, dV_l = sum da_l h_{l-1}^T, dc_l = sum da_l and dE_l /
// de_l from the per-CTA partials, do = sum dy h_L, do0 = sum dy.
__global__ void k_gnn_param_grads(GradArgs ga, float* __restrict__ grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NPARAM) return;
  const int n = ga.n;
  const size_t NH = (size_t)n * H;
  float s = 0.f;
  if (p < OFF_C0) {
    const int r = p / K, c = p - r * K;
    for (int i = 0; i < n; ++i) s = fmaf(ga.da0[(size_t)i * H + r], ga.x[(size_t)i * K + c], s);
  } else if (p < OFF_C0 + H) {
    const int r = p - OFF_C0;
    for (int i = 0; i < n; ++i) s += ga.da0[(size_t)i * H + r];
  } else if (p < OFF_O) {
    const int l = (p - lbase(1)) / LSZ + 1;
    const int q = p - lbase(l);
    const float* da = ga.da + (size_t)(l - 1) * NH;
    if (q < H * K + H) {
      // E (row r, col c) and e (row r) from the CTA partials
      const int r = q < H * K ? q / K : q - H * K;
      const int c = q < H * K ? q - (q / K) * K : K;
      const float* part = ga.part + (size_t)(l - 1) * ga.nblk * H * (K + 1);
      for (int b = 0; b < ga.nblk; ++b) s += part[(size_t)b * H * (K + 1) + r * (K + 1) + c];
    } else if (q < H * K + H + H * H) {
      const int t = q - (H * K + H), r = t / H, c = t - r * H;
      const float* m = ga.m + (size_t)(l - 1) * NH;
      for (int i = 0; i < n; ++i) s = fmaf(da[(size_t)i * H + r], m[(size_t)i * H + c], s);
    } else if (q < H * K + H + 2 * H * H) {
      const int t = q - (H * K + H + H * H), r = t / H, c = t - r * H;
      const float* hp = ga.h + (size_t)(l - 1) * NH;
      for (int i = 0; i < n; ++i) s = fmaf(da[(size_t)i * H + r], hp[(size_t)i * H + c], s);
    } else {
      const int r = q - (H * K + H + 2 * H * H);
      for (int i = 0; i < n; ++i) s += da[(size_t)i * H + r];
    }
  } else if (p < OFF_O0) {
    const int r = p - OFF_O;
    const float* hL = ga.h + (size_t)L * NH;
    for (int i = 0; i < n; ++i) s = fmaf(ga.dy[i], hL[(size_t)i * H + r], s);
  } else {
    for (int i = 0; i < n; ++i) s += ga.dy[i];
  }
  grad[p] = s;
}

// ---------------------------------------------------------------- inference on tensor cores
// bfloat16 copies of the layers' weights: per layer E_l (H x K), then
// [W_l V_l] (H x 2H, row n = W_l row n followed by V_l row n).
__global__ void k_gnn_weights_bf16(const float* __restrict__ th, __nv_bfloat16* __restrict__ wb) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= L * BLSZ) return;
  const int l = t / BLSZ + 1, q = t - (l - 1) * BLSZ;
  float v;
  if (q < H * K) {
    v = th[offE(l) + q];
  } else {
    const int r = (q - H * K) / (2 * H), c = (q - H * K) - r * 2 * H;
    v = c < H ? th[offW(l) + r * H + c] : th[offV(l) + r * H + c - H];
  }
  wb[t] = __float2bfloat16_rn(v);
}

__device__ __forceinline__ unsigned bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x (low half) = lo
  return *reinterpret_cast<const unsigned*>(&v);
}

// D += A B for one m16n8k16 tile: A 16 x 16 bfloat16 (row), B 16 x 8 (col),
// FP32 accumulators.
__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Layer l's messages on tensor cores: one warp per blob i; its edges in tiles
// of 16 (rows) against the 64 filter outputs (8 column tiles of 8), K = 16
// bases deep. Fragment ownership (m16n8k16): lane = 4 g + t holds A at rows
// g, g + 8 and columns 2t, 2t + 1, 2t + 8, 2t + 9; B at rows 2t, 2t + 1,
// 2t + 8, 2t + 9 and column g; D at rows g, g + 8 and columns 2t, 2t + 1.
// Each lane then sums relu(P + e) f_c hp_j over its two edge rows, and the
// eight lanes of a column pair add theirs. The gathers are latency-bound:
// each tile issues all of its neighbour rows' loads before any arithmetic,
// and the next tile's indices are fetched before the current one's products.
__global__ void __launch_bounds__(kWarps * 32, 3) k_gnn_msg_tc(const float* __restrict__ th,
                                                               const __nv_bfloat16* __restrict__ wb, int l, int n,
                                                               float invR, int kmax, const int* __restrict__ cnt,
                                                               const int* __restrict__ nidx,
                                                               const float* __restrict__ nr,
                                                               const float* __restrict__ hp, float* __restrict__ m) {
  static_assert(kWarps == 8, "one warp per column tile fills the staged fragments");
  __shared__ unsigned sB[8][2][32];  // per column tile, the two B registers of each lane
  __shared__ float2 sBias[8][4];     // per column tile, e_l at columns 2t, 2t + 1
  {
    const __nv_bfloat16* E = wb + (size_t)(l - 1) * BLSZ;
    const int nt = threadIdx.x >> 5, ln = threadIdx.x & 31;
    const int col = 8 * nt + (ln >> 2), t2 = 2 * (ln & 3);  // B column = filter output
    sB[nt][0][ln] = *reinterpret_cast<const unsigned*>(E + col * K + t2);
    sB[nt][1][ln] = *reinterpret_cast<const unsigned*>(E + col * K + t2 + 8);
    if (threadIdx.x < 32) {
      const float* eb = th + offEB(l);
      sBias[threadIdx.x >> 2][threadIdx.x & 3] =
          make_float2(eb[8 * (threadIdx.x >> 2) + 2 * (threadIdx.x & 3)],
                      eb[8 * (threadIdx.x >> 2) + 2 * (threadIdx.x & 3) + 1]);
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (i >= n) return;
  const int g = lane >> 2, t = lane & 3;
  float acc[8][2];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = 0.f;
  const int c = cnt[i];
  const int* ni = nidx + (size_t)i * kmax;
  const float* ri = nr + (size_t)i * kmax;
  // edge rows g and g + 8 of a tile; s = 1 (no edge): every basis and the
  // cutoff vanish, and row 0 of hp stands in for the neighbour
  int j0 = g < c ? ni[g] : 0, j1 = g + 8 < c ? ni[g + 8] : 0;
  float s0 = g < c ? ri[g] * invR : 1.f, s1 = g + 8 < c ? ri[g + 8] * invR : 1.f;
  for (int e0 = 0; e0 < c; e0 += 16) {
    float2 h0[8], h1[8];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      h0[nt] = *reinterpret_cast<const float2*>(hp + (size_t)j0 * H + 8 * nt + 2 * t);
      h1[nt] = *reinterpret_cast<const float2*>(hp + (size_t)j1 * H + 8 * nt + 2 * t);
    }
    const float cs0 = s0, cs1 = s1;
    const int r0 = e0 + 16 + g, r1 = e0 + 24 + g;
    j0 = r0 < c ? ni[r0] : 0;
    j1 = r1 < c ? ni[r1] : 0;
    s0 = r0 < c ? ri[r0] * invR : 1.f;
    s1 = r1 < c ? ri[r1] * invR : 1.f;
    unsigned a[4];
    a[0] = bf16x2(basis_k(cs0, 2 * t), basis_k(cs0, 2 * t + 1));
    a[1] = bf16x2(basis_k(cs1, 2 * t), basis_k(cs1, 2 * t + 1));
    a[2] = bf16x2(basis_k(cs0, 2 * t + 8), basis_k(cs0, 2 * t + 9));
    a[3] = bf16x2(basis_k(cs1, 2 * t + 8), basis_k(cs1, 2 * t + 9));
    const float fc0 = (1.f - cs0) * (1.f - cs0), fc1 = (1.f - cs1) * (1.f - cs1);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      float d[4] = {0.f, 0.f, 0.f, 0.f};
      mma_bf16(d, a, sB[nt][0][lane], sB[nt][1][lane]);
      const float2 bias = sBias[nt][t];
      acc[nt][0] += fc0 * fmaxf(d[0] + bias.x, 0.f) * h0[nt].x + fc1 * fmaxf(d[2] + bias.x, 0.f) * h1[nt].x;
      acc[nt][1] += fc0 * fmaxf(d[1] + bias.y, 0.f) * h0[nt].y + fc1 * fmaxf(d[3] + bias.y, 0.f) * h1[nt].y;
    }
  }
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) {
      acc[nt][0] += __shfl_xor_sync(0xffffffffu, acc[nt][0], o);
      acc[nt][1] += __shfl_xor_sync(0xffffffffu, acc[nt][1], o);
    }
    if (g == 0)
      *reinterpret_cast<float2*>(m + (size_t)i * H + 8 * nt + 2 * t) = make_float2(acc[nt][0], acc[nt][1]);
  }
}

// Layer l's node update on tensor cores: one warp per 16 blobs, a = [m hp]
// (16 x 128) times [W_l V_l]^T (128 x 64) in 8 k-steps and 8 column tiles,
// the weights staged in shared memory; h = hp + relu(a + c_l).
// The staged rows are padded to 136 elements (68 words) so that the eight
// rows one B fragment load touches fall in distinct banks.
constexpr int kNodeWarps = 4;
constexpr int kWVStride = 2 * H + 8;
__global__ void __launch_bounds__(kNodeWarps * 32) k_gnn_node_tc(const float* __restrict__ th,
                                                                 const __nv_bfloat16* __restrict__ wb, int l, int n,
                                                                 const float* __restrict__ m,
                                                                 const float* __restrict__ hp,
                                                                 float* __restrict__ h) {
  __shared__ __align__(16) __nv_bfloat16 sWV[H * kWVStride];
  const __nv_bfloat16* WV = wb + (size_t)(l - 1) * BLSZ + H * K;
  for (int q = threadIdx.x; q < H * 2 * H / 8; q += blockDim.x) {
    const int r = q / (2 * H / 8), c8 = q - r * (2 * H / 8);
    *reinterpret_cast<uint4*>(sWV + r * kWVStride + 8 * c8) = reinterpret_cast<const uint4*>(WV)[q];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int base = (blockIdx.x * kNodeWarps + (threadIdx.x >> 5)) * 16;
  if (base >= n) return;
  const int r0 = base + g, r1 = base + g + 8;
  const bool v0 = r0 < n, v1 = r1 < n;
  float d[8][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) d[nt][0] = d[nt][1] = d[nt][2] = d[nt][3] = 0.f;
  auto src = [&](int row, int kc) -> float2 {  // [m hp] at (row, kc), kc even
    const float* p = kc < H ? m + (size_t)row * H + kc : hp + (size_t)row * H + kc - H;
    return *reinterpret_cast<const float2*>(p);
  };
#pragma unroll
  for (int ks = 0; ks < 8; ++ks) {
    const int kc = 16 * ks + 2 * t;
    const float2 z = make_float2(0.f, 0.f);
    const float2 x00 = v0 ? src(r0, kc) : z, x10 = v1 ? src(r1, kc) : z;
    const float2 x01 = v0 ? src(r0, kc + 8) : z, x11 = v1 ? src(r1, kc + 8) : z;
    const unsigned a[4] = {bf16x2(x00.x, x00.y), bf16x2(x10.x, x10.y), bf16x2(x01.x, x01.y),
                           bf16x2(x11.x, x11.y)};
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int col = 8 * nt + g;
      const unsigned b0 = *reinterpret_cast<const unsigned*>(sWV + col * kWVStride + kc);
      const unsigned b1 = *reinterpret_cast<const unsigned*>(sWV + col * kWVStride + kc + 8);
      mma_bf16(d[nt], a, b0, b1);
    }
  }
  const float* cb = th + offC(l);
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int col = 8 * nt + 2 * t;
    const float2 c = make_float2(cb[col], cb[col + 1]);
    if (v0) {
      const float2 p = *reinterpret_cast<const float2*>(hp + (size_t)r0 * H + col);
      *reinterpret_cast<float2*>(h + (size_t)r0 * H + col) =
          make_float2(p.x + fmaxf(d[nt][0] + c.x, 0.f), p.y + fmaxf(d[nt][1] + c.y, 0.f));
    }
    if (v1) {
      const float2 p = *reinterpret_cast<const float2*>(hp + (size_t)r1 * H + col);
      *reinterpret_cast<float2*>(h + (size_t)r1 * H + col) =
          make_float2(p.x + fmaxf(d[nt][2] + c.x, 0.f), p.y + fmaxf(d[nt][3] + c.y, 0.f));
    }
  }
}

// Adam with bias correction; c1 = 1 - beta1^t, c2 = 1 - beta2^t.
__global__ void k_gnn_adam(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m1,
                           float* __restrict__ m2, int np, float lr, float b1, float b2, float c1, float c2,
                           float eps) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const float gp = g[p];
  const float a = b1 * m1[p] + (1.f - b1) * gp;
  const float v = b2 * m2[p] + (1.f - b2) * gp * gp;
  m1[p] = a;
  m2[p] = v;
  th[p] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
}

}  // namespace
}  // namespace ibrd

using namespace ibrd;

struct ibrd_gnn_s {
  int dev = 0;
  cudaStream_t s = nullptr;
  double cutoff = 16.0;
  int kmax = 64;
  float* th = nullptr;  // parameters
  float* g = nullptr;   // gradient
  float* m1 = nullptr;  // Adam moments
  float* m2 = nullptr;
  long long step = 0;
  // per-configuration workspaces (grow only)
  int cap = 0;
  int *cnt = nullptr, *nidx = nullptr, *oflow = nullptr;
  float4* p32 = nullptr;
  // forward: x (N x K), a0 (N x H), h_0 .. h_L ((L + 1) x N x H), m_l and
  // a_l (L x N x H each), y (N); backward: dy, da0, da_l, dm, dhv, dh, and
  // the per-CTA filter-gradient partials (L x CTAs x H x (K + 1))
  float *nr = nullptr, *x = nullptr, *a0 = nullptr, *h = nullptr, *m = nullptr, *a = nullptr, *y = nullptr;
  float *dy = nullptr, *da0 = nullptr, *da = nullptr, *dm = nullptr, *dhv = nullptr, *dh = nullptr;
  float* part = nullptr;
  __nv_bfloat16* wb = nullptr;  // bfloat16 layer weights for inference
  // cell list (grow only): per blob its cell, the blobs sorted by cell, the
  // scratch candidate lists; per cell its count, start and fill cursor
  int *cell_of = nullptr, *cell_blobs = nullptr, *tj = nullptr;
  float* tr = nullptr;
  int cell_cap = 0;
  int *cell_cnt = nullptr, *cell_start = nullptr, *cell_cursor = nullptr;
  double* loss = nullptr;  // device scalar
  double* host = nullptr;  // pinned
  std::string err;
};

namespace ibrd {
namespace {

struct GnnArgError {
  ibrd_status code;
  std::string msg;
};

template <typename T>
void galloc(T** p, size_t n) {
  cudaFree(*p);
  *p = nullptr;
  IBRD_CUDA(cudaMalloc(p, sizeof(T) * (n ? n : 1)));
}

template <typename F>
ibrd_status gnn_guarded(ibrd_gnn m, const char* name, F&& f) {
  if (!m) return IBRD_ERR_ARG;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != m->dev) cudaSetDevice(m->dev);
  ibrd_status st = IBRD_OK;
  try {
    m->err.clear();
    st = f();
  } catch (const GnnArgError& e) {
    m->err = std::string(name) + ": " + e.msg;
    st = e.code;
  } catch (const CudaError& e) {
    st = (e.code == cudaErrorMemoryAllocation) ? IBRD_ERR_OOM : IBRD_ERR_CUDA;
    cudaGetLastError();
    m->err = std::string(name) + ": " + e.what + ": " + cudaGetErrorString(e.code);
  } catch (const std::bad_alloc&) {
    m->err = std::string(name) + ": host allocation failed";
    st = IBRD_ERR_OOM;
  }
  if (prev >= 0 && prev != m->dev) cudaSetDevice(prev);
  return st;
}

void ensure_cap(ibrd_gnn m, int n) {
  if (n <= m->cap) return;
  const size_t N = (size_t)n, nb = (N + kWarps - 1) / kWarps;
  galloc(&m->cnt, N);
  galloc(&m->p32, N);
  galloc(&m->nidx, N * m->kmax);
  galloc(&m->nr, N * m->kmax);
  galloc(&m->x, N * K);
  galloc(&m->a0, N * H);
  galloc(&m->h, (L + 1) * N * H);
  galloc(&m->m, L * N * H);
  galloc(&m->a, L * N * H);
  galloc(&m->y, N);
  galloc(&m->dy, N);
  galloc(&m->da0, N * H);
  galloc(&m->da, L * N * H);
  galloc(&m->dm, N * H);
  galloc(&m->dhv, N * H);
  galloc(&m->dh, N * H);
  galloc(&m->part, L * nb * H * (K + 1));
  galloc(&m->cell_of, N);
  galloc(&m->cell_blobs, N);
  galloc(&m->tj, N * m->kmax);
  galloc(&m->tr, N * m->kmax);
  m->cap = n;
}

void check_config(ibrd_gnn m, const double* q, int n, double lx, double ly, double lz) {
  if (n < 1 || !q) throw GnnArgError{IBRD_ERR_ARG, "need n >= 1 blob positions"};
  if (!(lx > 0.0 && ly > 0.0 && lz > 0.0) || !std::isfinite(lx) || !std::isfinite(ly) || !std::isfinite(lz))
    throw GnnArgError{IBRD_ERR_ARG, "bad box"};
  if (2.0 * m->cutoff > std::min(lx, std::min(ly, lz)))
    throw GnnArgError{IBRD_ERR_ARG, "cutoff above half the shortest box side"};
}

// Cells per axis for the cell list: each side at least R (with room for
// rounding), at most 32; 0 when fewer than 3 fit.
int cells_per_axis(double L, double R) {
  const double c = std::floor(L / (R * (1.0 + 1e-6)));
  return c < 3.0 ? 0 : (int)std::min(c, 32.0);
}

// Neighbour lists of one configuration: from a cell list when every axis
// holds at least 3 cells of side R, else all pairs.
void neighbour_lists(ibrd_gnn m, const double* q, int n, double lx, double ly, double lz) {
  ensure_cap(m, n);
  const int nb = (n + kWarps - 1) / kWarps;
  IBRD_CUDA(cudaMemsetAsync(m->oflow, 0, sizeof(int), m->s));
  prof_begin(P_SETUP, m->s);
  // FP32 screen margin: the wrapped FP32 coordinates carry half an ulp of the
  // box side each (6e-8 L), a minimum-image difference a few ulps, the
  // distance under 1e-6 L with its own rounding; the margin is ten times that
  const float margin = (float)(1e-5 * std::max(lx, std::max(ly, lz)) + 1e-6 * m->cutoff);
  k_gnn_pos32<<<(n + 255) / 256, 256, 0, m->s>>>(q, n, lx, ly, lz, m->p32);
  prof_end(P_SETUP, m->s, "gnn_pos32");
  Cells cl{cells_per_axis(lx, m->cutoff), cells_per_axis(ly, m->cutoff), cells_per_axis(lz, m->cutoff), lx, ly,
           lz};
  if (cl.nx && cl.ny && cl.nz) {
    const int ncell = cl.nx * cl.ny * cl.nz;
    if (ncell > m->cell_cap) {
      galloc(&m->cell_cnt, ncell);
      galloc(&m->cell_start, ncell + 1);
      galloc(&m->cell_cursor, ncell);
      m->cell_cap = ncell;
    }
    IBRD_CUDA(cudaMemsetAsync(m->cell_cnt, 0, sizeof(int) * ncell, m->s));
    prof_begin(P_SETUP, m->s);
    k_gnn_cell_count<<<(n + 255) / 256, 256, 0, m->s>>>(q, n, cl, m->cell_of, m->cell_cnt);
    prof_end(P_SETUP, m->s, "gnn_cell_count");
    prof_begin(P_SETUP, m->s);
    k_gnn_cell_scan<<<1, 1024, 0, m->s>>>(m->cell_cnt, ncell, m->cell_start, m->cell_cursor);
    prof_end(P_SETUP, m->s, "gnn_cell_scan");
    prof_begin(P_SETUP, m->s);
    k_gnn_cell_fill<<<(n + 255) / 256, 256, 0, m->s>>>(n, m->cell_of, m->cell_cursor, m->cell_blobs);
    prof_end(P_SETUP, m->s, "gnn_cell_fill");
    prof_begin(P_SETUP, m->s);
    k_gnn_neighbours_cells<<<ncell, kWarps * 32, 0, m->s>>>(q, m->p32, cl, m->cutoff, margin, m->cell_start,
                                                            m->cell_blobs, m->kmax, m->tj, m->tr, m->cnt,
                                                            m->nidx, m->nr, m->oflow);
    prof_end(P_SETUP, m->s, "gnn_neighbours_cells");
  } else {
    prof_begin(P_SETUP, m->s);
    k_gnn_neighbours<<<nb, kWarps * 32, 0, m->s>>>(q, m->p32, n, lx, ly, lz, m->cutoff, margin, m->kmax, m->cnt,
                                                   m->nidx, m->nr, m->oflow);
    prof_end(P_SETUP, m->s, "gnn_neighbours");
  }
}

float* hbuf(ibrd_gnn m, int n, int l) { return m->h + (size_t)l * n * H; }
float* lbuf(float* base, int n, int l) { return base + (size_t)(l - 1) * n * H; }  // l = 1 .. L

// Neighbour lists and the FP32 forward pass (y in m->y); with bf16 the
// layers' dense products run on the tensor cores instead.
void forward(ibrd_gnn m, const double* q, int n, double lx, double ly, double lz, bool bf16 = false) {
  neighbour_lists(m, q, n, lx, ly, lz);
  const int nb = (n + kWarps - 1) / kWarps;
  const float invR = (float)(1.0 / m->cutoff);
  prof_begin(P_SETUP, m->s);
  k_gnn_layer0<<<nb, kWarps * 32, 0, m->s>>>(m->th, n, invR, m->kmax, m->cnt, m->nr, m->x, m->a0, hbuf(m, n, 0));
  prof_end(P_SETUP, m->s, "gnn_layer0");
  if (bf16) {
    prof_begin(P_SETUP, m->s);
    k_gnn_weights_bf16<<<(L * BLSZ + 255) / 256, 256, 0, m->s>>>(m->th, m->wb);
    prof_end(P_SETUP, m->s, "gnn_weights_bf16");
  }
  for (int l = 1; l <= L; ++l) {
    if (bf16) {
      prof_begin(P_SETUP, m->s);
      k_gnn_msg_tc<<<nb, kWarps * 32, 0, m->s>>>(m->th, m->wb, l, n, invR, m->kmax, m->cnt, m->nidx, m->nr,
                                                 hbuf(m, n, l - 1), lbuf(m->m, n, l));
      prof_end(P_SETUP, m->s, "gnn_msg_tc");
      prof_begin(P_SETUP, m->s);
      const int nt = (n + 16 * kNodeWarps - 1) / (16 * kNodeWarps);
      k_gnn_node_tc<<<nt, kNodeWarps * 32, 0, m->s>>>(m->th, m->wb, l, n, lbuf(m->m, n, l), hbuf(m, n, l - 1),
                                                      hbuf(m, n, l));
      prof_end(P_SETUP, m->s, "gnn_node_tc");
    } else {
      prof_begin(P_SETUP, m->s);
      k_gnn_mp<<<nb, kWarps * 32, 0, m->s>>>(m->th, l, n, invR, m->kmax, m->cnt, m->nidx, m->nr, hbuf(m, n, l - 1),
                                             lbuf(m->m, n, l), lbuf(m->a, n, l), hbuf(m, n, l));
      prof_end(P_SETUP, m->s, "gnn_mp");
    }
  }
  prof_begin(P_SETUP, m->s);
  k_gnn_out<<<nb, kWarps * 32, 0, m->s>>>(m->th, n, hbuf(m, n, L), m->y);
  prof_end(P_SETUP, m->s, "gnn_out");
}

void check_overflow(ibrd_gnn m) {
  int of = 0;
  IBRD_CUDA(cudaMemcpyAsync(&of, m->oflow, sizeof(int), cudaMemcpyDeviceToHost, m->s));
  IBRD_CUDA(cudaStreamSynchronize(m->s));
  if (of) throw GnnArgError{IBRD_ERR_ARG, "a blob has more neighbours than max_neighbours"};
}

// Loss and gradient of one configuration (after the FP32 forward); gradient
// in m->g. Layers run in reverse: dh enters layer l (dy o at the last), its
// node update gives da_l, dm and dhv, its messages the dh entering layer l - 1
// (at the first, da0) and the filter partials.
void backward(ibrd_gnn m, int n, const double* lam) {
  const int nb = (n + kWarps - 1) / kWarps;
  const float invR = (float)(1.0 / m->cutoff);
  prof_begin(P_SETUP, m->s);
  k_gnn_loss<<<1, 1024, 0, m->s>>>(m->y, lam, n, m->dy, m->loss);
  prof_end(P_SETUP, m->s, "gnn_loss");
  for (int l = L; l >= 1; --l) {
    prof_begin(P_SETUP, m->s);
    k_gnn_back_node<<<nb, kWarps * 32, 0, m->s>>>(m->th, l, n, l == L ? nullptr : m->dh, m->dy, lbuf(m->a, n, l),
                                                  lbuf(m->da, n, l), m->dm, m->dhv);
    prof_end(P_SETUP, m->s, "gnn_back_node");
    prof_begin(P_SETUP, m->s);
    k_gnn_back_edges<<<nb, kWarps * 32, 0, m->s>>>(
        m->th, l, n, invR, m->kmax, m->cnt, m->nidx, m->nr, hbuf(m, n, l - 1), m->dm, m->dhv,
        l == 1 ? m->a0 : nullptr, l == 1 ? m->da0 : m->dh, m->part + (size_t)(l - 1) * nb * H * (K + 1));
    prof_end(P_SETUP, m->s, "gnn_back_edges");
  }
  GradArgs ga{n, nb, m->x, m->da0, m->h, m->m, m->da, m->dy, m->part};
  prof_begin(P_SETUP, m->s);
  k_gnn_param_grads<<<(NPARAM + 255) / 256, 256, 0, m->s>>>(ga, m->g);
  prof_end(P_SETUP, m->s, "gnn_param_grads");
}

void adam(ibrd_gnn m, const float* grad, double lr) {
  m->step++;
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = (float)(1.0 - std::pow(b1, (double)m->step));
  const float c2 = (float)(1.0 - std::pow(b2, (double)m->step));
  prof_begin(P_SETUP, m->s);
  k_gnn_adam<<<(NPARAM + 255) / 256, 256, 0, m->s>>>(m->th, grad, m->m1, m->m2, NPARAM, (float)lr, (float)b1,
                                                     (float)b2, c1, c2, 1e-8f);
  prof_end(P_SETUP, m->s, "gnn_adam");
}

void check_lam(ibrd_gnn m, const double* lam, int n) {
  if (!lam) throw GnnArgError{IBRD_ERR_ARG, "null multipliers"};
  (void)m;
  (void)n;
}

}  // namespace
}  // namespace ibrd

extern "C" {

int ibrd_gnn_num_params(void) { return NPARAM; }

ibrd_status ibrd_gnn_create(ibrd_gnn* out, double cutoff, int max_neighbours, void* stream) {
  if (!out) return IBRD_ERR_ARG;
  *out = nullptr;
  if (!(cutoff > 0.0) || !std::isfinite(cutoff) || max_neighbours < 1 || max_neighbours > 1024)
    return IBRD_ERR_ARG;
  ibrd_gnn m = new (std::nothrow) ibrd_gnn_s();
  if (!m) return IBRD_ERR_OOM;
  cudaGetDevice(&m->dev);
  m->s = (cudaStream_t)stream;
  m->cutoff = cutoff;
  m->kmax = max_neighbours;
  const ibrd_status st = gnn_guarded(m, "ibrd_gnn_create", [&]() {
    galloc(&m->th, NPARAM);
    galloc(&m->g, NPARAM);
    galloc(&m->m1, NPARAM);
    galloc(&m->m2, NPARAM);
    galloc(&m->oflow, 1);
    galloc(&m->loss, 1);
    galloc(&m->wb, L * BLSZ);
    IBRD_CUDA(cudaMallocHost(&m->host, sizeof(double) * 8));
    IBRD_CUDA(cudaMemsetAsync(m->th, 0, sizeof(float) * NPARAM, m->s));
    IBRD_CUDA(cudaMemsetAsync(m->m1, 0, sizeof(float) * NPARAM, m->s));
    IBRD_CUDA(cudaMemsetAsync(m->m2, 0, sizeof(float) * NPARAM, m->s));
    IBRD_CUDA(cudaStreamSynchronize(m->s));
    return IBRD_OK;
  });
  if (st != IBRD_OK) {
    ibrd_gnn_destroy(m);
    return st;
  }
  *out = m;
  return IBRD_OK;
}

void ibrd_gnn_destroy(ibrd_gnn m) {
  if (!m) return;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != m->dev) cudaSetDevice(m->dev);
  for (void* p : {(void*)m->th, (void*)m->g, (void*)m->m1, (void*)m->m2, (void*)m->cnt, (void*)m->nidx,
                  (void*)m->oflow, (void*)m->nr, (void*)m->x, (void*)m->a0, (void*)m->h, (void*)m->m,
                  (void*)m->a, (void*)m->y, (void*)m->dy, (void*)m->da0, (void*)m->da, (void*)m->dm,
                  (void*)m->dhv, (void*)m->dh, (void*)m->part, (void*)m->loss, (void*)m->p32, (void*)m->wb,
                  (void*)m->cell_of, (void*)m->cell_blobs, (void*)m->tj, (void*)m->tr, (void*)m->cell_cnt,
                  (void*)m->cell_start, (void*)m->cell_cursor})
    if (p) cudaFree(p);
  if (m->host) cudaFreeHost(m->host);
  if (prev >= 0 && prev != m->dev) cudaSetDevice(prev);
  delete m;
}

const char* ibrd_gnn_last_error(ibrd_gnn m) { return m ? m->err.c_str() : "null handle"; }

ibrd_status ibrd_gnn_set_params(ibrd_gnn m, const float* theta, int reset_optimizer) {
  return gnn_guarded(m, "ibrd_gnn_set_params", [&]() {
    if (!theta) throw GnnArgError{IBRD_ERR_ARG, "null parameters"};
    IBRD_CUDA(cudaMemcpyAsync(m->th, theta, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, m->s));
    if (reset_optimizer) {
      IBRD_CUDA(cudaMemsetAsync(m->m1, 0, sizeof(float) * NPARAM, m->s));
      IBRD_CUDA(cudaMemsetAsync(m->m2, 0, sizeof(float) * NPARAM, m->s));
      m->step = 0;
    }
    IBRD_CUDA(cudaStreamSynchronize(m->s));
    return IBRD_OK;
  });
}

ibrd_status ibrd_gnn_init_params(ibrd_gnn m, unsigned long long seed) {
  return gnn_guarded(m, "ibrd_gnn_init_params", [&]() {
    // splitmix64 stream -> uniform in [-1, 1) (53-bit mantissa)
    unsigned long long st = seed;
    auto next = [&st]() {
      unsigned long long z = (st += 0x9E3779B97F4A7C15ull);
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      return (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
    };
    std::vector<float> th(NPARAM, 0.f);
    auto fill = [&](int off, int count, double lim) {
      for (int k = 0; k < count; ++k) th[off + k] = (float)(lim * next());
    };
    fill(OFF_W0, H * K, 1.0 / std::sqrt((double)K));
    for (int l = 1; l <= L; ++l) {
      fill(offE(l), H * K, 1.0 / std::sqrt((double)K));
      fill(offW(l), H * H, 1.0 / std::sqrt((double)H));
      fill(offV(l), H * H, 1.0 / std::sqrt((double)H));
    }
    fill(OFF_O, H, 1.0 / std::sqrt((double)H));
    IBRD_CUDA(cudaMemcpyAsync(m->th, th.data(), sizeof(float) * NPARAM, cudaMemcpyHostToDevice, m->s));
    IBRD_CUDA(cudaMemsetAsync(m->m1, 0, sizeof(float) * NPARAM, m->s));
    IBRD_CUDA(cudaMemsetAsync(m->m2, 0, sizeof(float) * NPARAM, m->s));
    m->step = 0;
    IBRD_CUDA(cudaStreamSynchronize(m->s));
    return IBRD_OK;
  });
}

ibrd_status ibrd_gnn_get_params(ibrd_gnn m, float* theta) {
  return gnn_guarded(m, "ibrd_gnn_get_params", [&]() {
    if (!theta) throw GnnArgError{IBRD_ERR_ARG, "null parameters"};
    IBRD_CUDA(cudaMemcpyAsync(theta, m->th, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, m->s));
    IBRD_CUDA(cudaStreamSynchronize(m->s));
    return IBRD_OK;
  });
}

ibrd_status ibrd_gnn_neighbours(ibrd_gnn m, const double* q, int n, double lx, double ly, double lz, int* count,
                                int* index, float* dist) {
  return gnn_guarded(m, "ibrd_gnn_neighbours", [&]() {
    check_config(m, q, n, lx, ly, lz);
    if (!count || !index || !dist) throw GnnArgError{IBRD_ERR_ARG, "null output"};
    neighbour_lists(m, q, n, lx, ly, lz);
    check_overflow(m);
    IBRD_CUDA(cudaMemcpyAsync(count, m->cnt, sizeof(int) * n, cudaMemcpyDeviceToDevice, m->s));
    IBRD_CUDA(cudaMemcpyAsync(index, m->nidx, sizeof(int) * (size_t)n * m->kmax, cudaMemcpyDeviceToDevice, m->s));
    IBRD_CUDA(cudaMemcpyAsync(dist, m->nr, sizeof(float) * (size_t)n * m->kmax, cudaMemcpyDeviceToDevice, m->s));
    return IBRD_OK;
  });
}

ibrd_status ibrd_gnn_forward(ibrd_gnn m, const double* q, int n, double lx, double ly, double lz, float* y) {
  return gnn_guarded(m, "ibrd_gnn_forward", [&]() {
    check_config(m, q, n, lx, ly, lz);
    if (!y) throw GnnArgError{IBRD_ERR_ARG, "null output"};
    forward(m, q, n, lx, ly, lz);
    check_overflow(m);
    IBRD_CUDA(cudaMemcpyAsync(y, m->y, sizeof(float) * n, cudaMemcpyDeviceToDevice, m->s));
    return IBRD_OK;
  });
}

ibrd_status ibrd_gnn_predict(ibrd_gnn m, const double* q, int n, double lx, double ly, double lz, double total,
                             double* lambda0) {
  return gnn_guarded(m, "ibrd_gnn_predict", [&]() {
    check_config(m, q, n, lx, ly, lz);
    if (!lambda0 || !std::isfinite(total)) throw GnnArgError{IBRD_ERR_ARG, "bad output or total"};
    forward(m, q, n, lx, ly, lz, /*bf16=*/true);
    prof_begin(P_SETUP, m->s);
    k_gnn_softmax<<<1, 1024, 0, m->s>>>(m->y, n, total, lambda0);
    prof_end(P_SETUP, m->s, "gnn_softmax");
    check_overflow(m);
    return IBRD_OK;
  });
}

ibrd_status ibrd_gnn_loss_grad(ibrd_gnn m, const double* q, int n, double lx, double ly, double lz,
                               const double* lam, double* loss, float* grad) {
  return gnn_guarded(m, "ibrd_gnn_loss_grad", [&]() {
    check_config(m, q, n, lx, ly, lz);
    check_lam(m, lam, n);
    forward(m, q, n, lx, ly, lz);
    backward(m, n, lam);
    if (grad) IBRD_CUDA(cudaMemcpyAsync(grad, m->g, sizeof(float) * NPARAM, cudaMemcpyDeviceToDevice, m->s));
    IBRD_CUDA(cudaMemcpyAsync(m->host, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->s));
    check_overflow(m);
    if (loss) *loss = m->host[0];
    return IBRD_OK;
  });
}

ibrd_status ibrd_gnn_adam_step(ibrd_gnn m, const float* grad, double lr) {
  return gnn_guarded(m, "ibrd_gnn_adam_step", [&]() {
    if (!grad || !(lr > 0.0)) throw GnnArgError{IBRD_ERR_ARG, "bad gradient or rate"};
    adam(m, grad, lr);
    return IBRD_OK;
  });
}

ibrd_status ibrd_gnn_train(ibrd_gnn m, int count, const double* const* q, const int* n, const double* boxes,
                           const double* const* lam, int epochs, double lr, double* epoch_loss) {
  return gnn_guarded(m, "ibrd_gnn_train", [&]() {
    if (count < 1 || !q || !n || !boxes || !lam || epochs < 1 || !(lr > 0.0))
      throw GnnArgError{IBRD_ERR_ARG, "bad training arguments"};
    for (int c = 0; c < count; ++c) {
      check_config(m, q[c], n[c], boxes[3 * c], boxes[3 * c + 1], boxes[3 * c + 2]);
      check_lam(m, lam[c], n[c]);
    }
    std::vector<double> losses((size_t)count);
    for (int ep = 0; ep < epochs; ++ep) {
      double sum = 0.0;
      for (int c = 0; c < count; ++c) {
        forward(m, q[c], n[c], boxes[3 * c], boxes[3 * c + 1], boxes[3 * c + 2]);
        backward(m, n[c], lam[c]);
        adam(m, m->g, lr);
        IBRD_CUDA(cudaMemcpyAsync(m->host, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->s));
        check_overflow(m);  // synchronizes: the loss is on the host now
        sum += m->host[0];
      }
      if (epoch_loss) epoch_loss[ep] = sum / count;
    }
    return IBRD_OK;
  });
}

}  // extern "C"
