// Learned multiplier predictor: a small graph network over each blob's
// neighbours that predicts the relative sink strengths lambda_i / <lambda> of
// the diffusion-limited saddle point (Eq. saddle_point), used as the initial
// guess of the multipliers. The paper names a good treatment of the Schur
// complement for many blobs as open (Sec. III.E, Sec. V); this network is
// trained on (configuration, lambda) pairs produced by the saddle solver.
//
// Definition (width H = 64, K = 16 radial bases, cutoff R, s = r / R,
// f_c = (1 - s)^2, b_k = f_c exp(-((s - k/(K-1)) / sigma)^2), sigma = 1.5/(K-1)):
//   x_i  = sum_j b(r_ij)
//   h1_i = relu(W1 x_i + c1)
//   m_i  = sum_j f_c(r_ij) relu(E b(r_ij) + e) * h1_j
//   h2_i = h1_i + relu(W2 m_i + V2 h1_i + c2)
//   y_i  = o . h2_i + o0,   lambda0_i = T softmax(y)_i
// Loss: <((y - <y>) - (t - <t>))^2>, t = log lambda. Adam updates.
//
// Kernels: one warp per blob (lane l owns hidden rows l and l + 32); the
// neighbour lists are symmetric, so the backward pass gathers every edge
// contribution at its own node (no atomics). Parameters, activations and
// gradients are FP32; positions and the predicted multipliers FP64. The dense
// layers are 64-wide products over a few thousand blobs (a few MFLOP): they
// run on the FP32 pipes, well inside one launch's latency.
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
constexpr float kSigmaInv = (K - 1) / 1.5f;
// flat parameter layout (as in the FP64 reference)
constexpr int OFF_W1 = 0;
constexpr int OFF_C1 = OFF_W1 + H * K;
constexpr int OFF_E = OFF_C1 + H;
constexpr int OFF_EB = OFF_E + H * K;
constexpr int OFF_W2 = OFF_EB + H;
constexpr int OFF_V2 = OFF_W2 + H * H;
constexpr int OFF_C2 = OFF_V2 + H * H;
constexpr int OFF_O = OFF_C2 + H;
constexpr int OFF_O0 = OFF_O + H;
constexpr int NPARAM = OFF_O0 + 1;
constexpr int kWarps = 8;  // blobs per CTA
constexpr int kPad = H + 1; // shared-memory row stride of the 64 x 64 matrices

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

// FP32 copies of the positions (x, y, z, 0) for the neighbour screen.
__global__ void k_gnn_pos32(const double* __restrict__ q, int n, float4* __restrict__ p) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) p[j] = make_float4((float)q[3 * j], (float)q[3 * j + 1], (float)q[3 * j + 2], 0.f);
}

constexpr int kNbTile = 1024;  // positions staged in shared memory per pass

// Neighbours j != i with r_ij < R, in increasing j; count clipped to kmax,
// *overflow set when a list was clipped. FP64 is slow on this GPU, so every
// pair is measured in FP32 and only pairs within a margin of R (the margin far
// above the FP32 rounding of the coordinates) take the exact FP64 test: the
// neighbour sets are the FP64 definition's; a stored distance is the FP32 one
// (within a few ulps of the box side) away from the boundary. The CTA's 8 blobs
// scan tiles of FP32 positions staged in shared memory.
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
  const float flx = (float)lx, fly = (float)ly, flz = (float)lz;
  const float ilx = 1.f / flx, ily = 1.f / fly, ilz = 1.f / flz;
  const float rs = (float)R + margin, rs2 = rs * rs;
  const float ri = (float)R - margin, ri2 = ri > 0.f ? ri * ri : 0.f;
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
      double r = 0.0;
      bool in = false;
      if (jl < tn && j != i) {
        const float4 pj = tile[jl];
        float dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
        dx -= flx * rintf(dx * ilx);
        dy -= fly * rintf(dy * ily);
        dz -= flz * rintf(dz * ilz);
        const float d2 = dx * dx + dy * dy + dz * dz;
        if (d2 < rs2) {
          if (d2 < ri2) {
            // clearly inside: the FP32 distance is kept
            r = (double)sqrtf(d2);
            in = true;
          } else {
            // within the margin of R: the exact FP64 test decides
            r = min_image_dist(q, i, j, lx, ly, lz);
            in = r < R;
          }
        }
      }
      const unsigned bal = __ballot_sync(0xffffffffu, in);
      const int slot = c + __popc(bal & ((1u << lane) - 1u));
      if (in && slot < kmax) {
        nidx[(size_t)i * kmax + slot] = j;
        nr[(size_t)i * kmax + slot] = (float)r;
      }
      c += __popc(bal);
    }
  }
  if (active && lane == 0) {
    cnt[i] = c < kmax ? c : kmax;
    if (c > kmax) atomicOr(overflow, 1);
  }
}

// x_i, a1_i = W1 x_i + c1, h1_i = relu(a1_i).
__global__ void __launch_bounds__(kWarps * 32) k_gnn_layer1(const float* __restrict__ th, int n, float invR,
                                                            int kmax, const int* __restrict__ cnt,
                                                            const float* __restrict__ nr, float* __restrict__ x,
                                                            float* __restrict__ a1, float* __restrict__ h1) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (i >= n) return;
  const int k = lane & (K - 1);
  float xk = 0.f;
  const int c = cnt[i];
  for (int e = 0; e < c; ++e) xk += basis_k(nr[(size_t)i * kmax + e] * invR, k);
  if (lane < K) x[(size_t)i * K + lane] = xk;
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int row = lane + 32 * half;
    float a = th[OFF_C1 + row];
    for (int kk = 0; kk < K; ++kk) a = fmaf(th[OFF_W1 + row * K + kk], __shfl_sync(0xffffffffu, xk, kk), a);
    a1[(size_t)i * H + row] = a;
    h1[(size_t)i * H + row] = fmaxf(a, 0.f);
  }
}

// Loads W2 and V2 into shared memory with a padded row stride.
__device__ __forceinline__ void load_mats(const float* __restrict__ th, float* sW2, float* sV2) {
  for (int t = threadIdx.x; t < H * H; t += blockDim.x) {
    const int r = t / H, c = t - r * H;
    sW2[r * kPad + c] = th[OFF_W2 + t];
    sV2[r * kPad + c] = th[OFF_V2 + t];
  }
}

// m_i, a2_i = W2 m_i + V2 h1_i + c2, y_i = o . (h1_i + relu(a2_i)) + o0.
__global__ void __launch_bounds__(kWarps * 32) k_gnn_layer2(const float* __restrict__ th, int n, float invR,
                                                            int kmax, const int* __restrict__ cnt,
                                                            const int* __restrict__ nidx,
                                                            const float* __restrict__ nr,
                                                            const float* __restrict__ h1, float* __restrict__ m,
                                                            float* __restrict__ a2, float* __restrict__ y) {
  __shared__ float sW2[H * kPad], sV2[H * kPad];
  load_mats(th, sW2, sV2);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (i >= n) return;
  const int k = lane & (K - 1);
  float m0 = 0.f, m1 = 0.f;
  const int c = cnt[i];
  for (int e = 0; e < c; ++e) {
    const int j = nidx[(size_t)i * kmax + e];
    const float s = nr[(size_t)i * kmax + e] * invR;
    const float bk = basis_k(s, k);
    const float fc = (1.f - s) * (1.f - s);
    float p0 = th[OFF_EB + lane], p1 = th[OFF_EB + lane + 32];
    for (int kk = 0; kk < K; ++kk) {
      const float b = __shfl_sync(0xffffffffu, bk, kk);
      p0 = fmaf(th[OFF_E + lane * K + kk], b, p0);
      p1 = fmaf(th[OFF_E + (lane + 32) * K + kk], b, p1);
    }
    m0 = fmaf(fc * fmaxf(p0, 0.f), h1[(size_t)j * H + lane], m0);
    m1 = fmaf(fc * fmaxf(p1, 0.f), h1[(size_t)j * H + lane + 32], m1);
  }
  const float hi0 = h1[(size_t)i * H + lane], hi1 = h1[(size_t)i * H + lane + 32];
  float s0 = th[OFF_C2 + lane], s1 = th[OFF_C2 + lane + 32];
  for (int kk = 0; kk < H; ++kk) {
    const float mk = __shfl_sync(0xffffffffu, kk < 32 ? m0 : m1, kk & 31);
    const float hk = __shfl_sync(0xffffffffu, kk < 32 ? hi0 : hi1, kk & 31);
    s0 = fmaf(sW2[lane * kPad + kk], mk, fmaf(sV2[lane * kPad + kk], hk, s0));
    s1 = fmaf(sW2[(lane + 32) * kPad + kk], mk, fmaf(sV2[(lane + 32) * kPad + kk], hk, s1));
  }
  m[(size_t)i * H + lane] = m0;
  m[(size_t)i * H + lane + 32] = m1;
  a2[(size_t)i * H + lane] = s0;
  a2[(size_t)i * H + lane + 32] = s1;
  float v = th[OFF_O + lane] * (hi0 + fmaxf(s0, 0.f)) + th[OFF_O + lane + 32] * (hi1 + fmaxf(s1, 0.f));
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

// Loss of one configuration and dL/dy (one CTA): r = (y - <y>) - (t - <t>),
// L = <r^2>, dy = 2 r / n. out[0] = L.
__global__ void __launch_bounds__(1024) k_gnn_loss(const float* __restrict__ y, const double* __restrict__ lam,
                                                   int n, float* __restrict__ dy, double* __restrict__ out) {
  __shared__ double sh[32];
  double sy = 0.0, st = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    sy += (double)y[i];
    st += log(lam[i]);
  }
  const double my = block_sum(sy, sh) / n;
  const double mt = block_sum(st, sh) / n;
  double l2 = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double r = ((double)y[i] - my) - (log(lam[i]) - mt);
    dy[i] = (float)(2.0 * r / n);
    l2 += r * r;
  }
  const double L = block_sum(l2, sh) / n;
  if (threadIdx.x == 0) out[0] = L;
}

// lambda0_i = total * exp(y_i - max y) / sum_k exp(y_k - max y) (one CTA).
__global__ void __launch_bounds__(1024) k_gnn_softmax(const float* __restrict__ y, int n, double total,
                                                      double* __restrict__ lam0) {
  __shared__ double sh[32];
  __shared__ float smax[32];
  float mx = -INFINITY;
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
  const double ymax = (double)smax[0];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += exp((double)y[i] - ymax);
  const double S = block_sum(s, sh);
  for (int i = threadIdx.x; i < n; i += blockDim.x) lam0[i] = total * exp((double)y[i] - ymax) / S;
}

// Backward through the node layers: da2 = dy o * [a2 > 0], dm = W2^T da2,
// dh1 (direct) = dy o + V2^T da2.
__global__ void __launch_bounds__(kWarps * 32) k_gnn_back_node(const float* __restrict__ th, int n,
                                                               const float* __restrict__ dy,
                                                               const float* __restrict__ a2,
                                                               float* __restrict__ da2, float* __restrict__ dm,
                                                               float* __restrict__ dh1) {
  __shared__ float sW2[H * kPad], sV2[H * kPad];
  load_mats(th, sW2, sV2);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (i >= n) return;
  const float g = dy[i];
  const float dh0 = g * th[OFF_O + lane], dh1v = g * th[OFF_O + lane + 32];
  const float d0 = a2[(size_t)i * H + lane] > 0.f ? dh0 : 0.f;
  const float d1 = a2[(size_t)i * H + lane + 32] > 0.f ? dh1v : 0.f;
  float dm0 = 0.f, dm1 = 0.f, dv0 = dh0, dv1 = dh1v;
  for (int r = 0; r < H; ++r) {
    const float dr = __shfl_sync(0xffffffffu, r < 32 ? d0 : d1, r & 31);
    dm0 = fmaf(sW2[r * kPad + lane], dr, dm0);
    dm1 = fmaf(sW2[r * kPad + lane + 32], dr, dm1);
    dv0 = fmaf(sV2[r * kPad + lane], dr, dv0);
    dv1 = fmaf(sV2[r * kPad + lane + 32], dr, dv1);
  }
  da2[(size_t)i * H + lane] = d0;
  da2[(size_t)i * H + lane + 32] = d1;
  dm[(size_t)i * H + lane] = dm0;
  dm[(size_t)i * H + lane + 32] = dm1;
  dh1[(size_t)i * H + lane] = dv0;
  dh1[(size_t)i * H + lane + 32] = dv1;
}

// Backward through the message layer at blob i, over its own neighbour list
// (symmetric): dh1_i += sum_j f_c F_ij * dm_j (the messages of the j that used
// h1_i), and the filter gradient dP_ij = f_c dm_i * h1_j * [P_ij > 0] gives
// this CTA's partial sums of dE (H x K) and de (H). Then da1_i = dh1_i [a1 > 0].
__global__ void __launch_bounds__(kWarps * 32) k_gnn_back_edges(const float* __restrict__ th, int n, float invR,
                                                                int kmax, const int* __restrict__ cnt,
                                                                const int* __restrict__ nidx,
                                                                const float* __restrict__ nr,
                                                                const float* __restrict__ h1,
                                                                const float* __restrict__ a1,
                                                                const float* __restrict__ dm,
                                                                const float* __restrict__ dh1,
                                                                float* __restrict__ da1,
                                                                float* __restrict__ part) {
  __shared__ float sE[kWarps][H * (K + 1)];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i = blockIdx.x * kWarps + w;
  float gE0[K], gE1[K];
#pragma unroll
  for (int kk = 0; kk < K; ++kk) gE0[kk] = gE1[kk] = 0.f;
  float ge0 = 0.f, ge1 = 0.f;
  if (i < n) {
    const int k = lane & (K - 1);
    const float dmi0 = dm[(size_t)i * H + lane], dmi1 = dm[(size_t)i * H + lane + 32];
    float acc0 = dh1[(size_t)i * H + lane], acc1 = dh1[(size_t)i * H + lane + 32];
    const int c = cnt[i];
    for (int e = 0; e < c; ++e) {
      const int j = nidx[(size_t)i * kmax + e];
      const float s = nr[(size_t)i * kmax + e] * invR;
      const float bk = basis_k(s, k);
      const float fc = (1.f - s) * (1.f - s);
      float p0 = th[OFF_EB + lane], p1 = th[OFF_EB + lane + 32];
      float b[K];
#pragma unroll
      for (int kk = 0; kk < K; ++kk) {
        b[kk] = __shfl_sync(0xffffffffu, bk, kk);
        p0 = fmaf(th[OFF_E + lane * K + kk], b[kk], p0);
        p1 = fmaf(th[OFF_E + (lane + 32) * K + kk], b[kk], p1);
      }
      const float F0 = fmaxf(p0, 0.f), F1 = fmaxf(p1, 0.f);
      acc0 = fmaf(fc * F0, dm[(size_t)j * H + lane], acc0);
      acc1 = fmaf(fc * F1, dm[(size_t)j * H + lane + 32], acc1);
      const float q0 = p0 > 0.f ? fc * dmi0 * h1[(size_t)j * H + lane] : 0.f;
      const float q1 = p1 > 0.f ? fc * dmi1 * h1[(size_t)j * H + lane + 32] : 0.f;
      ge0 += q0;
      ge1 += q1;
#pragma unroll
      for (int kk = 0; kk < K; ++kk) {
        gE0[kk] = fmaf(q0, b[kk], gE0[kk]);
        gE1[kk] = fmaf(q1, b[kk], gE1[kk]);
      }
    }
    da1[(size_t)i * H + lane] = a1[(size_t)i * H + lane] > 0.f ? acc0 : 0.f;
    da1[(size_t)i * H + lane + 32] = a1[(size_t)i * H + lane + 32] > 0.f ? acc1 : 0.f;
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

// Parameter gradients that are sums over blobs, one thread per parameter,
// blobs added in increasing order: dW1 = sum da1 x^T, dc1 = sum da1,
// dW2 = sum da2 m^T, dV2 = sum da2 h1^T, dc2 = sum da2, do = sum dy h2,
// do0 = sum dy, and dE / de from the per-CTA partials.
__global__ void k_gnn_param_grads(int n, int nblk, const float* __restrict__ x, const float* __restrict__ h1,
                                  const float* __restrict__ m, const float* __restrict__ a2,
                                  const float* __restrict__ dy, const float* __restrict__ da1,
                                  const float* __restrict__ da2, const float* __restrict__ part,
                                  float* __restrict__ grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NPARAM) return;
  float s = 0.f;
  if (p < OFF_C1) {
    const int r = p / K, c = p - r * K;
    for (int i = 0; i < n; ++i) s = fmaf(da1[(size_t)i * H + r], x[(size_t)i * K + c], s);
  } else if (p < OFF_E) {
    const int r = p - OFF_C1;
    for (int i = 0; i < n; ++i) s += da1[(size_t)i * H + r];
  } else if (p < OFF_W2) {
    // E (row r, col c) and e (row r) from the CTA partials
    const int q = p - OFF_E;
    const int r = q < H * K ? q / K : q - H * K;
    const int c = q < H * K ? q - (q / K) * K : K;
    for (int b = 0; b < nblk; ++b) s += part[(size_t)b * H * (K + 1) + r * (K + 1) + c];
  } else if (p < OFF_V2) {
    const int q = p - OFF_W2, r = q / H, c = q - r * H;
    for (int i = 0; i < n; ++i) s = fmaf(da2[(size_t)i * H + r], m[(size_t)i * H + c], s);
  } else if (p < OFF_C2) {
    const int q = p - OFF_V2, r = q / H, c = q - r * H;
    for (int i = 0; i < n; ++i) s = fmaf(da2[(size_t)i * H + r], h1[(size_t)i * H + c], s);
  } else if (p < OFF_O) {
    const int r = p - OFF_C2;
    for (int i = 0; i < n; ++i) s += da2[(size_t)i * H + r];
  } else if (p < OFF_O0) {
    const int r = p - OFF_O;
    for (int i = 0; i < n; ++i)
      s = fmaf(dy[i], h1[(size_t)i * H + r] + fmaxf(a2[(size_t)i * H + r], 0.f), s);
  } else {
    for (int i = 0; i < n; ++i) s += dy[i];
  }
  grad[p] = s;
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
  float *nr = nullptr, *x = nullptr, *a1 = nullptr, *h1 = nullptr, *m = nullptr, *a2 = nullptr, *y = nullptr;
  float *dy = nullptr, *da1 = nullptr, *da2 = nullptr, *dm = nullptr, *dh1 = nullptr, *part = nullptr;
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
  galloc(&m->a1, N * H);
  galloc(&m->h1, N * H);
  galloc(&m->m, N * H);
  galloc(&m->a2, N * H);
  galloc(&m->y, N);
  galloc(&m->dy, N);
  galloc(&m->da1, N * H);
  galloc(&m->da2, N * H);
  galloc(&m->dm, N * H);
  galloc(&m->dh1, N * H);
  galloc(&m->part, nb * H * (K + 1));
  m->cap = n;
}

void check_config(ibrd_gnn m, const double* q, int n, double lx, double ly, double lz) {
  if (n < 1 || !q) throw GnnArgError{IBRD_ERR_ARG, "need n >= 1 blob positions"};
  if (!(lx > 0.0 && ly > 0.0 && lz > 0.0) || !std::isfinite(lx) || !std::isfinite(ly) || !std::isfinite(lz))
    throw GnnArgError{IBRD_ERR_ARG, "bad box"};
  if (2.0 * m->cutoff > std::min(lx, std::min(ly, lz)))
    throw GnnArgError{IBRD_ERR_ARG, "cutoff above half the shortest box side"};
}

// Neighbour lists and the forward pass for one configuration.
void forward(ibrd_gnn m, const double* q, int n, double lx, double ly, double lz) {
  ensure_cap(m, n);
  const int nb = (n + kWarps - 1) / kWarps;
  const float invR = (float)(1.0 / m->cutoff);
  IBRD_CUDA(cudaMemsetAsync(m->oflow, 0, sizeof(int), m->s));
  prof_begin(P_SETUP, m->s);
  // FP32 screen margin: well above the FP32 error of a minimum-image distance
  // (a few ulps of the box side)
  const float margin = (float)(1e-3 * m->cutoff + 1e-5 * std::max(lx, std::max(ly, lz)));
  k_gnn_pos32<<<(n + 255) / 256, 256, 0, m->s>>>(q, n, m->p32);
  prof_end(P_SETUP, m->s, "gnn_pos32");
  prof_begin(P_SETUP, m->s);
  k_gnn_neighbours<<<nb, kWarps * 32, 0, m->s>>>(q, m->p32, n, lx, ly, lz, m->cutoff, margin, m->kmax, m->cnt,
                                                 m->nidx, m->nr, m->oflow);
  prof_end(P_SETUP, m->s, "gnn_neighbours");
  prof_begin(P_SETUP, m->s);
  k_gnn_layer1<<<nb, kWarps * 32, 0, m->s>>>(m->th, n, invR, m->kmax, m->cnt, m->nr, m->x, m->a1, m->h1);
  prof_end(P_SETUP, m->s, "gnn_layer1");
  prof_begin(P_SETUP, m->s);
  k_gnn_layer2<<<nb, kWarps * 32, 0, m->s>>>(m->th, n, invR, m->kmax, m->cnt, m->nidx, m->nr, m->h1, m->m, m->a2,
                                             m->y);
  prof_end(P_SETUP, m->s, "gnn_layer2");
}

void check_overflow(ibrd_gnn m) {
  int of = 0;
  IBRD_CUDA(cudaMemcpyAsync(&of, m->oflow, sizeof(int), cudaMemcpyDeviceToHost, m->s));
  IBRD_CUDA(cudaStreamSynchronize(m->s));
  if (of) throw GnnArgError{IBRD_ERR_ARG, "a blob has more neighbours than max_neighbours"};
}

// Loss and gradient of one configuration (after forward); gradient in m->g.
void backward(ibrd_gnn m, int n, const double* lam) {
  const int nb = (n + kWarps - 1) / kWarps;
  const float invR = (float)(1.0 / m->cutoff);
  prof_begin(P_SETUP, m->s);
  k_gnn_loss<<<1, 1024, 0, m->s>>>(m->y, lam, n, m->dy, m->loss);
  prof_end(P_SETUP, m->s, "gnn_loss");
  prof_begin(P_SETUP, m->s);
  k_gnn_back_node<<<nb, kWarps * 32, 0, m->s>>>(m->th, n, m->dy, m->a2, m->da2, m->dm, m->dh1);
  prof_end(P_SETUP, m->s, "gnn_back_node");
  prof_begin(P_SETUP, m->s);
  k_gnn_back_edges<<<nb, kWarps * 32, 0, m->s>>>(m->th, n, invR, m->kmax, m->cnt, m->nidx, m->nr, m->h1, m->a1,
                                                 m->dm, m->dh1, m->da1, m->part);
  prof_end(P_SETUP, m->s, "gnn_back_edges");
  prof_begin(P_SETUP, m->s);
  k_gnn_param_grads<<<(NPARAM + 255) / 256, 256, 0, m->s>>>(n, nb, m->x, m->h1, m->m, m->a2, m->dy, m->da1,
                                                            m->da2, m->part, m->g);
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
                  (void*)m->oflow, (void*)m->nr, (void*)m->x, (void*)m->a1, (void*)m->h1, (void*)m->m,
                  (void*)m->a2, (void*)m->y, (void*)m->dy, (void*)m->da1, (void*)m->da2, (void*)m->dm,
                  (void*)m->dh1, (void*)m->part, (void*)m->loss, (void*)m->p32})
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
    fill(OFF_W1, H * K, 1.0 / std::sqrt((double)K));
    fill(OFF_E, H * K, 1.0 / std::sqrt((double)K));
    fill(OFF_W2, H * H, 1.0 / std::sqrt((double)H));
    fill(OFF_V2, H * H, 1.0 / std::sqrt((double)H));
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
    forward(m, q, n, lx, ly, lz);
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
    forward(m, q, n, lx, ly, lz);
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
