// Block preconditioner of the Schur complement M = J A^-1 S (Sec. III.E,
// Appendix A) for the inner GMRES of the approximate Schur preconditioner.
//
// The paper leaves a good treatment of M for many blobs open (Sec. III.E,
// Sec. V). M_ij for i != j is the periodic Green's function of chi L between
// the two blobs, smoothed by the kernels; beyond the kernels' support that is
//   G(r) = 1 / (4 pi chi r) + C_box / chi + r^2 / (6 chi V)
// (the expansion of the zero-mean periodic Green's function of -Laplace; for a
// cube of side L, C_box = -2.837297 / (4 pi L), the constant of Sec. IV.A's
// Eq. a_phi). With the diagonal M_ii = gamma (measured by the library), row i
// of P is row i of the inverse of the model restricted to blob i and its
// neighbours within the cutoff: a sparse approximate inverse that needs no
// solve. GMRES on P M converges in fewer iterations than on M.
//
// Set-up (per blob configuration): positions to FP32 inside the box; one warp
// per blob collects the neighbours within the cutoff (all pairs; the nearest
// kBlockMax - 1 of the first 128 found when more), then one warp per blob
// builds the model block and solves it for the row by Gaussian elimination
// with partial pivoting (FP32: the block's condition number is about ten, the
// preconditioner approximate). Application: one warp per blob, lane = slot.
#include <cmath>

#include "internal.h"
#include "schur_block.h"

namespace ibrd {
namespace {

constexpr int kWarps = 8;  // blobs per CTA

// positions wrapped into [0, L) in FP32
__global__ void k_block_pos(const double* __restrict__ q, int n, double lx, double ly, double lz,
                            float4* __restrict__ p) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double x = q[3 * i], y = q[3 * i + 1], z = q[3 * i + 2];
  x -= lx * floor(x / lx);
  y -= ly * floor(y / ly);
  z -= lz * floor(z / lz);
  p[i] = make_float4((float)x, (float)y, (float)z, 0.f);
}

__device__ __forceinline__ float min_image_r2(float4 a, float4 b, float lx, float ly, float lz) {
  float dx = b.x - a.x, dy = b.y - a.y, dz = b.z - a.z;
  dx -= lx * rintf(dx / lx);
  dy -= ly * rintf(dy / ly);
  dz -= lz * rintf(dz / lz);
  return dx * dx + dy * dy + dz * dz;
}

// One warp per blob i: slot 0 = i, slots 1..c its neighbours within rc (the
// nearest kBlockMax - 1 when more); cnt[i] = c + 1.
constexpr int kCand = 128;  // candidates a warp keeps before choosing the nearest
__global__ void __launch_bounds__(kWarps * 32) k_block_neighbours(const float4* __restrict__ p, int n, float lx,
                                                                  float ly, float lz, float rc2,
                                                                  int* __restrict__ idx, int* __restrict__ cnt) {
  __shared__ int ci[kWarps][kCand];
  __shared__ float cr[kWarps][kCand];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i = blockIdx.x * kWarps + w;
  if (i >= n) return;  // whole warps leave together
  const float4 pi = p[i];
  int c = 0;  // candidates found (all of them, kept or not)
  for (int j0 = 0; j0 < n; j0 += 32) {
    const int j = j0 + lane;
    bool hit = false;
    float r2 = 0.f;
    if (j < n && j != i) {
      r2 = min_image_r2(pi, p[j], lx, ly, lz);
      hit = r2 < rc2;
    }
    const unsigned b = __ballot_sync(0xffffffffu, hit);
    if (hit) {
      const int slot = c + __popc(b & ((1u << lane) - 1u));
      if (slot < kCand) {
        ci[w][slot] = j;
        cr[w][slot] = r2;
      }
    }
    c += __popc(b);
  }
  __syncwarp();
  const int kept = c < kCand ? c : kCand;
  int* out = idx + (size_t)i * kBlockMax;
  if (lane == 0) out[0] = i;
  if (kept <= kBlockMax - 1) {
    for (int s = lane; s < kept; s += 32) out[1 + s] = ci[w][s];
    if (lane == 0) cnt[i] = kept + 1;
    return;
  }
  // more candidates than slots: the nearest kBlockMax - 1, one per round (key:
  // the distance's bits, which order like the value for r2 >= 0, then the slot)
  for (int r = 0; r < kBlockMax - 1; ++r) {
    unsigned long long best = ~0ull;
    for (int s = lane; s < kept; s += 32) {
      const unsigned long long key = ((unsigned long long)__float_as_uint(cr[w][s]) << 32) | (unsigned)s;
      best = key < best ? key : best;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
      best = ob < best ? ob : best;
    }
    const int bs = (int)(best & 0xFFFFFFFFu);
    if (lane == 0) {
      out[1 + r] = ci[w][bs];
      cr[w][bs] = INFINITY;  // taken: the bits of +inf order above every distance
    }
    __syncwarp();
  }
  if (lane == 0) cnt[i] = kBlockMax;
}

// One warp per blob i: the model block B over its slots (lane a owns row a),
// B p = e_0 by Gaussian elimination with partial pivoting; val[i][s] = p_s.
__global__ void __launch_bounds__(kWarps * 32) k_block_rows(const float4* __restrict__ p, int n, float lx, float ly,
                                                            float lz, BlockModel mdl, const int* __restrict__ idx,
                                                            const int* __restrict__ cnt, float* __restrict__ val) {
  __shared__ float B[kWarps][kBlockMax][kBlockMax + 1];
  __shared__ float rhs[kWarps][kBlockMax];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i = blockIdx.x * kWarps + w;
  if (i >= n) return;
  const int k = cnt[i];
  const int* J = idx + (size_t)i * kBlockMax;
  float (*b)[kBlockMax + 1] = B[w];
  if (lane < k) {  // row `lane`
    const float4 pa = p[J[lane]];
    for (int c = 0; c < k; ++c) {
      float v = mdl.diag;
      if (c != lane) {
        const float r = fmaxf(sqrtf(min_image_r2(pa, p[J[c]], lx, ly, lz)), mdl.rmin);
        v = mdl.a / r + mdl.c0 + mdl.c2 * r * r;
      }
      b[lane][c] = v;
    }
    rhs[w][lane] = lane == 0 ? 1.f : 0.f;
  }
  __syncwarp();
  for (int c = 0; c < k; ++c) {
    // pivot: the largest |b[a][c]| over rows a >= c (the same row in every lane)
    float best = (lane >= c && lane < k) ? fabsf(b[lane][c]) : -1.f;
    int row = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int orow = __shfl_xor_sync(0xffffffffu, row, o);
      if (ob > best || (ob == best && orow < row)) {
        best = ob;
        row = orow;
      }
    }
    if (row != c) {  // swap rows c and row, lane = column
      for (int col = lane; col < k; col += 32) {
        const float t = b[c][col];
        b[c][col] = b[row][col];
        b[row][col] = t;
      }
      if (lane == 0) {
        const float t = rhs[w][c];
        rhs[w][c] = rhs[w][row];
        rhs[w][row] = t;
      }
    }
    __syncwarp();
    const float piv = b[c][c];
    if (lane > c && lane < k && piv != 0.f) {
      const float f = b[lane][c] / piv;
      for (int col = c + 1; col < k; ++col) b[lane][col] -= f * b[c][col];
      rhs[w][lane] -= f * rhs[w][c];
    }
    __syncwarp();
  }
  // back substitution: x_a = (rhs_a - sum_{l > a} b[a][l] x_l) / b[a][a]
  float xa = 0.f;  // lane a's unknown once known
  for (int a = k - 1; a >= 0; --a) {
    float t = (lane > a && lane < k) ? b[a][lane] * xa : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    const float d = b[a][a];
    const float xv = d != 0.f ? (rhs[w][a] - t) / d : 0.f;
    if (lane == a) xa = xv;
  }
  if (lane < k) val[(size_t)i * kBlockMax + lane] = xa;
}

// Sum over the block (256 threads) in the order of the library's two-stage
// reductions (warps by shuffles, then warp 0 over the warps' sums); thread 0.
__device__ __forceinline__ double block_sum256(double v) {
  __shared__ double sw[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sw[wid] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? sw[threadIdx.x] : 0.0;
  if (wid == 0)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  return v;
}

// y = P (x - shift): one warp per blob (grid-stride), lane = slot; per-CTA
// sums of y for the mean. With a ticket, the last CTA to finish (ticket taken
// after a fence; no CTA waits) also adds the per-CTA sums, as the library's
// finalize kernel does, into *mean = scale * sum(y), and resets the ticket.
template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kWarps * 32) k_block_apply(const int* __restrict__ idx, const int* __restrict__ cnt,
                                                             const float* __restrict__ val, const Tin* __restrict__ x,
                                                             const double* __restrict__ shift, int n,
                                                             Tout* __restrict__ y, double* __restrict__ partial,
                                                             unsigned* __restrict__ ticket, double* __restrict__ mean,
                                                             double scale) {
  __shared__ double ws[kWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const double sh = shift ? *shift : 0.0;
  double sum = 0.0;  // lane 0: this warp's blobs
  for (int i = blockIdx.x * kWarps + w; i < n; i += gridDim.x * kWarps) {
    const int k = cnt[i];
    double t = 0.0;
    if (lane < k) {
      const size_t o = (size_t)i * kBlockMax + lane;
      t = (double)val[o] * ((double)x[idx[o]] - sh);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) {
      y[i] = (Tout)t;
      sum += t;
    }
  }
  if (lane == 0) ws[w] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int v = 0; v < kWarps; ++v) s += ws[v];
    partial[blockIdx.x] = s;
  }
  if (!ticket) return;
  __shared__ bool last;
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double acc = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) acc += __ldcg(partial + i);
  acc = block_sum256(acc);
  if (threadIdx.x == 0) {
    *mean = acc * scale;
    *ticket = 0u;
  }
}

}  // namespace

double periodic_constant(double lx, double ly, double lz) {
  // Ewald splitting of the zero-mean periodic Green's function of -Laplace:
  // G(r) - 1 / (4 pi r) at r -> 0 = real-space images + reciprocal sum
  // - beta / (2 pi^1.5) - 1 / (4 beta^2 V). Shells per axis reach
  // beta r = 6.5 in real space and k^2 / (4 beta^2) = 42 in reciprocal space
  // (both terms below 1e-18 there), whatever the box's shape.
  const double V = lx * ly * lz, pi = 3.14159265358979323846;
  const double beta = std::sqrt(pi) / std::cbrt(V);
  const double rcut = 6.5 / beta, kcut = 2.0 * beta * std::sqrt(42.0);
  const int rx = (int)std::ceil(rcut / lx), ry = (int)std::ceil(rcut / ly), rz = (int)std::ceil(rcut / lz);
  const int kx = (int)std::ceil(kcut * lx / (2 * pi)), ky = (int)std::ceil(kcut * ly / (2 * pi)),
            kz = (int)std::ceil(kcut * lz / (2 * pi));
  double real = 0.0, recip = 0.0;
  for (int a = -rx; a <= rx; ++a)
    for (int b = -ry; b <= ry; ++b)
      for (int c = -rz; c <= rz; ++c) {
        if (!a && !b && !c) continue;
        const double r = std::sqrt((a * lx) * (a * lx) + (b * ly) * (b * ly) + (c * lz) * (c * lz));
        if (r < rcut) real += std::erfc(beta * r) / (4.0 * pi * r);
      }
  for (int a = -kx; a <= kx; ++a)
    for (int b = -ky; b <= ky; ++b)
      for (int c = -kz; c <= kz; ++c) {
        if (!a && !b && !c) continue;
        const double k2 = 4.0 * pi * pi * ((a / lx) * (a / lx) + (b / ly) * (b / ly) + (c / lz) * (c / lz));
        if (k2 < kcut * kcut) recip += std::exp(-k2 / (4.0 * beta * beta)) / k2;
      }
  return real - beta / (2.0 * std::pow(pi, 1.5)) + recip / V - 1.0 / (4.0 * beta * beta * V);
}

void launch_block_setup(const double* q, int n, double lx, double ly, double lz, double cutoff, BlockModel mdl,
                        float4* pos, int* idx, int* cnt, float* val, cudaStream_t s) {
  if (n <= 0) return;
  prof_begin(P_SETUP, s);
  k_block_pos<<<(n + 255) / 256, 256, 0, s>>>(q, n, lx, ly, lz, pos);
  prof_end(P_SETUP, s, "block_pos");
  const int blocks = (n + kWarps - 1) / kWarps;
  prof_begin(P_SETUP, s);
  k_block_neighbours<<<blocks, kWarps * 32, 0, s>>>(pos, n, (float)lx, (float)ly, (float)lz,
                                                    (float)(cutoff * cutoff), idx, cnt);
  prof_end(P_SETUP, s, "block_neighbours");
  prof_begin(P_SETUP, s);
  k_block_rows<<<blocks, kWarps * 32, 0, s>>>(pos, n, (float)lx, (float)ly, (float)lz, mdl, idx, cnt, val);
  prof_end(P_SETUP, s, "block_rows");
}

template <typename Tin, typename Tout>
void launch_block_apply(const int* idx, const int* cnt, const float* val, const Tin* x, const double* shift, int n,
                        Tout* y, double* partial, cudaStream_t s, unsigned* ticket, double* mean, double mean_scale) {
  static_assert(kWarps * 32 == kRedThreads, "the mean's reduction follows the finalize kernel's thread mapping");
  prof_begin(P_SMALL, s);
  k_block_apply<Tin, Tout><<<kBlockApplyBlocks, kWarps * 32, 0, s>>>(idx, cnt, val, x, shift, n, y, partial,
                                                                     mean ? ticket : nullptr, mean, mean_scale);
  // slots (index and value) read once, x gathered, y written
  prof_end(P_SMALL, s, "block_apply", (8.0 * kBlockMax + 2.0 * sizeof(Tin) + sizeof(Tout)) * n);
}

template void launch_block_apply<double, double>(const int*, const int*, const float*, const double*, const double*,
                                                 int, double*, double*, cudaStream_t, unsigned*, double*, double);
template void launch_block_apply<float, float>(const int*, const int*, const float*, const float*, const double*,
                                               int, float*, double*, cudaStream_t, unsigned*, double*, double);

}  // namespace ibrd
