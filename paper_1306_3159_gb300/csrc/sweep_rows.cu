// Row-resident red-black Gauss-Seidel sweep for large FP32 levels (Sec. III.E:
// the multigrid smoother of the Helmholtz problem A = alpha I - chi L).
//
// One full sweep (red cells from the old black values, then black cells from
// the new red values; red = (i + j + k) even) in one pass over memory, for
// levels whose rows are 128 or 256 cells long:
//
// * A warp owns whole x-rows: lane l holds the 4-cell groups 4 l + 128 s
//   (s < NS = nx / 128) of its row, so the x-neighbours of a group's end cells
//   come from the neighbouring lanes by shuffles, and the periodic wrap in x is
//   the shuffle from lane 31 to lane 0. No x-halo exists.
// * A CTA owns TY rows of every plane of a z-chunk, plus one halo row on each
//   side in y whose red cells it also updates (the black cells at the tile's
//   edge rows need them); the neighbouring CTA computes the same red values
//   from the same old data, bit for bit.
// * Planes arrive by TMA: one thread issues 3-D tensor-map box copies (the
//   tile's rows plus 2-row halos of x, the tile's rows plus 1-row halos of b)
//   into a ring of R planes, completing on one mbarrier per ring slot. The
//   periodic wrap in y is the halo boxes' start row, taken modulo ny on the
//   host side of the index (every box starts at x = 0, so the 16-byte rule on
//   the innermost coordinate holds).
// * Each thread keeps its row of planes p-2 .. p+1 in registers (the
//   z-neighbours); only the y-neighbour rows are read from shared memory: the
//   old rows for the red update of plane p, and the red-updated rows (a
//   separate double-buffered array, so no row is read while it is written)
//   for the black update of plane p-1 in the same phase. One barrier per
//   plane.
//
// Every mbarrier wait is bounded: a wait that gives up sets *err, drains the
// copies still in flight (again with a bound) and ends the CTA; the host
// turns the flag into IBRD_ERR_TIMEOUT.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "internal.h"

namespace ibrd {
namespace {

constexpr int kRowsTY = 8;    // tile rows per CTA
constexpr int kRowsRing = 4;  // planes in the TMA ring (prefetch distance 2)
constexpr unsigned kDrainLimit = 1u << 26;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
// true when the phase with this parity completed within `limit` tries
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, unsigned limit) {
  for (unsigned i = 0; i < limit; ++i) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}
__device__ __forceinline__ void tma_load3(unsigned dst, const CUtensorMap* map, int x, int y, int z, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];\n" ::"r"(dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

__device__ __forceinline__ int wrapm(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// Gauss-Seidel update of the active cells of one row held as NS 4-vectors
// per lane: active cells are e = a, a + 2 of every group (e = x mod 4). Their
// x-neighbours are inactive cells (unchanged by this update): inside the
// group, or the previous lane's last cell (a = 0) / the next lane's first
// cell (a = 1), with lane 0 / lane 31 taking it from the adjacent slot. u and
// dn are the rows j - 1 and j + 1, zm and zp the planes k - 1 and k + 1, bb
// the right-hand side with its shift removed.
template <int NS>
__device__ __forceinline__ void rb_row(float4 (&v)[NS], const float4* u, const float4* dn, const float4 (&zm)[NS],
                                       const float4 (&zp)[NS], const float4 (&bb)[NS], int a, float off, float inv,
                                       int lane) {
  float t[NS];
  if (a == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) t[s] = __shfl_sync(0xffffffffu, v[s].w, (lane + 31) & 31);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const float L = lane == 0 ? t[(s + NS - 1) % NS] : t[s];
      const float4 uu = u[32 * s], dd = dn[32 * s];
      v[s].x = (bb[s].x + off * (((L + v[s].y) + (uu.x + dd.x)) + (zm[s].x + zp[s].x))) * inv;
      v[s].z = (bb[s].z + off * (((v[s].y + v[s].w) + (uu.z + dd.z)) + (zm[s].z + zp[s].z))) * inv;
    }
  } else {
#pragma unroll
    for (int s = 0; s < NS; ++s) t[s] = __shfl_sync(0xffffffffu, v[s].x, (lane + 1) & 31);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const float R = lane == 31 ? t[(s + 1) % NS] : t[s];
      const float4 uu = u[32 * s], dd = dn[32 * s];
      v[s].y = (bb[s].y + off * (((v[s].x + v[s].z) + (uu.y + dd.y)) + (zm[s].y + zp[s].y))) * inv;
      v[s].w = (bb[s].w + off * (((v[s].z + R) + (uu.w + dd.w)) + (zm[s].w + zp[s].w))) * inv;
    }
  }
}

// Grid: (ny / TY, z-chunks). Block: (TY + 2) warps; warp w owns row
// y0 - 1 + w (w = 0 and w = TY + 1 are the halo rows: red cells only).
// Shared memory: XS[R][TY + 4][nx] (old x, rows y0-2 .. y0+TY+1),
// BS[R][TY + 2][nx] (b, rows y0-1 .. y0+TY), RS[2][TY + 2][nx] (rows after the
// red update), R mbarriers.
template <int NS>
__global__ void __launch_bounds__((kRowsTY + 2) * 32, 2)
    k_rbgs_rows(const __grid_constant__ CUtensorMap mx_tile, const __grid_constant__ CUtensorMap mx_pair,
                const __grid_constant__ CUtensorMap mb_tile, const __grid_constant__ CUtensorMap mb_one,
                float* __restrict__ xout, const double* __restrict__ bshift, int ny, int nz, int zc, float inv,
                float off, double* __restrict__ part, int* __restrict__ err, unsigned wait_limit) {
  constexpr int TY = kRowsTY, R = kRowsRing, NX = 128 * NS;
  constexpr int XROWS = TY + 4, BROWS = TY + 2, RROWS = TY + 2;
  constexpr unsigned XBYTES = XROWS * NX * 4, BBYTES = BROWS * NX * 4;
  extern __shared__ __align__(1024) unsigned char sm_raw[];
  float* XS = reinterpret_cast<float*>(sm_raw);
  float* BS = XS + R * XROWS * NX;
  float* RS = BS + R * BROWS * NX;
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(RS + 2 * RROWS * NX);

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int y0 = blockIdx.x * TY;
  const int k0 = blockIdx.y * zc, k1 = min(k0 + zc, nz);
  const size_t plane = (size_t)NX * ny;
  const float sh = bshift ? (float)(*bshift) : 0.f;
  const bool interior = w >= 1 && w <= TY;
  // this warp's row: parity of y (ny is even, so the wrap keeps it)
  const int ypar = (y0 - 1 + w) & 1;
  const int q0 = k0 - 2;  // first plane in the ring

  if (tid == 0) {
    for (int s = 0; s < R; ++s) mbar_init(smem_u32(bars + s), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();

  // copies of plane q (x rows y0-2 .. y0+TY+1, b rows y0-1 .. y0+TY) into its slot
  auto issue = [&](int q) {
    const int s = (q - q0) % R;
    const unsigned bar = smem_u32(bars + s);
    const int z = wrapm(q, nz);
    float* xs = XS + s * XROWS * NX;
    float* bs = BS + s * BROWS * NX;
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    mbar_expect_tx(bar, XBYTES + BBYTES);
    tma_load3(smem_u32(xs), &mx_pair, 0, wrapm(y0 - 2, ny), z, bar);
    tma_load3(smem_u32(xs + 2 * NX), &mx_tile, 0, y0, z, bar);
    tma_load3(smem_u32(xs + (TY + 2) * NX), &mx_pair, 0, wrapm(y0 + TY, ny), z, bar);
    tma_load3(smem_u32(bs), &mb_one, 0, wrapm(y0 - 1, ny), z, bar);
    tma_load3(smem_u32(bs + NX), &mb_tile, 0, y0, z, bar);
    tma_load3(smem_u32(bs + (TY + 1) * NX), &mb_one, 0, wrapm(y0 + TY, ny), z, bar);
  };
  auto wait_plane = [&](int q, unsigned limit) {
    const int u = q - q0;
    return mbar_wait(smem_u32(bars + (u % R)), (unsigned)((u / R) & 1), limit);
  };
  auto xrow = [&](int q, int r) { return reinterpret_cast<const float4*>(XS + ((q - q0) % R) * XROWS * NX + r * NX); };
  auto brow = [&](int q, int r) { return reinterpret_cast<const float4*>(BS + ((q - q0) % R) * BROWS * NX + r * NX); };
  auto rrow = [&](int q, int r) { return reinterpret_cast<float4*>(RS + (q & 1) * RROWS * NX + r * NX); };

  const int last = k1 + 1;  // last plane loaded
  if (tid == 0)
    for (int q = q0; q < q0 + R && q <= last; ++q) issue(q);
  int issued = min(q0 + R - 1, last);

  float4 A[NS], B[NS], C[NS], D[NS], BX[NS], BY[NS];
  bool ok = wait_plane(q0, wait_limit) && wait_plane(q0 + 1, wait_limit);
  if (ok) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      B[s] = xrow(q0, w + 1)[lane + 32 * s];
      C[s] = xrow(q0 + 1, w + 1)[lane + 32 * s];
    }
  }
  ok = !__syncthreads_or(!ok);
  // planes up to `done` have landed (the same value in every thread: it only
  // advances after a barrier all threads passed with their waits met)
  int done = ok ? q0 + 1 : q0 - 1;
  float acc = 0.f, comp = 0.f;  // Kahan sum of the new x (tile rows)

  // Phase p: red cells of plane p (all warps), black cells of plane p - 1
  // (tile warps, p - 1 >= k0), store of plane p - 1. pm2 .. pp1 are this
  // thread's row of planes p - 2 .. p + 1; bm1 / b0 its b of planes p - 1 / p.
  auto phase = [&](float4 (&pm2)[NS], float4 (&pm1)[NS], float4 (&p0)[NS], float4 (&pp1)[NS],
                   float4 (&bm1)[NS], float4 (&b0)[NS], int p) -> bool {
    if (p > k1 || !ok) return false;
    // plane p + 3 takes the slot of plane p - 1, last read before the barrier
    // that ended phase p - 1
    if (tid == 0 && p + 3 <= last) issue(p + 3);
    if (p + 3 <= last) issued = p + 3;
    bool good = wait_plane(p + 1, wait_limit);
    if (good) {
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        pp1[s] = xrow(p + 1, w + 1)[lane + 32 * s];
        float4 t = brow(p, w)[lane + 32 * s];
        t.x -= sh, t.y -= sh, t.z -= sh, t.w -= sh;
        b0[s] = t;
      }
      // red cells of plane p from the old rows y - 1, y + 1 of plane p
      rb_row<NS>(p0, xrow(p, w) + lane, xrow(p, w + 2) + lane, pm1, pp1, b0, (ypar + p) & 1, off, inv, lane);
      float4* rr = rrow(p, w);
#pragma unroll
      for (int s = 0; s < NS; ++s) rr[lane + 32 * s] = p0[s];
      if (interior && p - 1 >= k0) {
        // black cells of plane p - 1 from the red-updated rows of plane p - 1
        rb_row<NS>(pm1, rrow(p - 1, w - 1) + lane, rrow(p - 1, w + 1) + lane, pm2, p0, bm1, (ypar + p) & 1, off,
                   inv, lane);
        float4* dst = reinterpret_cast<float4*>(xout + (size_t)(p - 1) * plane + (size_t)(y0 - 1 + w) * NX);
#pragma unroll
        for (int s = 0; s < NS; ++s) dst[lane + 32 * s] = pm1[s];
        if (part) {
          float t = 0.f;
#pragma unroll
          for (int s = 0; s < NS; ++s) t += (pm1[s].x + pm1[s].y) + (pm1[s].z + pm1[s].w);
          const float yk = t - comp, tk = acc + yk;
          comp = (tk - acc) - yk;
          acc = tk;
        }
      }
    }
    ok = !__syncthreads_or(!good);
    if (ok) done = p + 1;
    return ok;
  };
  for (int p = k0 - 1; p <= k1; p += 4) {
    if (!phase(A, B, C, D, BX, BY, p)) break;
    if (!phase(B, C, D, A, BY, BX, p + 1)) break;
    if (!phase(C, D, A, B, BX, BY, p + 2)) break;
    if (!phase(D, A, B, C, BY, BX, p + 3)) break;
  }
  if (!ok) {
    // a plane wait gave up: drain the copies still in flight, report, stop
    for (int q = done + 1; q <= issued; ++q) wait_plane(q, kDrainLimit);
    if (tid == 0) atomicOr(err, 1);
    return;
  }
  if (part) {
    double v = (double)acc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __shared__ double ws[TY + 2];
    if (lane == 0) ws[w] = v;
    __syncthreads();
    if (tid == 0) {
      double sum = 0.0;
      for (int i = 0; i < TY + 2; ++i) sum += ws[i];
      part[blockIdx.x + gridDim.x * blockIdx.y] = sum;
    }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  if (!fn) throw CudaError{cudaErrorNotSupported, "cuTensorMapEncodeTiled entry point"};
  return fn;
}

// Tensor map of an FP32 field [nz][ny][nx] with boxes of nx x rows x 1.
CUtensorMap field_map(const float* f, Dims d, int rows) {
  CUtensorMap m;
  std::memset(&m, 0, sizeof(m));
  const cuuint64_t dims[3] = {(cuuint64_t)d.nx, (cuuint64_t)d.ny, (cuuint64_t)d.nz};
  const cuuint64_t strides[2] = {(cuuint64_t)d.nx * 4, (cuuint64_t)d.nx * d.ny * 4};
  const cuuint32_t box[3] = {(cuuint32_t)d.nx, (cuuint32_t)rows, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(f), dims, strides, box,
                                 es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw CudaError{cudaErrorInvalidValue, "cuTensorMapEncodeTiled"};
  return m;
}

template <int NS>
constexpr size_t rows_smem() {
  constexpr int NX = 128 * NS;
  return sizeof(float) * (size_t)NX * (kRowsRing * (kRowsTY + 4) + kRowsRing * (kRowsTY + 2) + 2 * (kRowsTY + 2)) +
         8 * kRowsRing;
}

template <int NS>
void rows_launch(dim3 g, cudaStream_t s, const CUtensorMap (&m)[4], float* xout, const double* bshift, Dims d,
                 int zc, float inv, float off, double* part, int* err, unsigned limit) {
  constexpr size_t sm = rows_smem<NS>();
  static std::atomic<unsigned long long> attr{0};
  ensure_smem_attr((const void*)k_rbgs_rows<NS>, (int)sm, attr);
  k_rbgs_rows<NS><<<g, (kRowsTY + 2) * 32, sm, s>>>(m[0], m[1], m[2], m[3], xout, bshift, d.ny, d.nz, zc, inv, off,
                                                     part, err, limit);
}

}  // namespace

bool rows_sweep_ok(Dims d) {
  return (d.nx == 128 || d.nx == 256) && d.ny % kRowsTY == 0 && d.ny >= kRowsTY && d.nz % 2 == 0 && d.nz >= 4;
}

int rows_sweep_default_zc(Dims d) {
  // about one wave of two resident CTAs per SM
  const int cols = d.ny / kRowsTY;
  int chunks = (2 * 152) / cols;
  chunks = chunks < 1 ? 1 : chunks;
  int zc = (d.nz + chunks - 1) / chunks;
  return zc < 2 ? 2 : zc;
}

int launch_rows_sweep(const float* xin, float* xout, const float* b, const double* bshift, Dims d, Stencil st,
                      int zc, double* part, int part_cap, cudaStream_t s) {
  if (!rows_sweep_ok(d) || !aligned16(xin) || !aligned16(xout) || !aligned16(b) || xin == xout || b == xout)
    throw CudaError{cudaErrorInvalidValue, "row sweep arguments"};
  zc = zc < 2 ? 2 : (zc > d.nz ? d.nz : zc);
  const CUtensorMap m[4] = {field_map(xin, d, kRowsTY), field_map(xin, d, 2), field_map(b, d, kRowsTY),
                            field_map(b, d, 1)};
  dim3 g(d.ny / kRowsTY, (d.nz + zc - 1) / zc);
  const int nblk = (int)(g.x * g.y);
  if (nblk > part_cap) part = nullptr;
  const float inv = (float)(1.0 / st.diag), off = (float)st.off;
  int* err = wait_error_flag();
  const unsigned limit = wait_limit();
  if (d.nx == 256)
    rows_launch<2>(g, s, m, xout, bshift, d, zc, inv, off, part, err, limit);
  else
    rows_launch<1>(g, s, m, xout, bshift, d, zc, inv, off, part, err, limit);
  return part ? nblk : 0;
}

}  // namespace ibrd
