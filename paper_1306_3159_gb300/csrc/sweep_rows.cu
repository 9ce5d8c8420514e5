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
//   old rows for the red update of plane p, and the red cells after that
//   update (a separate double-buffered array holding two values per 4-cell
//   group, so no row is read while it is written) for the black update of
//   plane p-1 in the same step. One barrier per plane; thread 0 alone waits
//   on the TMA barriers, one plane ahead.
// * Odd z-chunks march downwards, so that adjacent chunks meet at their
//   common halo planes at the same time (L2 hits, not DRAM re-reads).
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
constexpr int kCoarseRing = 3;  // coarse planes in the ring of the fused prolongation
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
// cell (a = 1), with lane 0 / lane 31 taking it from the adjacent slot. zm and
// zp are the planes k - 1 and k + 1, bb the right-hand side with its shift
// removed. The y-neighbours (rows j - 1, j + 1) are full rows (u, dn: float4
// per group, the active cells' values at components a, a + 2) or, PACKED,
// the neighbour rows' red-updated cells only (float2 per group: exactly the
// values at this row's black positions).
template <int NS, bool PACKED>
__device__ __forceinline__ void rb_row(float4 (&v)[NS], const void* u, const void* dn, const float4 (&zm)[NS],
                                       const float4 (&zp)[NS], const float4 (&bb)[NS], int a, float off, float inv,
                                       int lane) {
  float t[NS];
  auto nb = [&](const void* row, int s, int k) -> float {  // k-th active cell's neighbour in `row`
    if constexpr (PACKED) {
      const float2 q = reinterpret_cast<const float2*>(row)[32 * s];
      return k == 0 ? q.x : q.y;
    } else {
      const float4 q = reinterpret_cast<const float4*>(row)[32 * s];
      return a == 0 ? (k == 0 ? q.x : q.z) : (k == 0 ? q.y : q.w);
    }
  };
  if (a == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) t[s] = __shfl_sync(0xffffffffu, v[s].w, (lane + 31) & 31);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const float L = lane == 0 ? t[(s + NS - 1) % NS] : t[s];
      const float u0 = nb(u, s, 0), d0 = nb(dn, s, 0), u1 = nb(u, s, 1), d1 = nb(dn, s, 1);
      v[s].x = (bb[s].x + off * (((L + v[s].y) + (u0 + d0)) + (zm[s].x + zp[s].x))) * inv;
      v[s].z = (bb[s].z + off * (((v[s].y + v[s].w) + (u1 + d1)) + (zm[s].z + zp[s].z))) * inv;
    }
  } else {
#pragma unroll
    for (int s = 0; s < NS; ++s) t[s] = __shfl_sync(0xffffffffu, v[s].x, (lane + 1) & 31);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const float R = lane == 31 ? t[(s + 1) % NS] : t[s];
      const float u0 = nb(u, s, 0), d0 = nb(dn, s, 0), u1 = nb(u, s, 1), d1 = nb(dn, s, 1);
      v[s].y = (bb[s].y + off * (((v[s].x + v[s].z) + (u0 + d0)) + (zm[s].y + zp[s].y))) * inv;
      v[s].w = (bb[s].w + off * (((v[s].z + R) + (u1 + d1)) + (zm[s].w + zp[s].w))) * inv;
    }
  }
}

// Adds to the fine row v the coarse correction of Sec. III.E (cell-centred
// trilinear prolongation) in the order every prolongation kernel uses: z
// between the row's parent coarse plane cp and the other plane co, then y
// between the parent coarse row cr and its neighbour nr on the row's side
// (coarse planes in shared memory, NX / 2 floats per row), then x. Lane l
// holds, per slot s, fine cells 4 g .. 4 g + 3 of group g = l + 32 s, over
// coarse cells 2 g, 2 g + 1; their x-neighbours 2 g - 1 and 2 g + 2 come from
// the adjacent lanes (lane 0 / 31 from the adjacent slot: the periodic wrap).
template <int NS>
__device__ __forceinline__ void add_correction(float4 (&v)[NS], const float* cp, const float* co, int cr, int nr,
                                               int lane) {
  constexpr int NXC = 64 * NS;
  float2 zy[NS];  // the pair after z and y (16 times its value)
  float tp[NS], tn[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const int o = 2 * (lane + 32 * s);
    const float2 pp = *reinterpret_cast<const float2*>(cp + cr * NXC + o);
    const float2 op = *reinterpret_cast<const float2*>(co + cr * NXC + o);
    const float2 pn = *reinterpret_cast<const float2*>(cp + nr * NXC + o);
    const float2 on = *reinterpret_cast<const float2*>(co + nr * NXC + o);
    zy[s] = make_float2(prolong_axis(prolong_axis(pp.x, op.x), prolong_axis(pn.x, on.x)),
                        prolong_axis(prolong_axis(pp.y, op.y), prolong_axis(pn.y, on.y)));
  }
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    tp[s] = __shfl_sync(0xffffffffu, zy[s].y, (lane + 31) & 31);
    tn[s] = __shfl_sync(0xffffffffu, zy[s].x, (lane + 1) & 31);
  }
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const float z0 = lane == 0 ? tp[(s + NS - 1) % NS] : tp[s];
    const float z3 = lane == 31 ? tn[(s + 1) % NS] : tn[s];
    v[s].x = prolong_add(v[s].x, prolong_axis(zy[s].x, z0));
    v[s].y = prolong_add(v[s].y, prolong_axis(zy[s].x, zy[s].y));
    v[s].z = prolong_add(v[s].z, prolong_axis(zy[s].y, zy[s].x));
    v[s].w = prolong_add(v[s].w, prolong_axis(zy[s].y, z3));
  }
}

// Grid: (ny / TY, z-chunks). Block: (TY + 2) warps; warp w owns row
// y0 - 1 + w (w = 0 and w = TY + 1 are the halo rows: red cells only).
// Shared memory: XS[R][TY + 4][nx] (old x, rows y0-2 .. y0+TY+1),
// BS[R][TY + 2][nx] (b, rows y0-1 .. y0+TY), RS[2][TY + 2][nx / 2] (the red
// cells of each row after the red update, two per 4-cell group), R mbarriers.
//
// March order: chunk c covers planes [k0, k1) and visits planes k0-2 .. k1+1
// upwards when c is even and k1+1 .. k0-2 downwards when c is odd, so that
// neighbouring chunks start (or end) at their common boundary at the same
// time and the halo planes they share come from L2. The Gauss-Seidel result
// does not depend on the order in which the cells of one colour are updated,
// so both directions give the same sweep. March index i = 0 .. zc + 3 names
// plane mp(i); step i updates the red cells of mp(i) and the black cells of
// mp(i - 1) (when that plane is in the chunk) and stores mp(i - 1).
//
// PRO: the sweep that follows the coarse-grid correction, with the
// correction fused: x (xin) arrives uncorrected, and every x value the sweep
// reads is x + P xc, P the cell-centred trilinear prolongation of the coarse
// field xc, in the arithmetic of the stand-alone prolongation kernel. The
// coarse planes arrive by TMA into a ring of kCoarseRing slots of TY / 2 + 4
// coarse rows (the parents of the tile's rows and their neighbours), riding
// on the barriers of the fine planes. Fine planes 2K - 1 and 2K share the
// coarse pair {K - 1, K}, so in march order every second fine plane brings a
// new coarse plane (coarse march plane j = i / 2 + 2 first serves the
// correction of fine march plane i + 1, i even). Each thread corrects its own
// row of plane i + 1 in registers when it loads it and writes it back for the
// y-neighbour reads of step i + 1; the halo warps also correct the two outer
// x rows. Chunks hold an even number of planes so that the pairing is the same
// in both march directions.
template <int NS, bool PRO>
__global__ void __launch_bounds__((kRowsTY + 2) * 32, 2)
    k_rbgs_rows(const __grid_constant__ CUtensorMap mx_tile, const __grid_constant__ CUtensorMap mx_pair,
                const __grid_constant__ CUtensorMap mb_tile, const __grid_constant__ CUtensorMap mb_one,
                const __grid_constant__ CUtensorMap mc_half, const __grid_constant__ CUtensorMap mc_pair,
                float* __restrict__ xout, const double* __restrict__ bshift, int ny, int nz, int zc, float inv,
                float off, double* __restrict__ part, int* __restrict__ err, unsigned wait_limit) {
  constexpr int TY = kRowsTY, R = kRowsRing, NX = 128 * NS;
  constexpr int XROWS = TY + 4, BROWS = TY + 2, RROWS = TY + 2, RW = NX / 2;
  constexpr int NXC = NX / 2, CROWS = TY / 2 + 4;
  constexpr unsigned XBYTES = XROWS * NX * 4, BBYTES = BROWS * NX * 4, CBYTES = CROWS * NXC * 4;
  extern __shared__ __align__(1024) unsigned char sm_raw[];
  float* XS = reinterpret_cast<float*>(sm_raw);
  float* BS = XS + R * XROWS * NX;
  float* RS = BS + R * BROWS * NX;
  float* CS = RS + 2 * RROWS * RW;
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(CS + (PRO ? kCoarseRing * CROWS * NXC : 0));

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int y0 = blockIdx.x * TY;
  const int k0 = blockIdx.y * zc, k1 = min(k0 + zc, nz);
  const bool down = blockIdx.y & 1;
  const size_t plane = (size_t)NX * ny;
  const float sh = bshift ? (float)(*bshift) : 0.f;
  const bool interior = w >= 1 && w <= TY;
  // this warp's row: parity of y (ny is even, so the wrap keeps it)
  const int ypar = (y0 - 1 + w) & 1;
  const int last = k1 - k0 + 3;  // march index of the last plane
  auto mp = [&](int i) { return down ? k1 + 1 - i : k0 - 2 + i; };
  // coarse march plane j and the one a fine plane's copy brings (-1: none)
  auto cmp = [&](int j) { return down ? (k1 >> 1) + 1 - j : (k0 >> 1) - 2 + j; };
  auto cj_of = [&](int i) { return i <= 3 ? i : ((i & 1) ? (i + 3) >> 1 : -1); };
  // coarse rows of this warp's own row: its parent and the parent's neighbour
  const int cr = ((w + 1) >> 1) + 1, nr = (w & 1) ? cr - 1 : cr + 1;

  if (tid == 0) {
    for (int s = 0; s < R; ++s) mbar_init(smem_u32(bars + s), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();

  // copies of march plane i (x rows y0-2 .. y0+TY+1, b rows y0-1 .. y0+TY) into its slot
  // box start rows, wrapped once (march planes lie in [-2, nz + 1], coarse
  // march planes in [-2, nz / 2 + 1]: one compare wraps them)
  const int ya = wrapm(y0 - 2, ny), yb = wrapm(y0 + TY, ny), yh = wrapm(y0 - 1, ny);
  const int nyc = ny >> 1, nzc = nz >> 1, yc = y0 >> 1;
  const int yca = wrapm(yc - 2, nyc), ycb = wrapm(yc + TY / 2, nyc);
  auto issue = [&](int i) {
    const int s = i % R;
    const unsigned bar = smem_u32(bars + s);
    int z = mp(i);
    z += z < 0 ? nz : (z >= nz ? -nz : 0);
    float* xs = XS + s * XROWS * NX;
    float* bs = BS + s * BROWS * NX;
    const int j = PRO ? cj_of(i) : -1;
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    mbar_expect_tx(bar, XBYTES + BBYTES + (j >= 0 ? CBYTES : 0u));
    tma_load3(smem_u32(xs), &mx_pair, 0, ya, z, bar);
    tma_load3(smem_u32(xs + 2 * NX), &mx_tile, 0, y0, z, bar);
    tma_load3(smem_u32(xs + (TY + 2) * NX), &mx_pair, 0, yb, z, bar);
    tma_load3(smem_u32(bs), &mb_one, 0, yh, z, bar);
    tma_load3(smem_u32(bs + NX), &mb_tile, 0, y0, z, bar);
    tma_load3(smem_u32(bs + (TY + 1) * NX), &mb_one, 0, yb, z, bar);
    if (PRO && j >= 0) {
      // coarse rows y0/2 - 2 .. y0/2 + TY/2 + 1 of coarse plane cmp(j)
      float* cs = CS + (j % kCoarseRing) * CROWS * NXC;
      int kc = cmp(j);
      kc += kc < 0 ? nzc : (kc >= nzc ? -nzc : 0);
      tma_load3(smem_u32(cs), &mc_pair, 0, yca, kc, bar);
      tma_load3(smem_u32(cs + 2 * NXC), &mc_half, 0, yc, kc, bar);
      tma_load3(smem_u32(cs + (TY / 2 + 2) * NXC), &mc_pair, 0, ycb, kc, bar);
    }
  };
  // thread 0 alone polls the barriers; the CTA barrier that follows every
  // wait publishes the landed plane to the other threads
  auto wait_plane = [&](int i, unsigned limit) {
    return mbar_wait(smem_u32(bars + (i % R)), (unsigned)((i / R) & 1), limit);
  };
  auto xrow = [&](int i, int r) { return reinterpret_cast<const float4*>(XS + (i % R) * XROWS * NX + r * NX); };
  auto brow = [&](int i, int r) { return reinterpret_cast<const float4*>(BS + (i % R) * BROWS * NX + r * NX); };
  auto rrow = [&](int i, int r) { return reinterpret_cast<float2*>(RS + (i & 1) * RROWS * RW + r * RW); };
  auto xroww = [&](int i, int r) { return reinterpret_cast<float4*>(XS + (i % R) * XROWS * NX + r * NX); };
  auto cslot = [&](int j) -> const float* { return CS + (j % kCoarseRing) * CROWS * NXC; };
  // PRO, halo warps: correct x row 0 (warp 0) or TY + 3 (warp TY + 1) of
  // march plane i in shared memory; cp / co: parent / other coarse plane
  const bool outer = w == 0 || w == TY + 1;
  auto fix_outer = [&](int i, const float* cp, const float* co) {
    const bool top = w == 0;
    float4 v[NS];
    float4* row = xroww(i, top ? 0 : TY + 3) + lane;
#pragma unroll
    for (int s = 0; s < NS; ++s) v[s] = row[32 * s];
    add_correction<NS>(v, cp, co, top ? 1 : CROWS - 2, top ? 0 : CROWS - 1, lane);
#pragma unroll
    for (int s = 0; s < NS; ++s) row[32 * s] = v[s];
  };

  bool ok = true;
  if (tid == 0) {
    // PRO: plane 3's copy brings coarse plane 3 into the slot of coarse
    // plane 0, which the prologue still reads: it is issued after it
    for (int i = 0; i < (PRO ? 3 : R) && i <= last; ++i) issue(i);
    ok = wait_plane(0, wait_limit) && wait_plane(1, wait_limit) && wait_plane(2, wait_limit);
  }
  int issued = PRO ? 2 : min(R - 1, last);
  ok = !__syncthreads_or(!ok);
  // march planes up to `done` have landed (the same value in every thread:
  // it only advances after a barrier that every thread passed)
  int done = ok ? 2 : -1;

  float4 A[NS], B[NS], C[NS], D[NS], BX[NS], BY[NS];
  if (ok) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      B[s] = xrow(0, w + 1)[lane + 32 * s];
      C[s] = xrow(1, w + 1)[lane + 32 * s];
    }
    if constexpr (PRO) {
      // fine march planes 0 and 1 have the parent coarse plane 1; the other
      // plane is 0 for plane 0 and 2 for plane 1
      add_correction<NS>(B, cslot(1), cslot(0), cr, nr, lane);
      add_correction<NS>(C, cslot(1), cslot(2), cr, nr, lane);
#pragma unroll
      for (int s = 0; s < NS; ++s) xroww(1, w + 1)[lane + 32 * s] = C[s];
      if (outer) fix_outer(1, cslot(1), cslot(2));
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
  }
  __syncthreads();  // step 1 refills plane 0's slot
  if (PRO && ok) {
    if (tid == 0) issue(3);
    issued = 3;
  }
  float acc = 0.f, comp = 0.f;  // Kahan sum of the new x (tile rows)

  // Step i: pm2 .. pp1 are this thread's row of march planes i - 2 .. i + 1,
  // bm1 / b0 its b of march planes i - 1 / i. Planes i and i + 1 have landed.
  auto step = [&](float4 (&pm2)[NS], float4 (&pm1)[NS], float4 (&p0)[NS], float4 (&pp1)[NS], float4 (&bm1)[NS],
                  float4 (&b0)[NS], int i, bool odd) -> bool {
    if (i > last - 1 || !ok) return false;
    // plane i + 3 takes the slot of plane i - 1, last read before the barrier
    // that ended step i - 1 (PRO, even i: its copy brings coarse plane
    // i / 2 + 3 into the slot of coarse plane i / 2, last read in step i - 1)
    if (tid == 0 && i + 3 <= last) issue(i + 3);
    if (i + 3 <= last) issued = i + 3;
    const int z = mp(i);
#pragma unroll
    for (int s = 0; s < NS; ++s) pp1[s] = xrow(i + 1, w + 1)[lane + 32 * s];
    if constexpr (PRO) {
      // correct plane i + 1: odd i keeps the coarse pair of step i - 1, whose
      // newer plane is the parent; even i brings coarse plane i / 2 + 2 (the
      // other) and the parent is the plane before it
      const int jp = odd ? ((i - 1) >> 1) + 2 : (i >> 1) + 1;
      const int jo = odd ? jp - 1 : jp + 1;
      add_correction<NS>(pp1, cslot(jp), cslot(jo), cr, nr, lane);
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      float4 t = brow(i, w)[lane + 32 * s];
      t.x -= sh, t.y -= sh, t.z -= sh, t.w -= sh;
      b0[s] = t;
    }
    const int a = (ypar + z) & 1;
    // red cells of plane mp(i) from the old rows y - 1, y + 1 of that plane
    rb_row<NS, false>(p0, xrow(i, w) + lane, xrow(i, w + 2) + lane, pm1, pp1, b0, a, off, inv, lane);
    float2* rr = rrow(i, w);
#pragma unroll
    for (int s = 0; s < NS; ++s)
      rr[lane + 32 * s] = a == 0 ? make_float2(p0[s].x, p0[s].z) : make_float2(p0[s].y, p0[s].w);
    if (interior && i >= 3) {
      // black cells of plane mp(i - 1) from the red cells of its rows y - 1, y + 1
      rb_row<NS, true>(pm1, rrow(i - 1, w - 1) + lane, rrow(i - 1, w + 1) + lane, pm2, p0, bm1, a, off, inv,
                       lane);
      float4* dst = reinterpret_cast<float4*>(xout + (size_t)mp(i - 1) * plane + (size_t)(y0 - 1 + w) * NX);
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
    if constexpr (PRO) {
      // the corrected rows of plane i + 1 for the y-neighbour reads of step
      // i + 1 (nothing reads that plane's rows in this step); the outer rows
      // from the halo warps; then the writers' proxy fence, as TMA later
      // refills the slot
      const int jp = odd ? ((i - 1) >> 1) + 2 : (i >> 1) + 1;
      const int jo = odd ? jp - 1 : jp + 1;
#pragma unroll
      for (int s = 0; s < NS; ++s) xroww(i + 1, w + 1)[lane + 32 * s] = pp1[s];
      if (outer) fix_outer(i + 1, cslot(jp), cslot(jo));
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    bool good = true;
    if (tid == 0 && i + 2 <= last) good = wait_plane(i + 2, wait_limit);
    ok = !__syncthreads_or(!good);
    if (ok) done = i + 2;
    return ok;
  };
  for (int i = 1; i < last; i += 4) {
    if (!step(A, B, C, D, BX, BY, i, true)) break;
    if (!step(B, C, D, A, BY, BX, i + 1, false)) break;
    if (!step(C, D, A, B, BX, BY, i + 2, true)) break;
    if (!step(D, A, B, C, BY, BX, i + 3, false)) break;
  }
  if (!ok) {
    // a plane wait gave up: drain the copies still in flight, report, stop
    if (tid == 0) {
      for (int i = done + 1; i <= issued; ++i) wait_plane(i, kDrainLimit);
      atomicOr(err, 1);
    }
    __syncthreads();
    return;
  }
  if (part) {
    double v = (double)acc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    double* ws = reinterpret_cast<double*>(RS);  // no step reads RS after the last barrier
    if (lane == 0) ws[w] = v;
    __syncthreads();
    if (tid == 0) {
      double sum = 0.0;
      for (int i = 0; i < TY + 2; ++i) sum += ws[i];
      part[blockIdx.x + gridDim.x * blockIdx.y] = sum;
    }
  }
}

// First red-black sweep from x = 0 fused with the residual restriction, for
// the same levels as the sweep above: x = one sweep of A x = b - shift from
// zero (red cells (b - shift) / diag, black cells from their red neighbours,
// the arithmetic of k_rb_zero_f32v) and bc = mean over the 8 children of
// b - shift - A x, in one pass over b (HBM: read b, write x and bc).
//
// Layout as in k_rbgs_rows: warp w owns row y0 - 1 + w of every plane; a ring
// of R b-planes (rows y0-2 .. y0+TY+1) arrives by TMA; the march order
// alternates between even and odd z-chunks. Step i forms x on march plane i
// (all warps, rows y0-1 .. y0+TY: the edge rows' residuals need them) from b
// of planes i-1 .. i+1, and the residual of march plane i-1 (tile warps) from
// x of planes i-2 .. i; x rows go through shared memory (XB, double-buffered)
// for the y-neighbours. Restriction: the two cells of a coarse cell along x
// sit in one lane, the two planes along z are summed in registers over two
// steps, and the two rows along y belong to warps w (even y) and w + 1 (odd
// y): when a plane pair is complete the odd row's warp leaves its sums in
// shared memory (RY) and the even row's warp adds them one step later (after
// the step's barrier) and writes the coarse row. Chunks start on even planes
// and hold an even number of them, so plane pairs never straddle chunks.
template <int NS>
__global__ void __launch_bounds__((kRowsTY + 2) * 32, 2)
    k_zr_rows(const __grid_constant__ CUtensorMap mb_tile, const __grid_constant__ CUtensorMap mb_pair,
              float* __restrict__ xout, float* __restrict__ bc, const double* __restrict__ bshift, int ny, int nz,
              int zc, float inv, float off, float diag, int* __restrict__ err, unsigned wait_limit) {
  constexpr int TY = kRowsTY, R = kRowsRing, NX = 128 * NS, NXC = NX / 2;
  constexpr int XROWS = TY + 4, XBROWS = TY + 2;
  constexpr unsigned BBYTES = XROWS * NX * 4;
  extern __shared__ __align__(1024) unsigned char sm_raw[];
  float* BSM = reinterpret_cast<float*>(sm_raw);        // R b planes, rows y0-2 .. y0+TY+1
  float* XB = BSM + R * XROWS * NX;                      // 2 x planes, rows y0-1 .. y0+TY
  float2* RY = reinterpret_cast<float2*>(XB + 2 * XBROWS * NX);  // TY/2 odd-row pair sums
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(RY + (TY / 2) * NXC / 2);

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int y0 = blockIdx.x * TY;
  const int k0 = blockIdx.y * zc, k1 = min(k0 + zc, nz);
  const bool down = blockIdx.y & 1;
  const size_t plane = (size_t)NX * ny;
  const int nyc = ny >> 1;
  const float sh = bshift ? (float)(*bshift) : 0.f;
  const bool interior = w >= 1 && w <= TY;
  const int y = y0 - 1 + w;
  const int ypar = y & 1;  // ny is even, so the wrap keeps it
  const int last = k1 - k0 + 3;
  auto mp = [&](int i) { return down ? k1 + 1 - i : k0 - 2 + i; };

  if (tid == 0) {
    for (int s = 0; s < R; ++s) mbar_init(smem_u32(bars + s), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  // box start rows wrapped once; march planes lie in [-2, nz + 1]
  const int ya = wrapm(y0 - 2, ny), yb = wrapm(y0 + TY, ny);
  auto issue = [&](int i) {
    const int s = i % R;
    const unsigned bar = smem_u32(bars + s);
    int z = mp(i);
    z += z < 0 ? nz : (z >= nz ? -nz : 0);
    float* bs = BSM + s * XROWS * NX;
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    mbar_expect_tx(bar, BBYTES);
    tma_load3(smem_u32(bs), &mb_pair, 0, ya, z, bar);
    tma_load3(smem_u32(bs + 2 * NX), &mb_tile, 0, y0, z, bar);
    tma_load3(smem_u32(bs + (TY + 2) * NX), &mb_pair, 0, yb, z, bar);
  };
  auto wait_plane = [&](int i, unsigned limit) {
    return mbar_wait(smem_u32(bars + (i % R)), (unsigned)((i / R) & 1), limit);
  };
  auto brow = [&](int i, int r) { return reinterpret_cast<const float4*>(BSM + (i % R) * XROWS * NX + r * NX); };
  auto xrow = [&](int i, int r) { return reinterpret_cast<float4*>(XB + (i & 1) * XBROWS * NX + r * NX); };

  bool ok = true;
  if (tid == 0) {
    for (int i = 0; i < R && i <= last; ++i) issue(i);
    ok = wait_plane(0, wait_limit) && wait_plane(1, wait_limit) && wait_plane(2, wait_limit);
  }
  int issued = min(R - 1, last);
  ok = !__syncthreads_or(!ok);
  int done = ok ? 2 : -1;

  auto shifted = [&](float4 t) {
    t.x -= sh, t.y -= sh, t.z -= sh, t.w -= sh;
    return t;
  };
  // b - shift of this thread's row: planes i-1, i, i+1 (march order)
  float4 B0[NS], B1[NS], B2[NS];
  // x of this thread's row: planes i-2, i-1, i
  float4 X0[NS], X1[NS], X2[NS];
  float2 acc[NS], held[NS];  // restriction sums: plane pair in progress / completed (even rows)
  if (ok) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      B0[s] = shifted(brow(0, w + 1)[lane + 32 * s]);
      B1[s] = shifted(brow(1, w + 1)[lane + 32 * s]);
    }
  }
  __syncthreads();  // step 1 refills plane 0's slot
  bool pending = false;  // an even row holds a completed pair to combine

  // x on march plane i from b' of planes i-1 (bm), i (b0), i+1 (bp) of this
  // row and rows y -/+ 1 of plane i (shared memory): red cells b'/diag, black
  // cells (b' + off * sum of the red neighbours' b'/diag) / diag.
  auto form_x = [&](float4 (&xo)[NS], const float4 (&bm)[NS], const float4 (&b0)[NS], const float4 (&bp)[NS],
                    int i, int a) {
    const float4* u = brow(i, w) + lane;
    const float4* dn = brow(i, w + 2) + lane;
    float tl[NS], tr[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      tl[s] = __shfl_sync(0xffffffffu, b0[s].w, (lane + 31) & 31);
      tr[s] = __shfl_sync(0xffffffffu, b0[s].x, (lane + 1) & 31);
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const float L = (lane == 0 ? tl[(s + NS - 1) % NS] : tl[s]) * inv;
      const float Rr = (lane == 31 ? tr[(s + 1) % NS] : tr[s]) * inv;
      const float4 uu = shifted(u[32 * s]), dd = shifted(dn[32 * s]);
      const float c0 = b0[s].x * inv, c1 = b0[s].y * inv, c2 = b0[s].z * inv, c3 = b0[s].w * inv;
      auto blk = [&](float bv, float l, float r, float uv, float dv, float zm, float zp) {
        return (bv + off * (((l + r) + (uv * inv + dv * inv)) + (zm * inv + zp * inv))) * inv;
      };
      float4 o;
      if (a == 0) {  // red at e = 0, 2
        o.x = c0;
        o.y = blk(b0[s].y, c0, c2, uu.y, dd.y, bm[s].y, bp[s].y);
        o.z = c2;
        o.w = blk(b0[s].w, c2, Rr, uu.w, dd.w, bm[s].w, bp[s].w);
      } else {  // red at e = 1, 3
        o.x = blk(b0[s].x, L, c1, uu.x, dd.x, bm[s].x, bp[s].x);
        o.y = c1;
        o.z = blk(b0[s].z, c1, c3, uu.z, dd.z, bm[s].z, bp[s].z);
        o.w = c3;
      }
      xo[s] = o;
    }
  };
  // residual b' - A x of this row on march plane i - 1, x-pair sums
  auto resid = [&](float2 (&p)[NS], const float4 (&xm)[NS], const float4 (&x0)[NS], const float4 (&xp)[NS],
                   const float4 (&b0)[NS], int i) {
    const float4* u = xrow(i - 1, w - 1) + lane;
    const float4* dn = xrow(i - 1, w + 1) + lane;
    float tl[NS], tr[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      tl[s] = __shfl_sync(0xffffffffu, x0[s].w, (lane + 31) & 31);
      tr[s] = __shfl_sync(0xffffffffu, x0[s].x, (lane + 1) & 31);
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const float L = lane == 0 ? tl[(s + NS - 1) % NS] : tl[s];
      const float Rr = lane == 31 ? tr[(s + 1) % NS] : tr[s];
      const float4 uu = u[32 * s], dd = dn[32 * s];
      auto r = [&](float bv, float c, float l, float rr, float uv, float dv, float zm, float zp) {
        return bv - (diag * c - off * (((l + rr) + (uv + dv)) + (zm + zp)));
      };
      const float r0 = r(b0[s].x, x0[s].x, L, x0[s].y, uu.x, dd.x, xm[s].x, xp[s].x);
      const float r1 = r(b0[s].y, x0[s].y, x0[s].x, x0[s].z, uu.y, dd.y, xm[s].y, xp[s].y);
      const float r2 = r(b0[s].z, x0[s].z, x0[s].y, x0[s].w, uu.z, dd.z, xm[s].z, xp[s].z);
      const float r3 = r(b0[s].w, x0[s].w, x0[s].z, Rr, uu.w, dd.w, xm[s].w, xp[s].w);
      p[s] = make_float2(r0 + r1, r2 + r3);
    }
  };
  // coarse row of an even fine row y: its held sums plus the odd row's (RY)
  auto combine = [&](int kc) {
    const float2* ry = RY + ((w - 1) >> 1) * (NXC / 2);
    float2* dst = reinterpret_cast<float2*>(bc + ((size_t)kc * nyc + (y >> 1)) * NXC);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const float2 o = ry[lane + 32 * s];
      dst[lane + 32 * s] = make_float2((held[s].x + o.x) * 0.125f, (held[s].y + o.y) * 0.125f);
    }
  };
  int kc_pending = 0;

  // Step i: bm, b0, bp = b' of march planes i-1, i, i+1 (bp is loaded here);
  // xm2, xm1, x0 = x of march planes i-2, i-1, i (x0 is formed here).
  auto step = [&](float4 (&bm)[NS], float4 (&b0)[NS], float4 (&bp)[NS], float4 (&xm2)[NS], float4 (&xm1)[NS],
                  float4 (&x0)[NS], int i) -> bool {
    if (i > last - 1 || !ok) return false;
    if (tid == 0 && i + 3 <= last) issue(i + 3);
    if (i + 3 <= last) issued = i + 3;
    if (pending) {  // the odd row left its sums in RY before the last barrier
      combine(kc_pending);
      pending = false;
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) bp[s] = shifted(brow(i + 1, w + 1)[lane + 32 * s]);
    const int z = mp(i);
    form_x(x0, bm, b0, bp, i, (ypar + z) & 1);
    float4* xr = xrow(i, w);
#pragma unroll
    for (int s = 0; s < NS; ++s) xr[lane + 32 * s] = x0[s];
    if (interior && i >= 3) {
      const int zr = mp(i - 1);  // plane of the residual, in [k0, k1)
      float4* dst = reinterpret_cast<float4*>(xout + (size_t)zr * plane + (size_t)y * NX);
#pragma unroll
      for (int s = 0; s < NS; ++s) dst[lane + 32 * s] = xm1[s];
      float2 pr[NS];
      resid(pr, xm2, xm1, x0, bm, i);
      // march order visits a plane pair (2K, 2K + 1) upwards or downwards
      const bool first = down ? (zr & 1) : !(zr & 1);
#pragma unroll
      for (int s = 0; s < NS; ++s) acc[s] = first ? pr[s] : make_float2(acc[s].x + pr[s].x, acc[s].y + pr[s].y);
      if (!first) {
        if (ypar) {
          float2* ry = RY + ((w - 2) >> 1) * (NXC / 2);
#pragma unroll
          for (int s = 0; s < NS; ++s) ry[lane + 32 * s] = acc[s];
        } else {
#pragma unroll
          for (int s = 0; s < NS; ++s) held[s] = acc[s];
          pending = true;
          kc_pending = zr >> 1;
        }
      }
    }
    bool good = true;
    if (tid == 0 && i + 2 <= last) good = wait_plane(i + 2, wait_limit);
    ok = !__syncthreads_or(!good);
    if (ok) done = i + 2;
    return ok;
  };
  for (int i = 1; i < last; i += 6) {
    if (!step(B0, B1, B2, X0, X1, X2, i)) break;
    if (!step(B1, B2, B0, X1, X2, X0, i + 1)) break;
    if (!step(B2, B0, B1, X2, X0, X1, i + 2)) break;
    if (!step(B0, B1, B2, X0, X1, X2, i + 3)) break;
    if (!step(B1, B2, B0, X1, X2, X0, i + 4)) break;
    if (!step(B2, B0, B1, X2, X0, X1, i + 5)) break;
  }
  if (!ok) {
    if (tid == 0) {
      for (int i = done + 1; i <= issued; ++i) wait_plane(i, kDrainLimit);
      atomicOr(err, 1);
    }
    __syncthreads();
    return;
  }
  if (pending) combine(kc_pending);  // the last pair (its RY write preceded the last barrier)
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

template <int NS, bool PRO>
constexpr size_t rows_smem() {
  constexpr int NX = 128 * NS;
  return sizeof(float) * (size_t)NX *
             (kRowsRing * (kRowsTY + 4) + kRowsRing * (kRowsTY + 2) + (kRowsTY + 2) +
              (PRO ? kCoarseRing * (kRowsTY / 2 + 4) / 2 : 0)) +
         8 * kRowsRing;
}
// two CTAs per SM (228 KB of shared memory, 1 KB reserved per CTA)
static_assert(2 * (rows_smem<2, true>() + 1024) <= 228 * 1024, "two CTAs per SM");

template <int NS, bool PRO>
void rows_launch(dim3 g, cudaStream_t s, const CUtensorMap (&m)[6], float* xout, const double* bshift, Dims d,
                 int zc, float inv, float off, double* part, int* err, unsigned limit) {
  constexpr size_t sm = rows_smem<NS, PRO>();
  static std::atomic<unsigned long long> attr{0};
  ensure_smem_attr((const void*)k_rbgs_rows<NS, PRO>, (int)sm, attr);
  k_rbgs_rows<NS, PRO><<<g, (kRowsTY + 2) * 32, sm, s>>>(m[0], m[1], m[2], m[3], m[4], m[5], xout, bshift, d.ny,
                                                          d.nz, zc, inv, off, part, err, limit);
}

// The row sweep of xin into xout; with xc non-null, of xin + P xc (the fused
// prolongation, zc even).
int rows_sweep_any(const float* xin, const float* xc, float* xout, const float* b, const double* bshift, Dims d,
                   Stencil st, int zc, double* part, int part_cap, cudaStream_t s) {
  const Dims dc{d.nx / 2, d.ny / 2, d.nz / 2};
  const CUtensorMap mx = field_map(xin, d, kRowsTY), mx2 = field_map(xin, d, 2);
  const CUtensorMap m[6] = {mx, mx2, field_map(b, d, kRowsTY), field_map(b, d, 1),
                            xc ? field_map(xc, dc, kRowsTY / 2) : mx, xc ? field_map(xc, dc, 2) : mx2};
  dim3 g(d.ny / kRowsTY, (d.nz + zc - 1) / zc);
  const int nblk = (int)(g.x * g.y);
  if (nblk > part_cap) part = nullptr;
  const float inv = (float)(1.0 / st.diag), off = (float)st.off;
  int* err = wait_error_flag();
  const unsigned limit = wait_limit();
  if (d.nx == 256) {
    if (xc)
      rows_launch<2, true>(g, s, m, xout, bshift, d, zc, inv, off, part, err, limit);
    else
      rows_launch<2, false>(g, s, m, xout, bshift, d, zc, inv, off, part, err, limit);
  } else {
    if (xc)
      rows_launch<1, true>(g, s, m, xout, bshift, d, zc, inv, off, part, err, limit);
    else
      rows_launch<1, false>(g, s, m, xout, bshift, d, zc, inv, off, part, err, limit);
  }
  return part ? nblk : 0;
}

}  // namespace

bool rows_sweep_ok(Dims d) {
  return (d.nx == 128 || d.nx == 256) && d.ny % kRowsTY == 0 && d.ny >= kRowsTY && d.nz % 2 == 0 && d.nz >= 4;
}

int rows_sweep_default_zc(Dims d) {
  // about one wave of two resident CTAs per SM; an even number of planes, as
  // the sweep with the prolongation fused needs, so that both kernels split
  // a level into the same CTAs (and per-CTA partial sums)
  const int cols = d.ny / kRowsTY;
  int chunks = (2 * 152) / cols;
  chunks = chunks < 1 ? 1 : chunks;
  int zc = (d.nz + chunks - 1) / chunks;
  zc += zc & 1;
  return zc < 2 ? 2 : zc;
}

int launch_rows_sweep(const float* xin, float* xout, const float* b, const double* bshift, Dims d, Stencil st,
                      int zc, double* part, int part_cap, cudaStream_t s) {
  if (!rows_sweep_ok(d) || !aligned16(xin) || !aligned16(xout) || !aligned16(b) || xin == xout || b == xout)
    throw CudaError{cudaErrorInvalidValue, "row sweep arguments"};
  zc = zc < 2 ? 2 : (zc > d.nz ? d.nz : zc);
  return rows_sweep_any(xin, nullptr, xout, b, bshift, d, st, zc, part, part_cap, s);
}

int launch_rows_prolong_sweep(const float* xc, const float* xin, float* xout, const float* b, const double* bshift,
                              Dims d, Stencil st, int zc, double* part, int part_cap, cudaStream_t s) {
  if (!rows_sweep_ok(d) || !aligned16(xin) || !aligned16(xout) || !aligned16(b) || !aligned16(xc) || xin == xout ||
      b == xout || xc == xout)
    throw CudaError{cudaErrorInvalidValue, "prolongation + row sweep arguments"};
  zc = zc < 2 ? 2 : (zc > d.nz ? d.nz : zc);
  zc += zc & 1;  // even chunks: fine planes 2K - 1, 2K share their coarse pair in both march directions
  return rows_sweep_any(xin, xc, xout, b, bshift, d, st, zc, part, part_cap, s);
}


bool zero_restrict_rows_ok(Dims d) { return rows_sweep_ok(d); }

int zero_restrict_rows_default_zc(Dims d) {
  return rows_sweep_default_zc(d);  // even: plane pairs of the restriction stay inside a chunk
}

void launch_zero_restrict_rows(const float* b, const double* bshift, float* x, float* bc, Dims d, Stencil st,
                               int zc, cudaStream_t s) {
  if (!zero_restrict_rows_ok(d) || !aligned16(b) || !aligned16(x) || ((uintptr_t)bc & 7u) || b == x)
    throw CudaError{cudaErrorInvalidValue, "fused zero sweep + restriction arguments"};
  zc = zc < 2 ? 2 : (zc > d.nz ? d.nz : zc);
  zc += zc & 1;
  const CUtensorMap mt = field_map(b, d, kRowsTY), mpair = field_map(b, d, 2);
  dim3 g(d.ny / kRowsTY, (d.nz + zc - 1) / zc);
  const float inv = (float)(1.0 / st.diag), off = (float)st.off, diag = (float)st.diag;
  int* err = wait_error_flag();
  const unsigned limit = wait_limit();
  auto go = [&](auto kern, int ns) {
    const size_t sm = sizeof(float) * (size_t)(128 * ns) *
                          (kRowsRing * (kRowsTY + 4) + 2 * (kRowsTY + 2) + kRowsTY / 2 / 2) +
                      8 * kRowsRing;
    static std::atomic<unsigned long long> attr1{0}, attr2{0};
    ensure_smem_attr((const void*)kern, (int)sm, ns == 2 ? attr2 : attr1);
    kern<<<g, (kRowsTY + 2) * 32, sm, s>>>(mt, mpair, x, bc, bshift, d.ny, d.nz, zc, inv, off, diag, err, limit);
  };
  if (d.nx == 256)
    go(k_zr_rows<2>, 2);
  else
    go(k_zr_rows<1>, 1);
}

}  // namespace ibrd
