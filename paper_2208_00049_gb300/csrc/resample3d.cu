// 3D resampling kernels for m = 4 (8 taps per dimension), complex64.
//
// Same computation as the generic kernels in resample.cuh (Eq. SumOverNode,
// Eq. SumOverNodeAdjoint, Eq. InnerTensorStructure; Algorithm 3 / 4), laid
// out for the GB300 shared-memory pipe:
//
//  * tile + halo (T + 7 cells per dimension) in shared memory with a row pitch
//    of 18 complex: rows r and r + 4 are 4 * 18 * 2 = 144 = 16 (mod 32) banks
//    apart, so a half-warp reading 8 consecutive complex from each of the two
//    rows touches 32 distinct banks whatever the node's position;
//  * window values from the paper's POLYNOMIAL precomputation (Sec. 3.7.4,
//    item 5): per tap a degree-8 polynomial in zeta = t - 1/2, coefficients
//    built in FP64 on the device at plan time and held in registers here, so
//    one tap weight is 9 FMAs;
//  * complex x real products on packed FP32 pairs (fma.rn.f32x2);
//  * gather: a half-warp per node (a warp instruction serves two nodes);
//    lane (g, i2) of a half owns taps (i1 = j + 4g, i2), j = 0..3, and loops
//    over i0, then the half reduces its 16 partial sums (reduce-scatter:
//    one exchange splits real and imaginary parts between the two 8-lane
//    groups, three more sum each part, 4 shuffles instead of 8); the node
//    record is read with one 16-byte broadcast load and the w0 / w1 values
//    are handed out through a per-warp shared slot (three 16-byte broadcast
//    loads instead of twelve shuffles), since the shared-memory pipe, which
//    also carries the shuffles, is the binding resource;
//  * scatter (default): the region is accumulated in registers, see the
//    register-accumulating scatter below;
//  * scatter (shared-memory form): W warps (default 2, measured best of
//    1/2/4/8) share one accumulator tile, warp w updating only the planes i0
//    with (a0 + i0) = w (mod W), so no two warps touch the same element and
//    the read-modify-writes need no atomics; the tile (block plus halo) is
//    then added to the grid with vector global reductions;
//  * the node records of a work item are staged in shared memory with the tile;
//  * gather and node gradient: a region that lies inside the grid (no
//    periodic wrap; about 81 % of the items at 256^3 with 9 x 9 x 8 tiles)
//    is copied by the tensor memory accelerator, one 3D box of 18 x L1 x L0
//    points (cp.async.bulk.tensor, completion on a shared mbarrier) that
//    lands directly in the padded row layout; a region that wraps, or a tile
//    with odd T2 (whose rows start on odd points, not on the 16-byte
//    boundary the copy needs), is copied with 16-byte / 8-byte cp.async.
//    The mbarrier wait is bounded: a CTA whose copy does not arrive sets a
//    device flag that nfft_plan_sync reports as NFFT_ERR_TIMEOUT, and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdlib.h>
#include <string.h>

#include "nfft_internal.cuh"
#include "packed_f32x2.cuh"

namespace nfftgb {
namespace {

constexpr int kTaps = 8;
constexpr int kDeg = 8;             // polynomial degree 2m
constexpr int kCoef = kDeg + 1;
constexpr int kPitch = 18;          // shared row pitch (complex) along dim 2
constexpr int kMaxTile2 = 9;        // L2 = T2 + 7 <= 16: two rows per warp step
constexpr int kItemCap = 128;       // nodes per work item staged in shared memory
constexpr int kGatherSlot = 32;     // floats of window slot per gather warp
constexpr int kGatherMaxWarps = 8;
constexpr int kGatherTail = kGatherMaxWarps * kGatherSlot * 4 + 16;  // window slots + mbarrier (bytes)
// Bound on the wait for one region copy: 0.5 s of the global timer (a copy
// of 37 KB takes microseconds), and an iteration cap behind it.
constexpr unsigned long long kWaitNs = 500000000ull;
constexpr int kWaitSpinCap = 1 << 28;

// Set by a CTA whose bounded wait for a region copy gave up (read and
// cleared by fast3d_take_wait_timeout).
__device__ int g_wait_timeout;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Polls the mbarrier until the phase completes or kWaitNs have passed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (int i = 0; i < kWaitSpinCap; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63) == 63 && global_ns() - t0 > kWaitNs) return false;
  }
  return false;
}

// One 3D box of the grid's tensor map into shared memory (x the contiguous
// coordinate, in points; x * 8 bytes must be a multiple of 16).
__device__ __forceinline__ void tma_load_box(void* dst, const CUtensorMap* map, int x, int y, int z,
                                             uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// Bulk tensor reduction (add, element type of the map) of a shared-memory
// box into global memory; completion tracked by the issuing thread's bulk
// async-group.
__device__ __forceinline__ void tma_reduce_add_box(const CUtensorMap* map, const void* src, int x, int y, int z) {
  asm volatile(
      "cp.reduce.async.bulk.tensor.3d.global.shared::cta.add.tile.bulk_group"
      " [%0, {%1, %2, %3}], [%4];" ::"l"(reinterpret_cast<uint64_t>(map)),
      "r"(x), "r"(y), "r"(z), "r"(smem_u32(src))
      : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// The issuing thread's bulk operations have finished reading shared memory.
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// ... and are complete.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// One staged node = 8 words {t0, t1, t2, a0 | a1 << 8 | a2 << 16, perm, re v, im v, 0}
// (fractions, cell offsets in the tile, caller index, scatter input).  A warp
// reads a node with one 32-bit load per lane (lane & 7 -> word) and hands the
// words out with shuffles: one shared wavefront per node instead of one per
// field and quarter-warp.
constexpr int kRecWords = 8;
struct NodeStage {
  float w[kItemCap][kRecWords];
};

__device__ __forceinline__ int wrap1(int x, int n) {
  // region coordinates lie in [-n, 2n) when tile_d <= N~_d - 7 (checked on the host)
  return x < 0 ? x + n : (x >= n ? x - n : x);
}

__device__ __forceinline__ void tile_origin(const Geometry& g, int tile, int* tc) {
  tc[2] = tile % g.ntile[2];
  tile /= g.ntile[2];
  tc[1] = tile % g.ntile[1];
  tc[0] = tile / g.ntile[1];
}

__device__ __forceinline__ void load_coef(const float* poly, int d, int i, float* c) {
#pragma unroll
  for (int z = 0; z < kCoef; ++z) c[z] = poly[(d * kTaps + i) * kCoef + z];
}

__device__ __forceinline__ float horner(const float* c, float zeta) {
  float p = c[kDeg];
#pragma unroll
  for (int z = kDeg - 1; z >= 0; --z) p = fmaf(p, zeta, c[z]);
  return p;
}

// Stage the node records of one work item (CTA-wide).
__device__ __forceinline__ void stage_nodes(const Geometry& g, const NodeArrays& na, const int4& item,
                                            const int* tc, NodeStage& ns, const float2* fhat,
                                            int tid, int nthreads) {
  const int64_t M = g.M;
  const float* frac = reinterpret_cast<const float*>(na.frac);
  for (int i = tid; i < item.z; i += nthreads) {
    const int q = item.y + i;
    int pk = 0;
    float t[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      pk |= (na.cell[d * M + q] - tc[d] * g.T[d]) << (8 * d);
      t[d] = frac[d * M + q];
    }
    const int j = na.perm[q];
    const float2 v = fhat ? fhat[j] : make_float2(0.f, 0.f);
    float4* dst = reinterpret_cast<float4*>(ns.w[i]);
    dst[0] = make_float4(t[0], t[1], t[2], __int_as_float(pk));
    dst[1] = make_float4(__int_as_float(j), v.x, v.y, 0.f);
  }
}

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}

// Tile + halo into shared memory with cp.async (the caller waits with
// cp_async_wait_all before its barrier).  Shared row r holds the 18 grid
// points starting at start[2] - shift:
//  * shift = 1 (T2 even): start[2] - 1 = tc2 T2 - 4 is even, so each row is 9
//    aligned 16-byte chunks; N~ is even, so a chunk never straddles the
//    periodic wrap and wraps as a whole.  Three rows per warp step.
//  * shift = 0 (T2 odd): 8-byte copies of the L2 region points, two rows per
//    warp step.
__device__ __forceinline__ void load_tile(const Geometry& g, const int* start, const float2* grid,
                                          float2* tile, int warp, int lane, int nwarps, int shift) {
  const int L1 = g.L[1];
  const int rows = g.L[0] * L1;
  if (shift) {
    const int ro = lane / 9, q = lane - 9 * ro;
    if (ro < 3) {
      const int x = wrap1(start[2] - 1 + 2 * q, g.Nt[2]);
      for (int r = 3 * warp + ro; r < rows; r += 3 * nwarps) {
        const int r0 = r / L1, r1 = r - r0 * L1;
        const int g0 = wrap1(start[0] + r0, g.Nt[0]);
        const int g1 = wrap1(start[1] + r1, g.Nt[1]);
        cp_async16(tile + (r0 * L1 + r1) * kPitch + 2 * q, grid + ((int64_t)g0 * g.Nt[1] + g1) * g.Nt[2] + x);
      }
    }
  } else {
    const int half = lane >> 4, e = lane & 15;
    if (e < g.L[2]) {
      const int x = wrap1(start[2] + e, g.Nt[2]);
      for (int r = 2 * warp + half; r < rows; r += 2 * nwarps) {
        const int r0 = r / L1, r1 = r - r0 * L1;
        const int g0 = wrap1(start[0] + r0, g.Nt[0]);
        const int g1 = wrap1(start[1] + r1, g.Nt[1]);
        cp_async8(tile + (r0 * L1 + r1) * kPitch + e, grid + ((int64_t)g0 * g.Nt[1] + g1) * g.Nt[2] + x);
      }
    }
  }
}

// Region of one work item into shared memory (a TMA box where the CTA may
// use one and the region lies inside the grid, cp.async otherwise) and its
// node records staged; ends with a CTA barrier.  Returns false, uniformly
// over the CTA, when the bounded wait for a TMA copy gave up.
__device__ __forceinline__ bool load_region(const Geometry& g, const CUtensorMap* tmap, uint64_t* bar,
                                            unsigned& phase, bool tma_cta, unsigned tx_extra, const int* start,
                                            const float2* grid, float2* tile, int warp, int lane, int nwarps,
                                            int shift, const NodeArrays& na, const int4& item, const int* tc,
                                            NodeStage& ns) {
  const bool by_tma = tma_cta && shift && start[0] >= 0 && start[0] + g.L[0] <= g.Nt[0] && start[1] >= 0 &&
                      start[1] + g.L[1] <= g.Nt[1] && start[2] >= 1 && start[2] - 1 + kPitch <= g.Nt[2];
  if (by_tma) {
    if (threadIdx.x == 0) {
      // the previous item's reads of the tile (generic proxy) are ordered
      // before the copy's writes (async proxy) by the caller's barrier
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive_expect_tx(bar, (unsigned)(g.L[0] * g.L[1] * kPitch * (int)sizeof(float2)) + tx_extra);
      tma_load_box(tile, tmap, start[2] - 1, start[1], start[0], bar);
    }
  } else {
    load_tile(g, start, grid, tile, warp, lane, nwarps, shift);
  }
  stage_nodes(g, na, item, tc, ns, nullptr, threadIdx.x, blockDim.x);
  if (!by_tma) {
    cp_async_wait_all();
    __syncthreads();
    return true;
  }
  const bool done = mbar_wait_bounded(bar, phase);
  phase ^= 1u;
  if (__syncthreads_or(!done)) {
    // Last resort: the CTA returns and the host reads NFFT_ERR_TIMEOUT.  A
    // copy still in flight would land in shared memory the CTA no longer
    // uses; the test hook (tx_extra) makes the wait run out with the copy
    // already complete.
    if (threadIdx.x == 0) atomicExch(&g_wait_timeout, 1);
    return false;
  }
  return true;
}

// ---------------------------------------------------------------------------
template <int GW>
__global__ void __launch_bounds__(32 * GW)
    gather3d_m4_kernel(Geometry g, const float2* __restrict__ grid, NodeArrays na,
                       const float* __restrict__ poly, float2* __restrict__ fhat,
                       const __grid_constant__ CUtensorMap tmap, int tma_on) {
  static_assert(GW <= kGatherMaxWarps, "one window slot per warp");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  NodeStage& ns = *reinterpret_cast<NodeStage*>(smem_raw);
  float2* tile = reinterpret_cast<float2*>(smem_raw + sizeof(NodeStage));
  const int L1 = g.L[1];
  const int plane = L1 * kPitch;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int half = lane >> 4, lane16 = lane & 15;
  const int grp = lane16 >> 3, i2 = lane & 7;
  const int hbase = 16 * half;
  // this warp's window slot (after the tile): [16 half + i] = tap i of
  // dimension 0 (i < 8) or of dimension 1 (tap i - 8) of the half's node
  float* wslot = reinterpret_cast<float*>(tile + g.L[0] * plane) + kGatherSlot * warp;
  uint64_t* bar = reinterpret_cast<uint64_t*>(reinterpret_cast<float*>(tile + g.L[0] * plane) +
                                              kGatherMaxWarps * kGatherSlot);
  const bool tma_cta = (tma_on & 1) && (smem_u32(tile) & 127) == 0;
  const unsigned tx_extra = (unsigned)tma_on >> 8;
  if (tma_cta && threadIdx.x == 0) mbar_init(bar);
  unsigned phase = 0;
  // lane evaluates tap i2 of dimension grp (weights wA) and of dimension 2 (wB)
  float cA[kCoef], cB[kCoef];
  load_coef(poly, grp, i2, cA);
  load_coef(poly, 2, i2, cB);
  const int nitems = *na.n_items;
  const int shift = (g.T[2] & 1) ? 0 : 1;

  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int4 item = na.items[it];
    int tc[3], start[3];
    tile_origin(g, item.x, tc);
#pragma unroll
    for (int d = 0; d < 3; ++d) start[d] = tc[d] * g.T[d] + g.off;

    __syncthreads();
    if (!load_region(g, &tmap, bar, phase, tma_cta, tx_extra, start, grid, tile, warp, lane, GW, shift, na, item, tc, ns))
      return;

    for (int s0 = 2 * warp; s0 < item.z; s0 += 2 * GW) {
      const int s = min(s0 + half, item.z - 1);  // a half without a node repeats the last one
      const float4 rec = *reinterpret_cast<const float4*>(ns.w[s]);  // t0, t1, t2, packed offsets
      const float wA = horner(cA, (grp ? rec.y : rec.x) - 0.5f);
      const float wB = horner(cB, rec.z - 0.5f);
      const int pk = __float_as_int(rec.w);
      const int a0 = pk & 0xff, a1 = (pk >> 8) & 0xff, a2 = pk >> 16;
      __syncwarp();  // the previous node pair's slot reads are done
      wslot[lane] = wA;
      __syncwarp();
      const float4 w0lo = *reinterpret_cast<const float4*>(wslot + hbase);
      const float4 w0hi = *reinterpret_cast<const float4*>(wslot + hbase + 4);
      const float4 w1q = *reinterpret_cast<const float4*>(wslot + hbase + 8 + 4 * grp);
      const float w0v[kTaps] = {w0lo.x, w0lo.y, w0lo.z, w0lo.w, w0hi.x, w0hi.y, w0hi.z, w0hi.w};
      const float w1v[4] = {w1q.x * wB, w1q.y * wB, w1q.z * wB, w1q.w * wB};
      f32x2 w12[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) w12[j] = pack2(w1v[j], w1v[j]);
      const f32x2* p =
          reinterpret_cast<const f32x2*>(tile + (a0 * L1 + a1 + 4 * grp) * kPitch + a2 + i2 + shift);
      f32x2 acc = pack2(0.f, 0.f);
#pragma unroll
      for (int i0 = 0; i0 < kTaps; ++i0) {
        const f32x2* q = p + i0 * plane;
        f32x2 sum = mul2(q[0], w12[0]);
        sum = fma2(q[kPitch], w12[1], sum);
        sum = fma2(q[2 * kPitch], w12[2], sum);
        sum = fma2(q[3 * kPitch], w12[3], sum);
        acc = fma2(sum, pack2(w0v[i0], w0v[i0]), acc);
      }
      // reduce-scatter over the half: group 0 sums the real parts, group 1
      // the imaginary parts; lane16 = 0 ends with the real sum, lane16 = 8
      // with the imaginary sum
      const float2 r = unpack2(acc);
      float v = (grp ? r.y : r.x) + __shfl_xor_sync(0xffffffffu, grp ? r.x : r.y, 8);
      v += __shfl_xor_sync(0xffffffffu, v, 4);
      v += __shfl_xor_sync(0xffffffffu, v, 2);
      v += __shfl_xor_sync(0xffffffffu, v, 1);
      if (i2 == 0 && s0 + half < item.z) {
        const int jout = __float_as_int(ns.w[s][4]);
        reinterpret_cast<float*>(fhat + jout)[grp] = v;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Node gradient for m = 4, complex64 (the derivative of Eq. SumOverNode with
// respect to the node): the gather's tile, half-warp and lane layout, with
// each tap weighted three ways.  For dimension d the window of that
// dimension is replaced by its derivative:
//   D_d = sum_l ghat_l psi'(u_d) prod_{e != d} psi(u_e),
//   gk[j][d] = N~_d Re(conj(cot_j) D_d).
// The POLYNOMIAL window gives value and derivative in one Horner pass
// (d/dk = N~ d/dt, t the fraction of N~ k).
__device__ __forceinline__ float2 horner_d(const float* c, float zeta) {
  float p = c[kDeg], dp = 0.f;
#pragma unroll
  for (int z = kDeg - 1; z >= 0; --z) {
    dp = fmaf(dp, zeta, p);
    p = fmaf(p, zeta, c[z]);
  }
  return make_float2(p, dp);
}

template <int GW>
__global__ void __launch_bounds__(32 * GW)
    grad3d_m4_kernel(Geometry g, const float2* __restrict__ grid, NodeArrays na, const float* __restrict__ poly,
                     const float2* __restrict__ cot, float* __restrict__ gk,
                     const __grid_constant__ CUtensorMap tmap, int tma_on) {
  static_assert(2 * GW <= kGatherMaxWarps, "two window slots per warp");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  NodeStage& ns = *reinterpret_cast<NodeStage*>(smem_raw);
  float2* tile = reinterpret_cast<float2*>(smem_raw + sizeof(NodeStage));
  const int L1 = g.L[1];
  const int plane = L1 * kPitch;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int half = lane >> 4, lane16 = lane & 15;
  const int grp = lane16 >> 3, i2 = lane & 7;
  const int hbase = 16 * half;
  // this warp's window slots (after the tile): values at [16 half + i],
  // derivatives at [32 + 16 half + i] (tap i of dimension 0, tap i - 8 of
  // dimension 1)
  float* wslot = reinterpret_cast<float*>(tile + g.L[0] * plane) + 2 * kGatherSlot * warp;
  uint64_t* bar = reinterpret_cast<uint64_t*>(reinterpret_cast<float*>(tile + g.L[0] * plane) +
                                              kGatherMaxWarps * kGatherSlot);
  const bool tma_cta = (tma_on & 1) && (smem_u32(tile) & 127) == 0;
  const unsigned tx_extra = (unsigned)tma_on >> 8;
  if (tma_cta && threadIdx.x == 0) mbar_init(bar);
  unsigned phase = 0;
  float cA[kCoef], cB[kCoef];
  load_coef(poly, grp, i2, cA);
  load_coef(poly, 2, i2, cB);
  const int nitems = *na.n_items;
  const int shift = (g.T[2] & 1) ? 0 : 1;

  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int4 item = na.items[it];
    int tc[3], start[3];
    tile_origin(g, item.x, tc);
#pragma unroll
    for (int d = 0; d < 3; ++d) start[d] = tc[d] * g.T[d] + g.off;

    __syncthreads();
    if (!load_region(g, &tmap, bar, phase, tma_cta, tx_extra, start, grid, tile, warp, lane, GW, shift, na, item, tc, ns))
      return;

    for (int s0 = 2 * warp; s0 < item.z; s0 += 2 * GW) {
      const int s = min(s0 + half, item.z - 1);  // a half without a node repeats the last one
      const float4 rec = *reinterpret_cast<const float4*>(ns.w[s]);  // t0, t1, t2, packed offsets
      const int jout = __float_as_int(ns.w[s][4]);
      const float2 c = cot[jout];
      const float2 A = horner_d(cA, (grp ? rec.y : rec.x) - 0.5f);  // tap i2 of dimension grp: value, derivative
      const float2 Bw = horner_d(cB, rec.z - 0.5f);                 // tap i2 of dimension 2
      const int pk = __float_as_int(rec.w);
      const int a0 = pk & 0xff, a1 = (pk >> 8) & 0xff, a2 = pk >> 16;
      __syncwarp();  // the previous node pair's slot reads are done
      wslot[lane] = A.x;
      wslot[32 + lane] = A.y;
      __syncwarp();
      const float4 w0lo = *reinterpret_cast<const float4*>(wslot + hbase);
      const float4 w0hi = *reinterpret_cast<const float4*>(wslot + hbase + 4);
      const float4 d0lo = *reinterpret_cast<const float4*>(wslot + 32 + hbase);
      const float4 d0hi = *reinterpret_cast<const float4*>(wslot + 32 + hbase + 4);
      const float4 w1q = *reinterpret_cast<const float4*>(wslot + hbase + 8 + 4 * grp);
      const float4 d1q = *reinterpret_cast<const float4*>(wslot + 32 + hbase + 8 + 4 * grp);
      const float w0v[kTaps] = {w0lo.x, w0lo.y, w0lo.z, w0lo.w, w0hi.x, w0hi.y, w0hi.z, w0hi.w};
      const float dw0v[kTaps] = {d0lo.x, d0lo.y, d0lo.z, d0lo.w, d0hi.x, d0hi.y, d0hi.z, d0hi.w};
      const float w1v[4] = {w1q.x, w1q.y, w1q.z, w1q.w};
      const float dw1v[4] = {d1q.x, d1q.y, d1q.z, d1q.w};
      // rows j + 4 grp: w1 w2, w1' w2, w1 w2'
      f32x2 w12[4], d1[4], d2[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float a = w1v[j] * Bw.x, b = dw1v[j] * Bw.x, e = w1v[j] * Bw.y;
        w12[j] = pack2(a, a);
        d1[j] = pack2(b, b);
        d2[j] = pack2(e, e);
      }
      const f32x2* p =
          reinterpret_cast<const f32x2*>(tile + (a0 * L1 + a1 + 4 * grp) * kPitch + a2 + i2 + shift);
      f32x2 D0 = pack2(0.f, 0.f), D1 = D0, D2 = D0;
#pragma unroll
      for (int i0 = 0; i0 < kTaps; ++i0) {
        const f32x2* q = p + i0 * plane;
        f32x2 s12 = mul2(q[0], w12[0]), s1 = mul2(q[0], d1[0]), s2 = mul2(q[0], d2[0]);
#pragma unroll
        for (int j = 1; j < 4; ++j) {
          const f32x2 v = q[j * kPitch];
          s12 = fma2(v, w12[j], s12);
          s1 = fma2(v, d1[j], s1);
          s2 = fma2(v, d2[j], s2);
        }
        D0 = fma2(s12, pack2(dw0v[i0], dw0v[i0]), D0);
        D1 = fma2(s1, pack2(w0v[i0], w0v[i0]), D1);
        D2 = fma2(s2, pack2(w0v[i0], w0v[i0]), D2);
      }
      // Re(conj(cot) D_d) is linear in D_d: project each lane's partial sums
      // before reducing, three real sums over the half instead of six
      const float2 r0 = unpack2(D0), r1 = unpack2(D1), r2 = unpack2(D2);
      float e0 = c.x * r0.x + c.y * r0.y;
      float e1 = c.x * r1.x + c.y * r1.y;
      float e2 = c.x * r2.x + c.y * r2.y;
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        e0 += __shfl_xor_sync(0xffffffffu, e0, o);
        e1 += __shfl_xor_sync(0xffffffffu, e1, o);
        e2 += __shfl_xor_sync(0xffffffffu, e2, o);
      }
      if (lane16 == 0 && s0 + half < item.z) {
        float* o = gk + (int64_t)jout * 3;
        o[0] = (float)g.Nt[0] * e0;
        o[1] = (float)g.Nt[1] * e1;
        o[2] = (float)g.Nt[2] * e2;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// W warps share one accumulator tile; warp w updates only the planes
// i0 = i0a + j W (j = 0 .. 8/W - 1) with (a0 + i0a) = w (mod W).
template <int W>
__global__ void __launch_bounds__(32 * W)
    scatter3d_m4_kernel(Geometry g, float2* __restrict__ grid, NodeArrays na,
                        const float* __restrict__ poly, const float2* __restrict__ fhat) {
  constexpr int kPlanes = kTaps / W;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  NodeStage& ns = *reinterpret_cast<NodeStage*>(smem_raw);
  float2* acc = reinterpret_cast<float2*>(smem_raw + sizeof(NodeStage));
  const int L0 = g.L[0], L1 = g.L[1], L2 = g.L[2];
  const int plane = L1 * kPitch;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i2 = lane & 7;
  // row map: 8-lane group gq reads rows (gq & 1) * 4 + (gq >> 1) and that + 2
  const int gq = lane >> 3;
  const int ra = (gq & 1) * 4 + (gq >> 1), rb = ra + 2;
  // lanes 0..23 evaluate tap (lane & 7) of dimension lane >> 3
  float c[kCoef];
  const int dl = min(lane >> 3, 2);
  load_coef(poly, dl, i2, c);
  const int nitems = *na.n_items;
  const int n4 = (L0 * plane) / 2;  // float4 count (pitch is even)

  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int4 item = na.items[it];
    int tc[3], start[3];
    tile_origin(g, item.x, tc);
#pragma unroll
    for (int d = 0; d < 3; ++d) start[d] = tc[d] * g.T[d] + g.off;

    __syncthreads();  // previous flush done
    float4* acc4 = reinterpret_cast<float4*>(acc);
    for (int e = threadIdx.x; e < n4; e += blockDim.x) acc4[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    stage_nodes(g, na, item, tc, ns, fhat, threadIdx.x, blockDim.x);
    __syncthreads();

    for (int s = 0; s < item.z; ++s) {
      const float word = ns.w[s][lane & 7];
      const float t = __shfl_sync(0xffffffffu, word, dl);
      const int pk = __float_as_int(__shfl_sync(0xffffffffu, word, 3));
      const float2 v = make_float2(__shfl_sync(0xffffffffu, word, 5), __shfl_sync(0xffffffffu, word, 6));
      const float w = horner(c, t - 0.5f);
      const int a0 = pk & 0xff, a1 = (pk >> 8) & 0xff, a2 = pk >> 16;
      const int i0a = (warp - a0) & (W - 1);  // this warp's planes: i0a + j W
      const float w2 = __shfl_sync(0xffffffffu, w, 16 + i2);
      const float wa = __shfl_sync(0xffffffffu, w, 8 + ra) * w2;
      const float wb = __shfl_sync(0xffffffffu, w, 8 + rb) * w2;
      const f32x2 va = mul2(pack2(v.x, v.y), pack2(wa, wa));
      const f32x2 vb = mul2(pack2(v.x, v.y), pack2(wb, wb));
      f32x2* pa = reinterpret_cast<f32x2*>(acc + ((a0 + i0a) * L1 + a1 + ra) * kPitch + a2 + i2);
      f32x2* pb = pa + 2 * kPitch;
      f32x2 ta[kPlanes], tb[kPlanes];
#pragma unroll
      for (int j = 0; j < kPlanes; ++j) {
        ta[j] = pa[j * W * plane];
        tb[j] = pb[j * W * plane];
      }
#pragma unroll
      for (int j = 0; j < kPlanes; ++j) {
        const float w0 = __shfl_sync(0xffffffffu, w, i0a + j * W);
        const f32x2 ww0 = pack2(w0, w0);
        pa[j * W * plane] = fma2(va, ww0, ta[j]);
        pb[j * W * plane] = fma2(vb, ww0, tb[j]);
      }
      __syncwarp();
    }
    __syncthreads();

    // add block + halo back to the grid (periodic wrap only here)
    {
      const int half = lane >> 4, e = lane & 15;
      const int rows = L0 * L1;
      const int g2 = wrap1(start[2] + e, g.Nt[2]);
      for (int r = 2 * warp + half; r < rows; r += 2 * W) {
        const int r0 = r / L1, r1 = r - r0 * L1;
        if (e < L2) {
          const float2 val = acc[(r0 * L1 + r1) * kPitch + e];
          const int g0 = wrap1(start[0] + r0, g.Nt[0]);
          const int g1 = wrap1(start[1] + r1, g.Nt[1]);
          atomicAdd(grid + ((int64_t)g0 * g.Nt[1] + g1) * g.Nt[2] + g2, val);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Gather for m = 6 (K = 12 taps per dimension), complex64: the tile + halo
// (L_d = T_d + 11 <= 16 per dimension) in shared memory, one node per
// half-warp.  Per (i0) plane the node's 12 x 12 (i1, i2) taps are flattened,
// f = 12 i1 + i2, and lane l of the half takes f = 16 k + l, k = 0..8: every
// lane carries a tap (with one lane per i2 and a row of 12 taps, a quarter of
// the lanes idled), each lane's w1[i1] w2[i2] products are formed once per
// node, and the row pitch makes the 16 taps of one load conflict-free.  The
// 36 window values of every node are evaluated once per work item
// (POLYNOMIAL form, packed Horner, two taps per lane) into shared memory.
constexpr int kG12Taps = 12;
constexpr int kG12Warps = 8;
constexpr int kG12Threads = 32 * kG12Warps;
// Row pitch of the region copy: 28 complex = 12 bank pairs mod 16, so that
// tap (i1, i2) of a plane lies on bank pair (base + 12 i1 + i2) mod 16 and
// the 16 consecutive flattened taps f = 12 i1 + i2 a half-warp reads at once
// fall on 16 distinct bank pairs.
constexpr int kG12Pitch = 28;
constexpr int kG12Steps = kG12Taps * kG12Taps / 16;  // flattened (i1, i2) taps per lane and plane

struct G12Weights {
  float w0s[kItemCap][kG12Taps];
  float w1s[kItemCap][kG12Taps];
  float w2[kItemCap][16];
  f32x2 coef[3][kG12Taps / 2][kG12Taps + 1];
};

__device__ __forceinline__ size_t g12_tile_offset() { return sizeof(NodeStage) + sizeof(G12Weights); }

__global__ void __launch_bounds__(kG12Threads, 2)
    gather3d_k12_kernel(Geometry g, const float2* __restrict__ grid, NodeArrays na,
                        const float* __restrict__ poly, float2* __restrict__ fhat) {
  constexpr int K = kG12Taps, P = K / 2, kPerIter = 32 / P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  NodeStage& ns = *reinterpret_cast<NodeStage*>(smem_raw);
  G12Weights& wt = *reinterpret_cast<G12Weights*>(smem_raw + sizeof(NodeStage));
  float2* tile = reinterpret_cast<float2*>(smem_raw + g12_tile_offset());
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int half = lane >> 4, l16 = lane & 15;
  const int L1 = g.L[1], L2 = g.L[2];
  const int pitch = kG12Pitch, plane = L1 * pitch;
  // lane l16 takes the flattened taps f = 16 k + l16 of every (i0) plane:
  // (i1, i2) = (f / 12, f mod 12)
  int toff[kG12Steps], ti1[kG12Steps], ti2[kG12Steps];
#pragma unroll
  for (int k = 0; k < kG12Steps; ++k) {
    const int f = 16 * k + l16;
    ti1[k] = f / K;
    ti2[k] = f - K * ti1[k];
    toff[k] = ti1[k] * pitch + ti2[k];
  }
  // weight lanes: (wj, tp) = two taps of every dimension of node kPerIter (warp + it W) + wj
  const int wj = lane / P, tp = lane - P * (lane / P);
  for (int e = tid; e < 3 * P * (K + 1); e += kG12Threads) {
    const int d = e / (P * (K + 1)), pp = (e / (K + 1)) % P, z = e % (K + 1);
    wt.coef[d][pp][z] = pack2(poly[(d * K + 2 * pp) * (K + 1) + z], poly[(d * K + 2 * pp + 1) * (K + 1) + z]);
  }
  const int nitems = *na.n_items;

  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int4 item = na.items[it];
    int tc[3], start[3];
    tile_origin(g, item.x, tc);
#pragma unroll
    for (int d = 0; d < 3; ++d) start[d] = tc[d] * g.T[d] + g.off;
    const int count = item.z;

    __syncthreads();  // previous item's tile, records and weights no longer read
    {
      const int rows = g.L[0] * L1;
      for (int e = tid; e < rows * L2; e += kG12Threads) {
        const int r = e / L2, c = e - r * L2;
        const int r0 = r / L1, r1 = r - r0 * L1;
        const int g0 = wrap1(start[0] + r0, g.Nt[0]);
        const int g1 = wrap1(start[1] + r1, g.Nt[1]);
        const int g2 = wrap1(start[2] + c, g.Nt[2]);
        cp_async8(tile + r * pitch + c, grid + ((int64_t)g0 * g.Nt[1] + g1) * g.Nt[2] + g2);
      }
    }
    stage_nodes(g, na, item, tc, ns, nullptr, tid, kG12Threads);
    __syncthreads();  // records visible (the tile copies are waited for below)
    if (wj < kPerIter) {
#pragma unroll
      for (int d = 0; d < 3; ++d) {  // one dimension's coefficients in registers at a time
        f32x2 cpair[K + 1];
#pragma unroll
        for (int e = 0; e <= K; ++e) cpair[e] = wt.coef[d][tp][e];
        for (int s = kPerIter * warp + wj; s < count; s += kPerIter * kG12Warps) {
          const float z = ns.w[s][d] - 0.5f;
          const f32x2 zz = pack2(z, z);
          f32x2 pw = cpair[K];
#pragma unroll
          for (int e = K - 1; e >= 0; --e) pw = fma2(pw, zz, cpair[e]);
          const float2 w = unpack2(pw);  // taps 2 tp, 2 tp + 1
          if (d == 0) {
            *reinterpret_cast<float2*>(&wt.w0s[s][2 * tp]) = w;
          } else if (d == 1) {
            *reinterpret_cast<float2*>(&wt.w1s[s][2 * tp]) = w;
          } else {
            *reinterpret_cast<float2*>(&wt.w2[s][2 * tp]) = w;
            if (tp == 0) *reinterpret_cast<float4*>(&wt.w2[s][K]) = make_float4(0.f, 0.f, 0.f, 0.f);
          }
        }
      }
    }
    cp_async_wait_all();
    __syncthreads();

    for (int s0 = 2 * warp; s0 < count; s0 += 2 * kG12Warps) {
      const int s = min(s0 + half, count - 1);  // a half without a node repeats the last one
      const int pk = __float_as_int(ns.w[s][3]);
      const int a0 = pk & 0xff, a1 = (pk >> 8) & 0xff, a2 = pk >> 16;
      const f32x2* col = reinterpret_cast<const f32x2*>(tile + (a0 * L1 + a1) * pitch + a2);
      f32x2 w12[kG12Steps];  // w1[i1] w2[i2] of this lane's flattened taps
#pragma unroll
      for (int k = 0; k < kG12Steps; ++k) {
        const float w = wt.w1s[s][ti1[k]] * wt.w2[s][ti2[k]];
        w12[k] = pack2(w, w);
      }
      const float4* w0q = reinterpret_cast<const float4*>(&wt.w0s[s][0]);
      f32x2 acc = pack2(0.f, 0.f);
#pragma unroll
      for (int q = 0; q < K / 4; ++q) {
        const float4 x = w0q[q];
        const float xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          const f32x2* pl = col + (4 * q + h) * plane;
          f32x2 sum = mul2(pl[toff[0]], w12[0]);
#pragma unroll
          for (int k = 1; k < kG12Steps; ++k) sum = fma2(pl[toff[k]], w12[k], sum);
          acc = fma2(sum, pack2(xs[h], xs[h]), acc);
        }
      }
      float2 r = unpack2(acc);
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        r.x += __shfl_xor_sync(0xffffffffu, r.x, o);
        r.y += __shfl_xor_sync(0xffffffffu, r.y, o);
      }
      if (l16 == 0 && s0 + half < count) fhat[__float_as_int(ns.w[s][4])] = r;
    }
  }
}

size_t g12_smem_bytes(const Geometry& g) {
  return sizeof(NodeStage) + sizeof(G12Weights) + (size_t)g.L[0] * g.L[1] * kG12Pitch * sizeof(float2);
}

bool g12_supported(const Geometry& g, int cmax) {
  if (g.D != 3 || g.K != kG12Taps || g.closed || g.off != -5 || g.m != 6.0 || cmax > kItemCap) return false;
  for (int d = 0; d < 3; ++d)
    if (g.L[d] > 16 || g.T[d] > g.Nt[d] - kG12Taps + 1) return false;
  return g12_smem_bytes(g) <= 200 * 1024;
}

// ---------------------------------------------------------------------------
// Register-accumulating scatter, K = 2m taps per dimension (m = 4 and 6).
// Thread (r1, cc) of a 128-thread CTA owns the two region lines (., r1, cc)
// and (., r1, cc + 8) of the tile + halo in registers (acc[h][r0],
// r0 < L0 <= 16): a node at offset (a0, a1, a2) adds
//   v w1[r1 - a1] w2[c - a2] * w0[i0]   to acc[h][a0 + i0],  i0 = 0..K-1,
// c = cc + 8 h, so the accumulation costs 2K packed FMAs per thread and node
// and no shared-memory traffic.  Register indices must be static, so the
// nodes of a work item are counting-sorted by (a0, a1): each a0 bin runs a
// loop specialised to its a0, and a warp, which owns rows 4w .. 4w + 3,
// visits only the contiguous run of nodes whose a1 puts one of its rows in
// the footprint.  Tiles are at most 17 - K cells per dimension (regions of
// at most 16).  Per work item:
//  1. stage the node records and count them per (a0, a1) key;
//  2. scan the counts (one warp);
//  3. evaluate the 3K window values of every node once (POLYNOMIAL form; a
//     lane takes two taps of all three dimensions with packed Horner steps)
//     and store, at the node's sorted slot and shifted to region
//     coordinates: w0, v w1 per row, and w2 per thread column pair (zero
//     outside the footprint).  Stored once and paired in registers (a move
//     per value), w0 and w2 cost half the shared wavefronts of stored
//     (w, w) pairs: the main loop issues 2 + K/4 shared loads per thread
//     and node;
//  4. every warp runs over its node runs;
//  5. the region is added to the grid: a region inside the grid is written
//     to shared memory (over the weight arrays, which are done with) as a
//     box 18 points wide and added by one bulk tensor reduction
//     (cp.reduce.async.bulk.tensor, add, FP32) issued by one thread, whose
//     read of shared memory is waited for only before the next item's
//     weights are written; a region that wraps at a grid face is added with
//     vector global reductions.
constexpr int kRegAccLines = 16;                   // acc[h][r0], L0 <= 16
constexpr int kFlushPitch = 18;                    // points per box row (x0 even, region at x0 + lead)
constexpr int kRegAccThreads = 128;                // 16 rows r1 x 8 column pairs
constexpr int kRegAccWarps = kRegAccThreads / 32;  // warp w owns rows 4w .. 4w + 3
constexpr int kRegAccA = 9;                        // a_d < T_d <= 9
constexpr int kRegAccKeys = kRegAccA * kRegAccA;   // (a0, a1)

template <int K>
struct RegAccStage {
  static constexpr int kPairs = K / 2;   // tap pairs per dimension
  static constexpr int kWeightBytes = kItemCap * (K * 4 + kRegAccLines * 8 + 8 * 8);
  static constexpr int kBoxBytes = kRegAccLines * kRegAccLines * kFlushPitch * 8;
  float4 rec[kItemCap][2];               // {t0, t1, t2, pk}, {re v, im v, key, rank}
  int count[kRegAccKeys];
  int start[kRegAccKeys + 1];
  f32x2 coef[3][kPairs][K + 1];          // (tap 2 tp, tap 2 tp + 1) coefficient pairs, degree K
  // the weights of the current item; the flush box overlays them
  alignas(128) float w0s[kItemCap][K];   // w0, by slot
  f32x2 vw1[kItemCap][kRegAccLines];     // v w1[r - a1], by slot
  float2 w2s[kItemCap][8];               // cc -> (w2[cc - a2], w2[cc + 8 - a2]), by slot
  unsigned char pad[kBoxBytes > kWeightBytes ? kBoxBytes - kWeightBytes : 16];
  __device__ float2* box() { return reinterpret_cast<float2*>(&w0s[0][0]); }
};

// Compensation terms of the accumulators (COMP: one per accumulator; else
// one unused register pair).
template <bool COMP>
struct RegAccComp {
  f32x2 c[COMP ? 2 : 1][COMP ? kRegAccLines : 1];
};

template <int A0, int K, bool COMP>
__device__ __forceinline__ void regacc_node(const RegAccStage<K>& st, int s, int r1, int cc,
                                            f32x2 (&acc)[2][kRegAccLines], RegAccComp<COMP>& cp) {
  const f32x2 vw = st.vw1[s][r1];
  const float2 w2 = st.w2s[s][cc];
  const f32x2 vp0 = mul2(vw, pack2(w2.x, w2.x));
  const f32x2 vp1 = mul2(vw, pack2(w2.y, w2.y));
  const float4* wq = reinterpret_cast<const float4*>(&st.w0s[s][0]);
#pragma unroll
  for (int q = 0; q < K / 4; ++q) {
    const float4 x = wq[q];
    const float xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const f32x2 wa = pack2(xs[j], xs[j]);
      if constexpr (COMP) {
        two_sum_acc2(acc[0][A0 + 4 * q + j], cp.c[0][A0 + 4 * q + j], mul2(vp0, wa));
        two_sum_acc2(acc[1][A0 + 4 * q + j], cp.c[1][A0 + 4 * q + j], mul2(vp1, wa));
      } else {
        acc[0][A0 + 4 * q + j] = fma2(vp0, wa, acc[0][A0 + 4 * q + j]);
        acc[1][A0 + 4 * q + j] = fma2(vp1, wa, acc[1][A0 + 4 * q + j]);
      }
    }
  }
}

template <int A0, int K, bool COMP>
__device__ __forceinline__ void regacc_bin(const RegAccStage<K>& st, int lo, int hi, int r1, int cc,
                                           f32x2 (&acc)[2][kRegAccLines], RegAccComp<COMP>& cp) {
  if constexpr (A0 + K <= kRegAccLines) {  // a0 < T0 <= 17 - K
    const int s0 = st.start[A0 * kRegAccA + lo], s1 = st.start[A0 * kRegAccA + hi + 1];
    int s = s0;
    for (; s + 1 < s1; s += 2) {
      regacc_node<A0, K, COMP>(st, s, r1, cc, acc, cp);
      regacc_node<A0, K, COMP>(st, s + 1, r1, cc, acc, cp);
    }
    if (s < s1) regacc_node<A0, K, COMP>(st, s, r1, cc, acc, cp);
  }
}

// COMP (NFFT_FLAG_COMPENSATED): every accumulator carries the running sum of
// the rounding errors of its additions (TwoSum), added back at the flush;
// twice the accumulator registers, so two CTAs per SM instead of four.
template <int K, bool COMP>
__global__ void __launch_bounds__(kRegAccThreads, COMP ? 2 : 4)
    scatter3d_regacc_kernel(Geometry g, float2* __restrict__ grid, NodeArrays na,
                            const float* __restrict__ poly, const float2* __restrict__ fhat,
                            const __grid_constant__ CUtensorMap rmap, int tma_on) {
  using Stage = RegAccStage<K>;
  constexpr int P = Stage::kPairs;
  constexpr int kPerIter = 32 / P;  // nodes per warp and weight iteration
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Stage& st = *reinterpret_cast<Stage*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r1 = tid >> 3, cc = tid & 7;
  // a1 run of this warp: one of rows 4w .. 4w + 3 lies in [a1, a1 + K)
  const int lo = max(0, 4 * warp - (K - 1)), hi = min(kRegAccA - 1, 4 * warp + 3);
  // weight evaluation: lane (wj, tp) takes taps 2 tp, 2 tp + 1 of every
  // dimension for nodes kPerIter (warp + 4 it) + wj; coefficients as packed
  // pairs, kept in shared memory between items
  const int wj = lane / P, tp = lane - P * (lane / P);
  for (int e = tid; e < 3 * P * (K + 1); e += kRegAccThreads) {
    const int d = e / (P * (K + 1)), pp = (e / (K + 1)) % P, z = e % (K + 1);
    st.coef[d][pp][z] = pack2(poly[(d * K + 2 * pp) * (K + 1) + z], poly[(d * K + 2 * pp + 1) * (K + 1) + z]);
  }
  const int nitems = *na.n_items;
  const int L0 = g.L[0], L1 = g.L[1], L2 = g.L[2];
  const int64_t M = g.M;
  const float* frac = reinterpret_cast<const float*>(na.frac);
  for (int e = tid; e < kRegAccKeys; e += kRegAccThreads) st.count[e] = 0;
  float2* box = st.box();
  const bool tma_cta = tma_on && (smem_u32(box) & 127) == 0;

  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int4 item = na.items[it];
    int tc[3], start[3];
    tile_origin(g, item.x, tc);
#pragma unroll
    for (int d = 0; d < 3; ++d) start[d] = tc[d] * g.T[d] + g.off;
    const int count = item.z;

    __syncthreads();  // previous item done; counts cleared
    for (int i = tid; i < count; i += kRegAccThreads) {
      const int q = item.y + i;
      int a[3];
      float t[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        a[d] = na.cell[d * M + q] - tc[d] * g.T[d];
        t[d] = frac[d * M + q];
      }
      const float2 v = fhat[na.perm[q]];
      const int key = a[0] * kRegAccA + a[1];
      const int rank = atomicAdd(&st.count[key], 1);
      st.rec[i][0] = make_float4(t[0], t[1], t[2], __int_as_float(a[0] | (a[1] << 8) | (a[2] << 16)));
      st.rec[i][1] = make_float4(v.x, v.y, __int_as_float(key), __int_as_float(rank));
    }
    if (tma_cta) {
      // the previous item's box reduction has read shared memory before the
      // weight arrays it overlays are written again
      if (tid == 0) bulk_wait_read();
      __syncthreads();
    }
    {
      // clear the shifted rows of the slots in use (vw1: 8 float4, w2s: 4 float4 per slot)
      float4* z1 = reinterpret_cast<float4*>(&st.vw1[0][0]);
      float4* z2 = reinterpret_cast<float4*>(&st.w2s[0][0]);
      for (int e = tid; e < count * 8; e += kRegAccThreads) {
        z1[e] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (e < count * 4) z2[e] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    __syncthreads();
    if (warp == 0) {
      // exclusive scan of the 81 counts: lane owns keys 3 lane .. 3 lane + 2
      int cv[3], sum = 0;
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int key = 3 * lane + u;
        cv[u] = key < kRegAccKeys ? st.count[key] : 0;
        sum += cv[u];
      }
      int incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      int run = incl - sum;
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int key = 3 * lane + u;
        if (key <= kRegAccKeys) st.start[key] = run;
        run += cv[u];
      }
    }
    __syncthreads();
    if (wj < kPerIter) {
      f32x2 cpair[3][K + 1];
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int e = 0; e <= K; ++e) cpair[d][e] = st.coef[d][tp][e];
      for (int s = kPerIter * warp + wj; s < count; s += kPerIter * kRegAccWarps) {
        const float4 r0 = st.rec[s][0];
        const float4 rv = st.rec[s][1];
        const int pk = __float_as_int(r0.w);
        const int q = st.start[__float_as_int(rv.z)] + __float_as_int(rv.w);
        float2 w[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const float z = (d == 0 ? r0.x : (d == 1 ? r0.y : r0.z)) - 0.5f;
          const f32x2 zz = pack2(z, z);
          f32x2 pw = cpair[d][K];
#pragma unroll
          for (int e = K - 1; e >= 0; --e) pw = fma2(pw, zz, cpair[d][e]);
          w[d] = unpack2(pw);  // taps 2 tp, 2 tp + 1
        }
        *reinterpret_cast<float2*>(&st.w0s[q][2 * tp]) = w[0];
        const int r = ((pk >> 8) & 0xff) + 2 * tp;
        st.vw1[q][r] = pack2(rv.x * w[1].x, rv.y * w[1].x);
        st.vw1[q][r + 1] = pack2(rv.x * w[1].y, rv.y * w[1].y);
        // column c sits in pair cc = c & 7, half c >> 3 (two copies)
        const int c0 = (pk >> 16) + 2 * tp, c1 = c0 + 1;
        float* w2f = reinterpret_cast<float*>(&st.w2s[q][0]);
        w2f[2 * (c0 & 7) + (c0 >> 3)] = w[2].x;
        w2f[2 * (c1 & 7) + (c1 >> 3)] = w[2].y;
      }
    }
    __syncthreads();
    for (int e = tid; e < kRegAccKeys; e += kRegAccThreads) st.count[e] = 0;  // for the next item

    f32x2 acc[2][kRegAccLines];
    RegAccComp<COMP> cp;
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int r = 0; r < kRegAccLines; ++r) acc[h][r] = pack2(0.f, 0.f);
    if constexpr (COMP) {
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int r = 0; r < kRegAccLines; ++r) cp.c[h][r] = pack2(0.f, 0.f);
    }
    regacc_bin<0, K, COMP>(st, lo, hi, r1, cc, acc, cp);
    regacc_bin<1, K, COMP>(st, lo, hi, r1, cc, acc, cp);
    regacc_bin<2, K, COMP>(st, lo, hi, r1, cc, acc, cp);
    regacc_bin<3, K, COMP>(st, lo, hi, r1, cc, acc, cp);
    regacc_bin<4, K, COMP>(st, lo, hi, r1, cc, acc, cp);
    regacc_bin<5, K, COMP>(st, lo, hi, r1, cc, acc, cp);
    regacc_bin<6, K, COMP>(st, lo, hi, r1, cc, acc, cp);
    regacc_bin<7, K, COMP>(st, lo, hi, r1, cc, acc, cp);
    regacc_bin<8, K, COMP>(st, lo, hi, r1, cc, acc, cp);
    if constexpr (COMP) {
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int r = 0; r < kRegAccLines; ++r) acc[h][r] = add2(acc[h][r], cp.c[h][r]);
    }

    // add the region to the grid: one bulk tensor reduction of a box 18
    // points wide starting at the even x0 = start[2] - lead (columns outside
    // the region carry zeros) where the region lies inside the grid
    const int lead = start[2] & 1, x0 = start[2] - lead;
    const bool by_tma = tma_cta && x0 >= 0 && x0 + kFlushPitch <= g.Nt[2] && start[1] >= 0 &&
                        start[1] + L1 <= g.Nt[1] && start[0] >= 0 && start[0] + L0 <= g.Nt[0];
    if (by_tma) {
      __syncthreads();  // every warp is done with the weight arrays the box overlays
      if (r1 < L1) {
#pragma unroll
        for (int r = 0; r < kRegAccLines; ++r) {
          if (r < L0) {
            float2* row = box + (r * L1 + r1) * kFlushPitch;
            row[cc + lead] = unpack2(acc[0][r]);
            row[cc + 8 + lead] = unpack2(acc[1][r]);
            if (cc == 0) row[lead ? 0 : 16] = make_float2(0.f, 0.f);
            if (cc == 1) row[17] = make_float2(0.f, 0.f);
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) tma_reduce_add_box(&rmap, box, 2 * x0, start[1], start[0]);
      continue;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = cc + 8 * h;
      if (r1 < L1 && c < L2) {
        const int g1 = wrap1(start[1] + r1, g.Nt[1]);
        const int g2 = wrap1(start[2] + c, g.Nt[2]);
#pragma unroll
        for (int r = 0; r < kRegAccLines; ++r) {
          if (r < L0) {
            const int g0 = wrap1(start[0] + r, g.Nt[0]);
            atomicAdd(grid + ((int64_t)g0 * g.Nt[1] + g1) * g.Nt[2] + g2, unpack2(acc[h][r]));
          }
        }
      }
    }
  }
  if (tma_cta && tid == 0) bulk_wait_all();
}

// ---------------------------------------------------------------------------
// Register-resident gather, K = 2m taps per dimension: the ownership of the
// register-accumulating scatter turned around.  Thread (r1, cc) of a
// 128-thread CTA loads the two region lines (., r1, cc) and (., r1, cc + 8)
// of the tile + halo into registers (reg[h][r0], r0 < L0 <= 16) once per
// work item, and for a node at offset (a0, a1, a2) forms
//   p = w1[r1 - a1] (w2[cc - a2]     sum_i0 w0[i0] reg[0][a0 + i0]
//                  + w2[cc + 8 - a2] sum_i0 w0[i0] reg[1][a0 + i0]),
// 2K + 2 packed operations with static register indices (nodes
// counting-sorted by (a0, a1), one loop per a0 bin, as in the scatter).  The
// window values are stored once, as in the scatter: stored as (w, w) pairs
// they took twice the shared wavefronts, and the gather measured slower
// (0.95 against 0.90 ms at 160^3, m = 6).  The warp sums p over its lanes
// four nodes at a time: one exchange hands nodes s, s + 1 to lanes 0..15
// and s + 2, s + 3 to lanes 16..31, a second splits each half into 8-lane
// groups of one node, three more levels sum the groups (3 shuffles of a
// pair per node instead of 10 for a lone node).  Taps are read from
// registers, so the shared-memory pipe carries only the broadcast window
// loads and the shuffles, where the shared-tap gathers read every tap of
// every node from shared memory.  A warp stores its sum for a node in its
// own slot; after the node loop one thread per node adds the slots of the
// warps whose rows meet the node's footprint, in warp order, so the result
// does not depend on scheduling.
template <int K>
struct GatherRegStage {
  static constexpr int kPairs = K / 2;
  union {  // the records are done with once the window values are stored
    float4 rec[kItemCap][2];                      // {t0, t1, t2, pk}, {perm, 0, key, rank}
    f32x2 part[kRegAccWarps][kItemCap];           // per-warp sums, by slot
  };
  int count[kRegAccKeys];
  int start[kRegAccKeys + 1];
  f32x2 coef[3][kPairs][K + 1];                   // (tap 2 tp, tap 2 tp + 1) coefficient pairs
  alignas(16) float w0s[kItemCap][K];             // w0, by slot
  alignas(16) float w1r[kItemCap][kRegAccLines];  // w1[r - a1] by region row (zero outside), by slot
  alignas(16) float2 w2s[kItemCap][8];            // cc -> (w2[cc - a2], w2[cc + 8 - a2]), by slot
  int sperm[kItemCap];                            // caller index, by slot
  int sa1[kItemCap];                              // a1, by slot
};
// four CTAs per SM: 4 x (stage + 1 KB reserved) within the SM's 228 KB
static_assert(sizeof(GatherRegStage<12>) <= 56 * 1024, "four gather CTAs per SM");

template <int A0, int K>
__device__ __forceinline__ f32x2 gather_reg_node(const GatherRegStage<K>& st, int s, int r1, int cc,
                                                 const f32x2 (&reg)[2][kRegAccLines]) {
  const float u = st.w1r[s][r1];
  const float2 w2 = st.w2s[s][cc];
  const float4* wq = reinterpret_cast<const float4*>(&st.w0s[s][0]);
  f32x2 t0 = 0, t1 = 0;
#pragma unroll
  for (int q = 0; q < K / 4; ++q) {
    const float4 x = wq[q];
    const float xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const f32x2 wa = pack2(xs[j], xs[j]);
      if (q == 0 && j == 0) {
        t0 = mul2(reg[0][A0], wa);
        t1 = mul2(reg[1][A0], wa);
      } else {
        t0 = fma2(reg[0][A0 + 4 * q + j], wa, t0);
        t1 = fma2(reg[1][A0 + 4 * q + j], wa, t1);
      }
    }
  }
  const float u0 = u * w2.x, u1 = u * w2.y;
  return fma2(t1, pack2(u1, u1), mul2(t0, pack2(u0, u0)));
}

__device__ __forceinline__ f32x2 shfl_xor2(f32x2 v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }

// Sum of p[j] over the warp's lanes for the n <= 4 nodes s + j; lane 8 j
// stores the sum of node s + j in the warp's slot.
__device__ __forceinline__ void warp_sum4_store(f32x2 (&p)[4], f32x2* part, int s, int n, int lane) {
  const bool u16 = (lane & 16) != 0, u8 = (lane & 8) != 0;
  f32x2 k0 = u16 ? p[2] : p[0], k1 = u16 ? p[3] : p[1];
  k0 = add2(k0, shfl_xor2(u16 ? p[0] : p[2], 16));
  k1 = add2(k1, shfl_xor2(u16 ? p[1] : p[3], 16));
  f32x2 k = u8 ? k1 : k0;
  k = add2(k, shfl_xor2(u8 ? k0 : k1, 8));
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) k = add2(k, shfl_xor2(k, o));
  const int j = lane >> 3;
  if ((lane & 7) == 0 && j < n) part[s + j] = k;
}

template <int A0, int K>
__device__ __forceinline__ void gather_reg_bin(GatherRegStage<K>& st, int lo, int hi, int r1, int cc, int warp,
                                               int lane, const f32x2 (&reg)[2][kRegAccLines]) {
  if constexpr (A0 + K <= kRegAccLines) {  // a0 < T0 <= 17 - K
    const int s0 = st.start[A0 * kRegAccA + lo], s1 = st.start[A0 * kRegAccA + hi + 1];
    int s = s0;
    for (; s + 3 < s1; s += 4) {
      f32x2 p[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) p[j] = gather_reg_node<A0, K>(st, s + j, r1, cc, reg);
      warp_sum4_store(p, st.part[warp], s, 4, lane);
    }
    if (s < s1) {  // 1 to 3 nodes left (s1 is uniform over the warp)
      f32x2 p[4] = {0, 0, 0, 0};
      p[0] = gather_reg_node<A0, K>(st, s, r1, cc, reg);
      if (s + 1 < s1) p[1] = gather_reg_node<A0, K>(st, s + 1, r1, cc, reg);
      if (s + 2 < s1) p[2] = gather_reg_node<A0, K>(st, s + 2, r1, cc, reg);
      warp_sum4_store(p, st.part[warp], s, s1 - s, lane);
    }
  }
}

template <int K>
__global__ void __launch_bounds__(kRegAccThreads, 4)
    gather3d_reg_kernel(Geometry g, const float2* __restrict__ grid, NodeArrays na,
                        const float* __restrict__ poly, float2* __restrict__ fhat) {
  using Stage = GatherRegStage<K>;
  constexpr int P = Stage::kPairs;
  constexpr int kPerIter = 32 / P;  // nodes per warp and weight iteration
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Stage& st = *reinterpret_cast<Stage*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r1 = tid >> 3, cc = tid & 7;
  // a1 run of this warp: one of rows 4w .. 4w + 3 lies in [a1, a1 + K)
  const int lo = max(0, 4 * warp - (K - 1)), hi = min(kRegAccA - 1, 4 * warp + 3);
  const int wj = lane / P, tp = lane - P * (lane / P);
  for (int e = tid; e < 3 * P * (K + 1); e += kRegAccThreads) {
    const int d = e / (P * (K + 1)), pp = (e / (K + 1)) % P, z = e % (K + 1);
    st.coef[d][pp][z] = pack2(poly[(d * K + 2 * pp) * (K + 1) + z], poly[(d * K + 2 * pp + 1) * (K + 1) + z]);
  }
  const int nitems = *na.n_items;
  const int L0 = g.L[0], L1 = g.L[1], L2 = g.L[2];
  const int64_t M = g.M;
  const int64_t plane = (int64_t)g.Nt[1] * g.Nt[2];
  const float* frac = reinterpret_cast<const float*>(na.frac);
  const f32x2* gp = reinterpret_cast<const f32x2*>(grid);
  for (int e = tid; e < kRegAccKeys; e += kRegAccThreads) st.count[e] = 0;

  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int4 item = na.items[it];
    int tc[3], start[3];
    tile_origin(g, item.x, tc);
#pragma unroll
    for (int d = 0; d < 3; ++d) start[d] = tc[d] * g.T[d] + g.off;
    const int count = item.z;

    // the two region lines of this thread, issued first and consumed after
    // the window values (zero outside the region)
    f32x2 reg[2][kRegAccLines];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = cc + 8 * h;
      const bool ok = r1 < L1 && c < L2;
      const f32x2* src = gp;
      if (ok) src = gp + (int64_t)wrap1(start[1] + r1, g.Nt[1]) * g.Nt[2] + wrap1(start[2] + c, g.Nt[2]);
#pragma unroll
      for (int r = 0; r < kRegAccLines; ++r)
        reg[h][r] = (ok && r < L0) ? __ldg(src + wrap1(start[0] + r, g.Nt[0]) * plane) : 0ull;
    }

    __syncthreads();  // previous item's sums written out; counts cleared
    for (int i = tid; i < count; i += kRegAccThreads) {
      const int q = item.y + i;
      int a[3];
      float t[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        a[d] = na.cell[d * M + q] - tc[d] * g.T[d];
        t[d] = frac[d * M + q];
      }
      const int key = a[0] * kRegAccA + a[1];
      const int rank = atomicAdd(&st.count[key], 1);
      st.rec[i][0] = make_float4(t[0], t[1], t[2], __int_as_float(a[0] | (a[1] << 8) | (a[2] << 16)));
      st.rec[i][1] = make_float4(__int_as_float(na.perm[q]), 0.f, __int_as_float(key), __int_as_float(rank));
    }
    {
      // clear the shifted rows of the slots in use (w1r, w2s: 4 float4 each per slot)
      float4* z1 = reinterpret_cast<float4*>(&st.w1r[0][0]);
      float4* z2 = reinterpret_cast<float4*>(&st.w2s[0][0]);
      for (int e = tid; e < count * 4; e += kRegAccThreads) {
        z1[e] = make_float4(0.f, 0.f, 0.f, 0.f);
        z2[e] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    __syncthreads();
    if (warp == 0) {
      // exclusive scan of the 81 counts: lane owns keys 3 lane .. 3 lane + 2
      int cv[3], sum = 0;
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int key = 3 * lane + u;
        cv[u] = key < kRegAccKeys ? st.count[key] : 0;
        sum += cv[u];
      }
      int incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      int run = incl - sum;
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int key = 3 * lane + u;
        if (key <= kRegAccKeys) st.start[key] = run;
        run += cv[u];
      }
    }
    __syncthreads();
    if (wj < kPerIter) {
#pragma unroll
      for (int d = 0; d < 3; ++d) {  // one dimension's coefficients in registers at a time
        f32x2 cpair[K + 1];
#pragma unroll
        for (int e = 0; e <= K; ++e) cpair[e] = st.coef[d][tp][e];
        for (int s = kPerIter * warp + wj; s < count; s += kPerIter * kRegAccWarps) {
          const float4 r0 = st.rec[s][0];
          const float4 rv = st.rec[s][1];
          const int pk = __float_as_int(r0.w);
          const int q = st.start[__float_as_int(rv.z)] + __float_as_int(rv.w);
          const float z = (d == 0 ? r0.x : (d == 1 ? r0.y : r0.z)) - 0.5f;
          const f32x2 zz = pack2(z, z);
          f32x2 pw = cpair[K];
#pragma unroll
          for (int e = K - 1; e >= 0; --e) pw = fma2(pw, zz, cpair[e]);
          const float2 w = unpack2(pw);  // taps 2 tp, 2 tp + 1
          if (d == 0) {
            *reinterpret_cast<float2*>(&st.w0s[q][2 * tp]) = w;
            if (tp == 0) {
              st.sperm[q] = __float_as_int(rv.x);
              st.sa1[q] = (pk >> 8) & 0xff;
            }
          } else if (d == 1) {
            const int r = ((pk >> 8) & 0xff) + 2 * tp;
            st.w1r[q][r] = w.x;
            st.w1r[q][r + 1] = w.y;
          } else {
            // column c sits in pair cc = c & 7, half c >> 3
            const int c0 = (pk >> 16) + 2 * tp, c1 = c0 + 1;
            float* w2f = reinterpret_cast<float*>(&st.w2s[q][0]);
            w2f[2 * (c0 & 7) + (c0 >> 3)] = w.x;
            w2f[2 * (c1 & 7) + (c1 >> 3)] = w.y;
          }
        }
      }
    }
    __syncthreads();
    for (int e = tid; e < kRegAccKeys; e += kRegAccThreads) st.count[e] = 0;  // for the next item

    gather_reg_bin<0, K>(st, lo, hi, r1, cc, warp, lane, reg);
    gather_reg_bin<1, K>(st, lo, hi, r1, cc, warp, lane, reg);
    gather_reg_bin<2, K>(st, lo, hi, r1, cc, warp, lane, reg);
    gather_reg_bin<3, K>(st, lo, hi, r1, cc, warp, lane, reg);
    gather_reg_bin<4, K>(st, lo, hi, r1, cc, warp, lane, reg);
    gather_reg_bin<5, K>(st, lo, hi, r1, cc, warp, lane, reg);
    gather_reg_bin<6, K>(st, lo, hi, r1, cc, warp, lane, reg);
    gather_reg_bin<7, K>(st, lo, hi, r1, cc, warp, lane, reg);
    gather_reg_bin<8, K>(st, lo, hi, r1, cc, warp, lane, reg);
    __syncthreads();
    // sum the slots of the warps whose rows meet the node's footprint
    for (int s = tid; s < count; s += kRegAccThreads) {
      const int a1 = st.sa1[s];
      f32x2 acc = 0;
#pragma unroll
      for (int w = 0; w < kRegAccWarps; ++w)
        if (a1 >= max(0, 4 * w - (K - 1)) && a1 <= 4 * w + 3) acc = add2(acc, st.part[w][s]);
      fhat[st.sperm[s]] = unpack2(acc);
    }
  }
}

bool regacc_supported(const Geometry& g) {
  if (g.D != 3 || g.closed || (g.K != 8 && g.K != 12) || g.m != 0.5 * g.K || g.off != 1 - g.K / 2) return false;
  for (int d = 0; d < 3; ++d)
    if (g.T[d] > kRegAccLines + 1 - g.K || g.T[d] > g.Nt[d] - g.K + 1) return false;
  return true;
}

// Scatter form: NFFT_GB300_SCATTER=smem selects the shared-accumulator
// kernel below, anything else the register-accumulating one (where the tile
// allows it).
bool use_regacc(const Geometry& g) {
  static int smem_form = [] {
    const char* e = getenv("NFFT_GB300_SCATTER");
    return (e && strcmp(e, "smem") == 0) ? 1 : 0;
  }();
  // the shared-accumulator form exists for K = 8 only
  return regacc_supported(g) && (!smem_form || g.K != kTaps);
}

}  // namespace

bool fast_scatter_supported(const Geometry& g, int cmax) { return cmax <= kItemCap && use_regacc(g); }

namespace {

// Gather form: NFFT_GB300_GATHER=smem keeps the shared-tap kernels, =regs
// takes the register-resident one for K = 8 as well; by default it serves
// K = 12 (read at each launch, so that the forms can be compared in one
// process).
bool use_gather_reg(const Geometry& g) {
  if (!regacc_supported(g)) return false;
  const char* e = getenv("NFFT_GB300_GATHER");
  if (e && strcmp(e, "smem") == 0) return false;
  return g.K == kG12Taps || (e && strcmp(e, "regs") == 0);
}
void* gather_reg_kernel(int K) { return K == 12 ? (void*)gather3d_reg_kernel<12> : (void*)gather3d_reg_kernel<8>; }
size_t gather_reg_smem(int K) { return K == 12 ? sizeof(GatherRegStage<12>) : sizeof(GatherRegStage<8>); }

void* regacc_kernel(int K, bool comp) {
  if (comp) return K == 12 ? (void*)scatter3d_regacc_kernel<12, true> : (void*)scatter3d_regacc_kernel<8, true>;
  return K == 12 ? (void*)scatter3d_regacc_kernel<12, false> : (void*)scatter3d_regacc_kernel<8, false>;
}
size_t regacc_smem(int K) { return K == 12 ? sizeof(RegAccStage<12>) : sizeof(RegAccStage<8>); }

int gather_warps() {
  static int w = [] {
    const char* e = getenv("NFFT_GB300_GATHER_WARPS");
    const int v = e ? atoi(e) : 4;
    return (v == 2 || v == 4 || v == 8) ? v : 4;
  }();
  return w;
}

void* gather_kernel_for(int w) {
  switch (w) {
    case 2: return (void*)gather3d_m4_kernel<2>;
    case 8: return (void*)gather3d_m4_kernel<8>;
    default: return (void*)gather3d_m4_kernel<4>;
  }
}

int scatter_warps() {
  static int w = [] {
    const char* e = getenv("NFFT_GB300_SCATTER_WARPS");
    const int v = e ? atoi(e) : 2;
    return (v == 1 || v == 2 || v == 4 || v == 8) ? v : 4;
  }();
  return w;
}

void* scatter_kernel_for(int w) {
  switch (w) {
    case 1: return (void*)scatter3d_m4_kernel<1>;
    case 2: return (void*)scatter3d_m4_kernel<2>;
    case 8: return (void*)scatter3d_m4_kernel<8>;
    default: return (void*)scatter3d_m4_kernel<4>;
  }
}

size_t smem_bytes(const Geometry& g) {
  return sizeof(NodeStage) + (size_t)g.L[0] * g.L[1] * kPitch * sizeof(float2);
}

// the gather and the node gradient add the window slots and the region
// copy's mbarrier after the tile
size_t gather_smem_bytes(const Geometry& g) { return smem_bytes(g) + kGatherTail; }

// Tensor-memory-accelerator map of the grid for the region copies of the
// gather and the node gradient: 3D, 8-byte points, box {18, L1, L0} (a
// region with its padded rows).  False where the copy cannot be used (odd
// T2, a box larger than the grid or than 256 points, the driver entry point
// or the encoding unavailable); the kernels then use cp.async throughout.
using EncodeTiledFn = PFN_cuTensorMapEncodeTiled_v12000;

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return (EncodeTiledFn) nullptr;
    }
    return reinterpret_cast<EncodeTiledFn>(f);
  }();
  return fn;
}

// NFFT_GB300_GATHER_TMA=0 keeps every region copy on cp.async (read at each
// launch, so that both copy forms can be compared in one process).
bool use_region_tma() {
  const char* e = getenv("NFFT_GB300_GATHER_TMA");
  return !(e && strcmp(e, "0") == 0);
}

// Kernel argument tma_on: bit 0 = region copies by TMA; bits 8.. = bytes the
// mbarrier expects beyond the box (0 unless NFFT_GB300_TEST_TX_EXTRA is set:
// a test hook that makes the bounded wait run out with no copy in flight, so
// that the timeout path can be exercised without a fault).
int region_tma_arg(bool on) {
  if (!on) return 0;
  const char* e = getenv("NFFT_GB300_TEST_TX_EXTRA");
  const int extra = e ? atoi(e) : 0;
  return 1 | ((extra > 0 && extra <= 4096 ? extra : 0) << 8);
}

bool region_map(const Geometry& g, const void* grid, CUtensorMap* map) {
  memset(map, 0, sizeof(*map));
  if (!use_region_tma() || (g.T[2] & 1) || ((uintptr_t)grid & 15)) return false;
  const int box[3] = {kPitch, g.L[1], g.L[0]};
  const int dim[3] = {g.Nt[2], g.Nt[1], g.Nt[0]};
  for (int d = 0; d < 3; ++d)
    if (box[d] > 256 || box[d] > dim[d]) return false;
  if ((g.Nt[2] * sizeof(float2)) % 16 != 0) return false;
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t gdim[3] = {(cuuint64_t)dim[0], (cuuint64_t)dim[1], (cuuint64_t)dim[2]};
  const cuuint64_t gstride[2] = {(cuuint64_t)g.Nt[2] * sizeof(float2),
                                 (cuuint64_t)g.Nt[1] * g.Nt[2] * sizeof(float2)};
  const cuuint32_t bdim[3] = {(cuuint32_t)box[0], (cuuint32_t)box[1], (cuuint32_t)box[2]};
  const cuuint32_t estride[3] = {1, 1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<void*>(grid), gdim, gstride, bdim,
                        estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    memset(map, 0, sizeof(*map));
    return false;
  }
  return true;
}

// NFFT_GB300_SCATTER_TMA=0 keeps every scatter flush on vector global
// reductions (read at each launch, like NFFT_GB300_GATHER_TMA).
bool use_flush_tma() {
  const char* e = getenv("NFFT_GB300_SCATTER_TMA");
  return !(e && strcmp(e, "0") == 0);
}

// The grid as FP32 (real, imaginary interleaved) for the scatter's box
// reductions: box = 2 * kFlushPitch floats x L1 x L0.
bool flush_map(const Geometry& g, const void* grid, CUtensorMap* map) {
  memset(map, 0, sizeof(*map));
  if (!use_flush_tma() || ((uintptr_t)grid & 15)) return false;
  const int box[3] = {2 * kFlushPitch, g.L[1], g.L[0]};
  const int dim[3] = {2 * g.Nt[2], g.Nt[1], g.Nt[0]};
  for (int d = 0; d < 3; ++d)
    if (box[d] > 256 || box[d] > dim[d]) return false;
  if ((g.Nt[2] * sizeof(float2)) % 16 != 0) return false;
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t gdim[3] = {(cuuint64_t)dim[0], (cuuint64_t)dim[1], (cuuint64_t)dim[2]};
  const cuuint64_t gstride[2] = {(cuuint64_t)g.Nt[2] * sizeof(float2),
                                 (cuuint64_t)g.Nt[1] * g.Nt[2] * sizeof(float2)};
  const cuuint32_t bdim[3] = {(cuuint32_t)box[0], (cuuint32_t)box[1], (cuuint32_t)box[2]};
  const cuuint32_t estride[3] = {1, 1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(grid), gdim, gstride, bdim,
                        estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    memset(map, 0, sizeof(*map));
    return false;
  }
  return true;
}

template <typename K>
cudaError_t set_smem(K kern, size_t smem) {
  if (smem > 48 * 1024)
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaSuccess;
}

}  // namespace

bool fast3d_supported(const Geometry& g, int cmax) {
  if (g.K == kG12Taps) return g12_supported(g, cmax);
  if (g.D != 3 || g.K != kTaps || g.closed || g.off != -3 || g.m != 4.0) return false;
  if (g.T[2] > kMaxTile2 || cmax > kItemCap) return false;
  for (int d = 0; d < 3; ++d)
    if (g.T[d] > g.Nt[d] - kTaps + 1 || g.L[d] > 255) return false;
  return gather_smem_bytes(g) <= 200 * 1024;
}

int fast3d_ctas_per_sm(const Geometry& g, int kind) {
  if (kind == 2) {  // compensated scatter: the register-accumulating form only
    if (!regacc_supported(g)) return 0;
    const size_t smem = regacc_smem(g.K);
    void* k = regacc_kernel(g.K, true);
    if (set_smem(k, smem) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kRegAccThreads, smem) != cudaSuccess) return 0;
    return n;
  }
  if (kind == 1 && use_regacc(g)) {
    const size_t smem = regacc_smem(g.K);
    void* k = regacc_kernel(g.K, false);
    if (set_smem(k, smem) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kRegAccThreads, smem) != cudaSuccess) return 0;
    return n;
  }
  if (kind == 0 && use_gather_reg(g)) {
    const size_t smem = gather_reg_smem(g.K);
    void* k = gather_reg_kernel(g.K);
    if (set_smem(k, smem) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kRegAccThreads, smem) != cudaSuccess) return 0;
    return n;
  }
  if (kind == 0 && g.K == kG12Taps) {
    const size_t smem = g12_smem_bytes(g);
    if (set_smem(gather3d_k12_kernel, smem) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, gather3d_k12_kernel, kG12Threads, smem) != cudaSuccess)
      return 0;
    return n;
  }
  if (g.K != kTaps) return 0;
  const size_t smem = kind == 0 ? gather_smem_bytes(g) : smem_bytes(g);
  void* k = kind == 0 ? gather_kernel_for(gather_warps()) : scatter_kernel_for(scatter_warps());
  const int threads = kind == 0 ? 32 * gather_warps() : 32 * scatter_warps();
  if (set_smem(k, smem) != cudaSuccess) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, smem) != cudaSuccess) return 0;
  return n;
}

cudaError_t launch_gather3d_fast(const Geometry& g, const void* grid, const NodeArrays& na,
                                 const float* poly, void* fhat, int ctas, cudaStream_t s) {
  if (use_gather_reg(g)) {
    const size_t smem = gather_reg_smem(g.K);
    void* k = gather_reg_kernel(g.K);
    cudaError_t e = set_smem(k, smem);
    if (e != cudaSuccess) return e;
    auto kern = reinterpret_cast<void (*)(Geometry, const float2*, NodeArrays, const float*, float2*)>(k);
    kern<<<ctas, kRegAccThreads, smem, s>>>(g, (const float2*)grid, na, poly, (float2*)fhat);
    return cudaGetLastError();
  }
  if (g.K == kG12Taps) {
    const size_t smem = g12_smem_bytes(g);
    cudaError_t e = set_smem(gather3d_k12_kernel, smem);
    if (e != cudaSuccess) return e;
    gather3d_k12_kernel<<<ctas, kG12Threads, smem, s>>>(g, (const float2*)grid, na, poly, (float2*)fhat);
    return cudaGetLastError();
  }
  const size_t smem = gather_smem_bytes(g);
  const int w = gather_warps();
  void* k = gather_kernel_for(w);
  cudaError_t e = set_smem(k, smem);
  if (e != cudaSuccess) return e;
  CUtensorMap map;
  const int tma_on = region_tma_arg(region_map(g, grid, &map));
  auto kern = reinterpret_cast<void (*)(Geometry, const float2*, NodeArrays, const float*, float2*,
                                        const CUtensorMap, int)>(k);
  kern<<<ctas, 32 * w, smem, s>>>(g, (const float2*)grid, na, poly, (float2*)fhat, map, tma_on);
  return cudaGetLastError();
}

cudaError_t launch_grad3d_fast(const Geometry& g, const void* grid, const NodeArrays& na, const float* poly,
                               const void* cot, void* gk, int ctas, cudaStream_t s) {
  const size_t smem = gather_smem_bytes(g);
  cudaError_t e = set_smem(grad3d_m4_kernel<4>, smem);
  if (e != cudaSuccess) return e;
  CUtensorMap map;
  const int tma_on = region_tma_arg(region_map(g, grid, &map));
  grad3d_m4_kernel<4><<<ctas, 128, smem, s>>>(g, (const float2*)grid, na, poly, (const float2*)cot, (float*)gk,
                                              map, tma_on);
  return cudaGetLastError();
}

int grad3d_ctas_per_sm(const Geometry& g) {
  const size_t smem = gather_smem_bytes(g);
  if (set_smem(grad3d_m4_kernel<4>, smem) != cudaSuccess) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, grad3d_m4_kernel<4>, 128, smem) != cudaSuccess) return 0;
  return n;
}

cudaError_t launch_scatter3d_fast(const Geometry& g, void* grid, const NodeArrays& na,
                                  const float* poly, const void* fhat, int compensated, int ctas, cudaStream_t s) {
  if (compensated || use_regacc(g)) {
    const size_t smem = regacc_smem(g.K);
    void* k = regacc_kernel(g.K, compensated != 0);
    cudaError_t e = set_smem(k, smem);
    if (e != cudaSuccess) return e;
    CUtensorMap map;
    const int tma_on = flush_map(g, grid, &map) ? 1 : 0;
    auto kern = reinterpret_cast<void (*)(Geometry, float2*, NodeArrays, const float*, const float2*,
                                          const CUtensorMap, int)>(k);
    kern<<<ctas, kRegAccThreads, smem, s>>>(g, (float2*)grid, na, poly, (const float2*)fhat, map, tma_on);
    return cudaGetLastError();
  }
  const size_t smem = smem_bytes(g);
  const int w = scatter_warps();
  void* k = scatter_kernel_for(w);
  cudaError_t e = set_smem(k, smem);
  if (e != cudaSuccess) return e;
  auto kern = reinterpret_cast<void (*)(Geometry, float2*, NodeArrays, const float*, const float2*)>(k);
  kern<<<ctas, 32 * w, smem, s>>>(g, (float2*)grid, na, poly, (const float2*)fhat);
  return cudaGetLastError();
}

int fast3d_take_wait_timeout() {
  int h = 0;
  if (cudaMemcpyFromSymbol(&h, g_wait_timeout, sizeof(int)) != cudaSuccess) return -1;
  if (h) {
    const int z = 0;
    if (cudaMemcpyToSymbol(g_wait_timeout, &z, sizeof(int)) != cudaSuccess) return -1;
  }
  return h;
}

}  // namespace nfftgb
