// 2D kernels for m = 4 (8 taps per dimension), complex64, for single plans
// and for batches: a register-accumulating scatter and a warp-per-item
// gather.
//
// Same computation as the generic scatter (Eq. SumOverNodeAdjoint, Eq.
// InnerTensorStructure, Algorithm 4) with the tile + halo region held in
// registers: lane c of a warp owns the region column (., c), c < L1 <= 32,
// as 16 packed complex accumulators acc[r0] (r0 < L0 <= 16).  A node at tile
// offset (a0, a1) adds  v w1[c - a1] * w0[i0]  to acc[a0 + i0], i0 = 0..7:
// 8 packed FMAs per lane and node, no shared-memory accumulation.  Register
// indices must be static, so each staged chunk of 32 nodes is binned by a0
// with warp ballots and every bin runs a loop specialised to its a0.
//
// Each warp works on its own work items (no block-wide barriers): per chunk
// of 32 nodes, lane i loads node i (cells, fractions, value), evaluates its
// 16 window values and writes them at its bin slot in the warp's stage; the
// warp then runs over the bins.  After the item's last chunk the region is
// added to the grid with vector global reductions (periodic wrap only there).
//
// Window values come from the POLYNOMIAL representation (Sec. 3.7.4): the
// problem's coefficient table is copied into the warp's shared memory as
// (tap 2p, tap 2p + 1) pairs per item, and a lane evaluates the 16 values of
// its own node as 8 packed Horner chains of degree 2m whose coefficient loads
// are warp-wide broadcasts.
//
// The gather keeps the same one-warp-per-item structure (no block-wide
// barriers): the warp copies its item's region (<= 16 x 32) into its own
// shared-memory tile with coalesced row loads, then each lane takes one node
// (Eq. SumOverNode as the nested sum of Eq. InnerTensorStructure, packed
// complex FMAs) and writes fhat in the caller's order.
#include "packed_f32x2.cuh"
#include "resample.cuh"

namespace nfftgb {
namespace {

constexpr int k2Taps = 8;
constexpr int k2Lines = 16;                 // acc[r0], L0 <= 16
constexpr int k2Cols = 32;                  // one region column per lane, L1 <= 32
constexpr int k2Warps = 4;                  // independent warps per CTA
constexpr int k2Threads = 32 * k2Warps;
constexpr int k2Bins = 9;                   // a0 < T0 <= 9
constexpr int k2Deg = 2 * 4;                // POLYNOMIAL degree 2m
constexpr int k2Pairs = k2Taps / 2;

// POLYNOMIAL coefficients of one problem, (tap 2p, tap 2p + 1) pairs.
struct Poly2d {
  f32x2 c[2][k2Pairs][k2Deg + 1];
};

// Copies the coefficient table coef[(d * K + i) * (deg + 1) + z] (built by
// the plan or batch at creation) into the warp's pairs.
__device__ __forceinline__ void load_poly2d(const float* __restrict__ poly, Poly2d& pc, int lane) {
  constexpr int Z = k2Deg + 1;
  for (int e = lane; e < 2 * k2Pairs * Z; e += 32) {
    const int d = e / (k2Pairs * Z), p = (e / Z) % k2Pairs, z = e % Z;
    pc.c[d][p][z] = pack2(poly[(d * k2Taps + 2 * p) * Z + z], poly[(d * k2Taps + 2 * p + 1) * Z + z]);
  }
}

// Window values of taps 2p, 2p + 1 of dimension d at zeta = t - 1/2.
// The coefficients are read from shared memory at every use (lds_f32x2):
// held in registers across the node loop they would cost 144 registers.
__device__ __forceinline__ f32x2 poly2d_pair(const Poly2d& pc, int d, int p, f32x2 zz) {
  f32x2 w = lds_f32x2(&pc.c[d][p][k2Deg]);
#pragma unroll
  for (int z = k2Deg - 1; z >= 0; --z) w = fma2(w, zz, lds_f32x2(&pc.c[d][p][z]));
  return w;
}

// Node data of one chunk of 32 nodes of a work item (lane i: node base + i),
// loaded one chunk ahead of its use so that the load latency overlaps the
// current chunk's work (the kernels are latency-bound: one warp per item).
struct Chunk2d {
  int c0 = 0, c1 = 0, j = 0;  // cells, caller index
  float t0 = 0.f, t1 = 0.f;   // fractions
  __device__ __forceinline__ void load(const int* __restrict__ cell, const float* __restrict__ frac,
                                       const int* __restrict__ perm, int64_t M, const int4& item, int base,
                                       int lane) {
    if (base + lane < item.z) {
      const int q = item.y + base + lane;
      c0 = cell[q];
      c1 = cell[M + q];
      t0 = frac[q];
      t1 = frac[M + q];
      j = perm[q];
    }
  }
};

struct Stage2d {
  float w0[32][k2Taps];   // by slot (paired in registers: half the shared wavefronts of stored pairs)
  float w1[32][k2Taps];
  f32x2 v[32];
  int a1[32];
  Poly2d pc;
};

// Compensation terms (COMP: one per accumulator, TwoSum; else unused).
template <bool COMP>
struct Comp2d {
  f32x2 c[COMP ? k2Lines : 1];
};

template <int A0, bool COMP>
__device__ __forceinline__ void scatter2d_bin(const Stage2d& st, int s0, int s1, int lane,
                                              f32x2 (&acc)[k2Lines], Comp2d<COMP>& cp) {
  if constexpr (A0 + k2Taps <= k2Lines) {
    for (int s = s0; s < s1; ++s) {
      const int i1 = lane - st.a1[s];
      const float wv = st.w1[s][i1 & (k2Taps - 1)];
      const float p = (unsigned)i1 < (unsigned)k2Taps ? wv : 0.f;
      const f32x2 vp = mul2(st.v[s], pack2(p, p));
      const float4* wq = reinterpret_cast<const float4*>(&st.w0[s][0]);
#pragma unroll
      for (int q = 0; q < k2Taps / 4; ++q) {
        const float4 x = wq[q];
        const float xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if constexpr (COMP)
            two_sum_acc2(acc[A0 + 4 * q + j], cp.c[A0 + 4 * q + j], mul2(vp, pack2(xs[j], xs[j])));
          else
            acc[A0 + 4 * q + j] = fma2(vp, pack2(xs[j], xs[j]), acc[A0 + 4 * q + j]);
        }
      }
    }
  }
}

// One work item of one problem, by one warp.
template <bool COMP>
__device__ __forceinline__ void scatter2d_item(const Geometry& g, float2* __restrict__ grid,
                                               const int* __restrict__ cell, const float* __restrict__ frac,
                                               const int* __restrict__ perm, const float2* __restrict__ fhat,
                                               const float* __restrict__ poly, const int4& item, Stage2d& st,
                                               int lane) {
  const int64_t M = g.M;
  int tc[2];
  tile_coords<2>(g, item.x, tc);
  const int start0 = tc[0] * g.T[0] + g.off, start1 = tc[1] * g.T[1] + g.off;
  const unsigned lt = (1u << lane) - 1u;
  f32x2 acc[k2Lines];
  Comp2d<COMP> cp;
#pragma unroll
  for (int r = 0; r < k2Lines; ++r) acc[r] = pack2(0.f, 0.f);
  if constexpr (COMP) {
#pragma unroll
    for (int r = 0; r < k2Lines; ++r) cp.c[r] = pack2(0.f, 0.f);
  }
  Chunk2d next;
  next.load(cell, frac, perm, M, item, 0, lane);
  __syncwarp();  // the previous item's coefficients are no longer read
  load_poly2d(poly, st.pc, lane);

  for (int base = 0; base < item.z; base += 32) {
    const bool valid = base + lane < item.z;
    const Chunk2d cur = next;
    const float2 v = valid ? fhat[cur.j] : make_float2(0.f, 0.f);
    const int a0 = valid ? cur.c0 - tc[0] * g.T[0] : -1;
    if (base + 32 < item.z) next.load(cell, frac, perm, M, item, base + 32, lane);
    // counting sort of the chunk by a0 (ballots): bin starts bs[], own slot
    int bs[k2Bins + 1];
    int slot = 0, run = 0;
#pragma unroll
    for (int b = 0; b < k2Bins; ++b) {
      const unsigned m = __ballot_sync(0xffffffffu, a0 == b);
      bs[b] = run;
      if (a0 == b) slot = run + __popc(m & lt);
      run += __popc(m);
    }
    bs[k2Bins] = run;
    __syncwarp();  // the previous chunk's stage is no longer read
    if (valid) {
      // window values straight into the node's slot (one tap pair at a time)
      const float z0 = cur.t0 - 0.5f, z1 = cur.t1 - 0.5f;
      const f32x2 zz0 = pack2(z0, z0), zz1 = pack2(z1, z1);
#pragma unroll
      for (int p = 0; p < k2Pairs; ++p) {
        *reinterpret_cast<float2*>(&st.w0[slot][2 * p]) = unpack2(poly2d_pair(st.pc, 0, p, zz0));
        *reinterpret_cast<float2*>(&st.w1[slot][2 * p]) = unpack2(poly2d_pair(st.pc, 1, p, zz1));
      }
      st.v[slot] = pack2(v.x, v.y);
      st.a1[slot] = cur.c1 - tc[1] * g.T[1];
    }
    __syncwarp();
    scatter2d_bin<0, COMP>(st, bs[0], bs[1], lane, acc, cp);
    scatter2d_bin<1, COMP>(st, bs[1], bs[2], lane, acc, cp);
    scatter2d_bin<2, COMP>(st, bs[2], bs[3], lane, acc, cp);
    scatter2d_bin<3, COMP>(st, bs[3], bs[4], lane, acc, cp);
    scatter2d_bin<4, COMP>(st, bs[4], bs[5], lane, acc, cp);
    scatter2d_bin<5, COMP>(st, bs[5], bs[6], lane, acc, cp);
    scatter2d_bin<6, COMP>(st, bs[6], bs[7], lane, acc, cp);
    scatter2d_bin<7, COMP>(st, bs[7], bs[8], lane, acc, cp);
    scatter2d_bin<8, COMP>(st, bs[8], bs[9], lane, acc, cp);
  }
  if constexpr (COMP) {
#pragma unroll
    for (int r = 0; r < k2Lines; ++r) acc[r] = add2(acc[r], cp.c[r]);
  }

  if (lane < g.L[1]) {
    const int g1 = wrap_mod(start1 + lane, g.Nt[1]);
#pragma unroll
    for (int r = 0; r < k2Lines; ++r) {
      if (r < g.L[0]) {
        const int g0 = wrap_mod(start0 + r, g.Nt[0]);
        atomicAdd(grid + (int64_t)g0 * g.Nt[1] + g1, unpack2(acc[r]));
      }
    }
  }
}

// 5 CTAs per SM (96 registers): measured faster than the 4 the compiler
// would otherwise allow with the chunk prefetch's registers.  The compensated
// form (NFFT_FLAG_COMPENSATED) holds twice the accumulators: 3 CTAs per SM.
template <bool COMP>
__global__ void __launch_bounds__(k2Threads, COMP ? 3 : 5)
    scatter2d_regacc_kernel(Geometry g, float2* __restrict__ grid, NodeArrays na, const float* __restrict__ poly,
                            const float2* __restrict__ fhat) {
  __shared__ Stage2d stage[k2Warps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nitems = *na.n_items;
  const float* frac = reinterpret_cast<const float*>(na.frac);
  for (int it = blockIdx.x * k2Warps + warp; it < nitems; it += gridDim.x * k2Warps)
    scatter2d_item<COMP>(g, grid, na.cell, frac, na.perm, fhat, poly, na.items[it], stage[warp], lane);
}

__global__ void __launch_bounds__(k2Threads, 5)
    scatter2d_regacc_batch_kernel(const BatchProblem* __restrict__ probs, float2* __restrict__ grid, BatchNodes nb,
                                  const float* __restrict__ poly, const float2* __restrict__ fhat) {
  __shared__ Stage2d stage[k2Warps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nitems = *nb.n_items;
  const float* frac = reinterpret_cast<const float*>(nb.frac);
  for (int it = blockIdx.x * k2Warps + warp; it < nitems; it += gridDim.x * k2Warps) {
    const int4 item = nb.items[it];
    const BatchProblem& P = probs[item.w];
    scatter2d_item<false>(P.g, grid + P.grid_off, nb.cell + 2 * P.node_off, frac + 2 * P.node_off,
                          nb.perm + P.node_off, fhat + P.out_off, poly + P.poly_off, item, stage[warp], lane);
  }
}

struct GTile2d {
  // the region, row pitch 33 complex: with a pitch of 32 every row starts on
  // the same bank, so a lane's tap (a0 + i0, a1 + i1) fell on bank pair
  // (a1 + i1) mod 16 whatever its row, and lanes whose nodes share a1 mod 16
  // conflicted; one extra complex per row shifts row r by r bank pairs
  float2 t[k2Lines][k2Cols + 1];
  Poly2d pc;
};

// One work item of one problem (gather), by one warp.
__device__ __forceinline__ void gather2d_item(const Geometry& g, const float2* __restrict__ grid,
                                              const int* __restrict__ cell, const float* __restrict__ frac,
                                              const int* __restrict__ perm, float2* __restrict__ fhat,
                                              const float* __restrict__ poly, const int4& item, GTile2d& tl,
                                              int lane) {
  const int64_t M = g.M;
  int tc[2];
  tile_coords<2>(g, item.x, tc);
  const int start0 = tc[0] * g.T[0] + g.off, start1 = tc[1] * g.T[1] + g.off;
  Chunk2d next;  // the first chunk's node data in flight with the region loads
  next.load(cell, frac, perm, M, item, 0, lane);
  __syncwarp();  // the previous item's tile is no longer read
  if (lane < g.L[1]) {
    const int g1 = wrap_mod(start1 + lane, g.Nt[1]);
#pragma unroll
    for (int r = 0; r < k2Lines; ++r)  // independent loads in flight together
      if (r < g.L[0]) tl.t[r][lane] = grid[(int64_t)wrap_mod(start0 + r, g.Nt[0]) * g.Nt[1] + g1];
  }
  load_poly2d(poly, tl.pc, lane);
  __syncwarp();
  for (int base = 0; base < item.z; base += 32) {
    const bool valid = base + lane < item.z;
    const int a0 = valid ? next.c0 - tc[0] * g.T[0] : 0, a1 = valid ? next.c1 - tc[1] * g.T[1] : 0;
    const float z0 = next.t0 - 0.5f, z1 = next.t1 - 0.5f;
    const int jout = next.j;
    if (base + 32 < item.z) next.load(cell, frac, perm, M, item, base + 32, lane);
    const f32x2 zz0 = pack2(z0, z0), zz1 = pack2(z1, z1);
    float w0[k2Taps];
    f32x2 w1p[k2Taps];
#pragma unroll
    for (int p = 0; p < k2Pairs; ++p) {
      const float2 a = unpack2(poly2d_pair(tl.pc, 0, p, zz0)), b = unpack2(poly2d_pair(tl.pc, 1, p, zz1));
      w0[2 * p] = a.x;
      w0[2 * p + 1] = a.y;
      w1p[2 * p] = pack2(b.x, b.x);
      w1p[2 * p + 1] = pack2(b.y, b.y);
    }
    f32x2 acc = pack2(0.f, 0.f);
#pragma unroll
    for (int i0 = 0; i0 < k2Taps; ++i0) {
      const f32x2* row = reinterpret_cast<const f32x2*>(&tl.t[a0 + i0][a1]);
      f32x2 sum = mul2(row[0], w1p[0]);
#pragma unroll
      for (int i1 = 1; i1 < k2Taps; ++i1) sum = fma2(row[i1], w1p[i1], sum);
      acc = fma2(sum, pack2(w0[i0], w0[i0]), acc);
    }
    if (valid) fhat[jout] = unpack2(acc);
  }
}

// 9 CTAs per SM (at most 56 registers): the occupancy the gather was
// measured at; the kernel is latency-bound.
__global__ void __launch_bounds__(k2Threads, 9)
    gather2d_warp_kernel(Geometry g, const float2* __restrict__ grid, NodeArrays na, const float* __restrict__ poly,
                         float2* __restrict__ fhat) {
  __shared__ GTile2d tiles[k2Warps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nitems = *na.n_items;
  const float* frac = reinterpret_cast<const float*>(na.frac);
  for (int it = blockIdx.x * k2Warps + warp; it < nitems; it += gridDim.x * k2Warps)
    gather2d_item(g, grid, na.cell, frac, na.perm, fhat, poly, na.items[it], tiles[warp], lane);
}

__global__ void __launch_bounds__(k2Threads, 9)
    gather2d_warp_batch_kernel(const BatchProblem* __restrict__ probs, const float2* __restrict__ grid,
                               BatchNodes nb, const float* __restrict__ poly, float2* __restrict__ fhat) {
  __shared__ GTile2d tiles[k2Warps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nitems = *nb.n_items;
  const float* frac = reinterpret_cast<const float*>(nb.frac);
  for (int it = blockIdx.x * k2Warps + warp; it < nitems; it += gridDim.x * k2Warps) {
    const int4 item = nb.items[it];
    const BatchProblem& P = probs[item.w];
    gather2d_item(P.g, grid + P.grid_off, nb.cell + 2 * P.node_off, frac + 2 * P.node_off, nb.perm + P.node_off,
                  fhat + P.out_off, poly + P.poly_off, item, tiles[warp], lane);
  }
}

}  // namespace

bool scatter2d_supported(const Geometry& g) {
  if (g.D != 2 || g.K != k2Taps || g.closed || g.off != -3 || g.m != 4.0) return false;
  return g.T[0] <= k2Lines + 1 - k2Taps && g.L[1] <= k2Cols && g.T[0] <= g.Nt[0] - k2Taps + 1 &&
         g.T[1] <= g.Nt[1] - k2Taps + 1;
}

int scatter2d_ctas_per_sm(int compensated) {
  int n = 0;
  const void* k = compensated ? (const void*)scatter2d_regacc_kernel<true> : (const void*)scatter2d_regacc_kernel<false>;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, k2Threads, 0) != cudaSuccess) return 0;
  return n;
}

cudaError_t launch_scatter2d_fast(const Geometry& g, void* grid, const NodeArrays& na, const float* poly,
                                  const void* fhat, int compensated, int ctas, cudaStream_t s) {
  if (compensated)
    scatter2d_regacc_kernel<true><<<ctas, k2Threads, 0, s>>>(g, (float2*)grid, na, poly, (const float2*)fhat);
  else
    scatter2d_regacc_kernel<false><<<ctas, k2Threads, 0, s>>>(g, (float2*)grid, na, poly, (const float2*)fhat);
  return cudaGetLastError();
}

cudaError_t launch_scatter2d_fast_batch(const BatchProblem* probs, void* grid, const BatchNodes& nb,
                                        const float* poly, const void* fhat, int ctas, cudaStream_t s) {
  scatter2d_regacc_batch_kernel<<<ctas, k2Threads, 0, s>>>(probs, (float2*)grid, nb, poly, (const float2*)fhat);
  return cudaGetLastError();
}

int gather2d_ctas_per_sm() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, gather2d_warp_kernel, k2Threads, 0) != cudaSuccess) return 0;
  return n;
}

cudaError_t launch_gather2d_fast(const Geometry& g, const void* grid, const NodeArrays& na, const float* poly,
                                 void* fhat, int ctas, cudaStream_t s) {
  gather2d_warp_kernel<<<ctas, k2Threads, 0, s>>>(g, (const float2*)grid, na, poly, (float2*)fhat);
  return cudaGetLastError();
}

cudaError_t launch_gather2d_fast_batch(const BatchProblem* probs, const void* grid, const BatchNodes& nb,
                                       const float* poly, void* fhat, int ctas, cudaStream_t s) {
  gather2d_warp_batch_kernel<<<ctas, k2Threads, 0, s>>>(probs, (const float2*)grid, nb, poly, (float2*)fhat);
  return cudaGetLastError();
}

}  // namespace nfftgb
