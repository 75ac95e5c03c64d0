// 3D resampling kernels for m = 4 (8 taps per dimension), complex64.
//
// Same computation as the generic kernels in resample.cuh (Eq. SumOverNode,
// Eq. SumOverNodeAdjoint, Eq. InnerTensorStructure; Algorithm 3 / 4), laid
// out for the GB300 shared-memory pipe:
//
//  * one warp per node.  Lane l owns taps (i1, i2) = (row(l, 0), l & 7) and
//    (row(l, 1), l & 7) of the 8 x 8 cross-section and loops over i0, so a
//    node's 512 taps are 16 loads per lane.  The row map pairs rows r and
//    r + 4 inside each half-warp; with a row pitch of 18 complex (8 * 18 = 144
//    = 16 mod 32 banks) the two rows of a half-warp land in disjoint 16-bank
//    halves whatever the node's position, so every load is conflict-free.
//  * lanes 0..23 evaluate the node's 24 window values (psi^local_{d,j}, one
//    per lane) and hand them out with shuffles.
//  * complex x real products use packed FP32 FMA (fma.rn.f32x2).
//  * the scatter accumulates into a shared tile private to one warp, so the
//    read-modify-writes need no atomics; the tile (block plus halo) is added
//    back to the grid with vector global reductions.
//  * each work item's node records are staged in shared memory with the tile.
#include "nfft_internal.cuh"

namespace nfftgb {
namespace {

constexpr int kTaps = 8;
constexpr int kPitch = 18;          // shared row pitch (complex) along dim 2
constexpr int kMaxTile2 = 9;        // L2 = T2 + 7 <= 16: two rows per warp step
constexpr int kGatherWarps = 4;
constexpr int kItemCap = 128;       // nodes per work item staged in shared memory

struct NodeStage {
  int a[3][kItemCap];   // cell offset inside the tile, per dimension
  float t[3][kItemCap]; // fraction
  int perm[kItemCap];
  float2 v[kItemCap];   // scatter: fhat value of the node
};

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  unsigned long long ua, ub, uc, ud;
  asm("mov.b64 %0, {%1, %2};" : "=l"(ua) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(ub) : "f"(b.x), "f"(b.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(uc) : "f"(c.x), "f"(c.y));
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(ud) : "l"(ua), "l"(ub), "l"(uc));
  float2 d;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(ud));
  return d;
}

__device__ __forceinline__ int wrap1(int x, int n) {
  // region coordinates lie in [-n, 2n) when tile_d <= N~_d - 7 (checked on the host)
  return x < 0 ? x + n : (x >= n ? x - n : x);
}

// Row map: half-warp h, 8-lane group g = lane >> 3; pass p in {0, 1}.
__device__ __forceinline__ int lane_row(int lane, int pass) {
  const int g = lane >> 3;
  return (g & 1) * 4 + (g >> 1) + 2 * pass;
}

__device__ __forceinline__ void tile_origin(const Geometry& g, int tile, int* tc) {
  tc[2] = tile % g.ntile[2];
  tile /= g.ntile[2];
  tc[1] = tile % g.ntile[1];
  tc[0] = tile / g.ntile[1];
}

// Stage the node records of one work item (CTA-wide).
__device__ __forceinline__ void stage_nodes(const Geometry& g, const NodeArrays& na, const int4& item,
                                            const int* tc, NodeStage& ns, const float2* fhat,
                                            int tid, int nthreads) {
  const int64_t M = g.M;
  const float* frac = reinterpret_cast<const float*>(na.frac);
  for (int i = tid; i < item.z; i += nthreads) {
    const int q = item.y + i;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      ns.a[d][i] = na.cell[d * M + q] - tc[d] * g.T[d];
      ns.t[d][i] = frac[d * M + q];
    }
    const int j = na.perm[q];
    ns.perm[i] = j;
    if (fhat) ns.v[i] = fhat[j];
  }
}

// Window value of lane (d = lane >> 3, tap i = lane & 7) for the node staged at s.
__device__ __forceinline__ float lane_weight(const Geometry& g, const NodeStage& ns, int s, int lane) {
  const int d = min(lane >> 3, 2);
  const int i = lane & 7;
  const float t = ns.t[d][s];
  const float mm_u = float(1 + i) - t;        // m - u, u = t + m - 1 - i
  const float mp_u = float(2 * 4 - 1 - i) + t;  // m + u
  // select instead of indexing the parameter arrays with a lane-dependent d
  const float b = d == 0 ? (float)g.b[0] : (d == 1 ? (float)g.b[1] : (float)g.b[2]);
  const float nm = d == 0 ? (float)g.norm[0] : (d == 1 ? (float)g.norm[1] : (float)g.norm[2]);
  return kb_window<float>(mm_u, mp_u, b, nm);
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(32 * kGatherWarps)
    gather3d_m4_kernel(Geometry g, const float2* __restrict__ grid, NodeArrays na,
                       float2* __restrict__ fhat) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  NodeStage& ns = *reinterpret_cast<NodeStage*>(smem_raw);
  float2* tile = reinterpret_cast<float2*>(smem_raw + sizeof(NodeStage));
  const int L0 = g.L[0], L1 = g.L[1], L2 = g.L[2];
  const int plane = L1 * kPitch;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i2 = lane & 7;
  const int ra = lane_row(lane, 0), rb = lane_row(lane, 1);
  const int nitems = *na.n_items;

  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int4 item = na.items[it];
    int tc[3], start[3];
    tile_origin(g, item.x, tc);
#pragma unroll
    for (int d = 0; d < 3; ++d) start[d] = tc[d] * g.T[d] + g.off;

    __syncthreads();
    // tile + halo: two rows of <= 16 elements per warp step
    {
      const int half = lane >> 4, e = lane & 15;
      const int rows = L0 * L1;
      const int g2 = wrap1(start[2] + e, g.Nt[2]);
#pragma unroll 4
      for (int r = 2 * warp + half; r < rows; r += 2 * kGatherWarps) {
        const int r0 = r / L1, r1 = r - r0 * L1;
        if (e < L2) {
          const int g0 = wrap1(start[0] + r0, g.Nt[0]);
          const int g1 = wrap1(start[1] + r1, g.Nt[1]);
          tile[(r0 * L1 + r1) * kPitch + e] = grid[((int64_t)g0 * g.Nt[1] + g1) * g.Nt[2] + g2];
        }
      }
    }
    stage_nodes(g, na, item, tc, ns, nullptr, threadIdx.x, blockDim.x);
    __syncthreads();

    for (int s = warp; s < item.z; s += kGatherWarps) {
      const float w = lane_weight(g, ns, s, lane);
      const int a0 = ns.a[0][s], a1 = ns.a[1][s], a2 = ns.a[2][s];
      const float w2 = __shfl_sync(0xffffffffu, w, 16 + i2);
      const float wa = __shfl_sync(0xffffffffu, w, 8 + ra) * w2;
      const float wb = __shfl_sync(0xffffffffu, w, 8 + rb) * w2;
      const float2* pa = tile + (a0 * L1 + a1 + ra) * kPitch + a2 + i2;
      const float2* pb = pa + (rb - ra) * kPitch;
      const float2 wwa = make_float2(wa, wa), wwb = make_float2(wb, wb);
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int i0 = 0; i0 < kTaps; ++i0) {
        const float w0 = __shfl_sync(0xffffffffu, w, i0);
        const float2 va = pa[i0 * plane];
        const float2 vb = pb[i0 * plane];
        float2 sum = ffma2(va, wwa, make_float2(0.f, 0.f));
        sum = ffma2(vb, wwb, sum);
        acc = ffma2(sum, make_float2(w0, w0), acc);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
      }
      if (lane == 0) fhat[ns.perm[s]] = acc;
    }
  }
}

// ---------------------------------------------------------------------------
// One warp per CTA: the accumulator tile is private to the warp.
__global__ void __launch_bounds__(32)
    scatter3d_m4_kernel(Geometry g, float2* __restrict__ grid, NodeArrays na,
                        const float2* __restrict__ fhat) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  NodeStage& ns = *reinterpret_cast<NodeStage*>(smem_raw);
  float2* acc = reinterpret_cast<float2*>(smem_raw + sizeof(NodeStage));
  const int L0 = g.L[0], L1 = g.L[1], L2 = g.L[2];
  const int plane = L1 * kPitch;
  const int lane = threadIdx.x;
  const int i2 = lane & 7;
  const int ra = lane_row(lane, 0), rb = lane_row(lane, 1);
  const int nitems = *na.n_items;
  const int n4 = (L0 * plane) / 2;  // float4 count (pitch is even)

  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int4 item = na.items[it];
    int tc[3], start[3];
    tile_origin(g, item.x, tc);
#pragma unroll
    for (int d = 0; d < 3; ++d) start[d] = tc[d] * g.T[d] + g.off;

    __syncwarp();
    float4* acc4 = reinterpret_cast<float4*>(acc);
    for (int e = lane; e < n4; e += 32) acc4[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    stage_nodes(g, na, item, tc, ns, fhat, lane, 32);
    __syncwarp();

    for (int s = 0; s < item.z; ++s) {
      const float w = lane_weight(g, ns, s, lane);
      const int a0 = ns.a[0][s], a1 = ns.a[1][s], a2 = ns.a[2][s];
      const float2 v = ns.v[s];
      const float w2 = __shfl_sync(0xffffffffu, w, 16 + i2);
      const float wa = __shfl_sync(0xffffffffu, w, 8 + ra) * w2;
      const float wb = __shfl_sync(0xffffffffu, w, 8 + rb) * w2;
      const float2 va = make_float2(v.x * wa, v.y * wa);
      const float2 vb = make_float2(v.x * wb, v.y * wb);
      float2* pa = acc + (a0 * L1 + a1 + ra) * kPitch + a2 + i2;
      float2* pb = pa + (rb - ra) * kPitch;
      float2 ta[kTaps], tb[kTaps];
#pragma unroll
      for (int i0 = 0; i0 < kTaps; ++i0) {
        ta[i0] = pa[i0 * plane];
        tb[i0] = pb[i0 * plane];
      }
#pragma unroll
      for (int i0 = 0; i0 < kTaps; ++i0) {
        const float w0 = __shfl_sync(0xffffffffu, w, i0);
        const float2 ww0 = make_float2(w0, w0);
        ta[i0] = ffma2(va, ww0, ta[i0]);
        tb[i0] = ffma2(vb, ww0, tb[i0]);
      }
#pragma unroll
      for (int i0 = 0; i0 < kTaps; ++i0) {
        pa[i0 * plane] = ta[i0];
        pb[i0 * plane] = tb[i0];
      }
      __syncwarp();
    }

    // add block + halo back to the grid (periodic wrap only here)
    {
      const int half = lane >> 4, e = lane & 15;
      const int rows = L0 * L1;
      const int g2 = wrap1(start[2] + e, g.Nt[2]);
      for (int r = half; r < rows; r += 2) {
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

size_t smem_bytes(const Geometry& g) {
  return sizeof(NodeStage) + (size_t)g.L[0] * g.L[1] * kPitch * sizeof(float2);
}

}  // namespace

bool fast3d_supported(const Geometry& g, int cmax) {
  if (g.D != 3 || g.K != kTaps || g.closed) return false;
  if (g.T[2] > kMaxTile2 || cmax > kItemCap) return false;
  for (int d = 0; d < 3; ++d)
    if (g.T[d] > g.Nt[d] - kTaps + 1) return false;
  return smem_bytes(g) <= 200 * 1024;
}

int fast3d_ctas_per_sm(const Geometry& g, int kind) {
  const size_t smem = smem_bytes(g);
  void* k = kind == 0 ? (void*)gather3d_m4_kernel : (void*)scatter3d_m4_kernel;
  const int threads = kind == 0 ? 32 * kGatherWarps : 32;
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, smem) != cudaSuccess) return 0;
  return n;
}

cudaError_t launch_gather3d_fast(const Geometry& g, const void* grid, const NodeArrays& na, void* fhat,
                                 int ctas, cudaStream_t s) {
  const size_t smem = smem_bytes(g);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(gather3d_m4_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  gather3d_m4_kernel<<<ctas, 32 * kGatherWarps, smem, s>>>(g, (const float2*)grid, na, (float2*)fhat);
  return cudaGetLastError();
}

cudaError_t launch_scatter3d_fast(const Geometry& g, void* grid, const NodeArrays& na, const void* fhat,
                                  int ctas, cudaStream_t s) {
  const size_t smem = smem_bytes(g);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(scatter3d_m4_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  scatter3d_m4_kernel<<<ctas, 32, smem, s>>>(g, (float2*)grid, na, (const float2*)fhat);
  return cudaGetLastError();
}

}  // namespace nfftgb
