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
//    over i0, then the half reduces its 16 partial sums;
//  * scatter: four warps share one accumulator tile, warp w updating only the
//    planes i0 with (a0 + i0) = w (mod 4), so no two warps touch the same
//    element and the read-modify-writes need no atomics; the tile (block plus
//    halo) is then added to the grid with vector global reductions;
//  * the node records of a work item are staged in shared memory with the tile.
#include "nfft_internal.cuh"

namespace nfftgb {
namespace {

constexpr int kTaps = 8;
constexpr int kDeg = 8;             // polynomial degree 2m
constexpr int kCoef = kDeg + 1;
constexpr int kPitch = 18;          // shared row pitch (complex) along dim 2
constexpr int kMaxTile2 = 9;        // L2 = T2 + 7 <= 16: two rows per warp step
constexpr int kGatherWarps = 4;
constexpr int kScatterWarps = 4;
constexpr int kItemCap = 128;       // nodes per work item staged in shared memory

struct NodeStage {
  float4 rec[kItemCap];  // {t0, t1, t2, bits of a0 | a1 << 8 | a2 << 16}: fractions, cell offsets in the tile
  int perm[kItemCap];
  float2 v[kItemCap];    // scatter: the node's fhat value
};

// Packed pairs of FP32 (re, im) in one 64-bit register.
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pack2(float x, float y) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
  return r;
}
__device__ __forceinline__ float2 unpack2(f32x2 v) {
  float2 d;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(v));
  return d;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

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
    ns.rec[i] = make_float4(t[0], t[1], t[2], __int_as_float(pk));
    const int j = na.perm[q];
    ns.perm[i] = j;
    if (fhat) ns.v[i] = fhat[j];
  }
}

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Tile + halo rows: two rows of <= 16 elements per warp step, copied with
// cp.async (the caller waits with cp_async_wait_all before its barrier).
__device__ __forceinline__ void load_tile(const Geometry& g, const int* start, const float2* grid,
                                          float2* tile, int warp, int lane, int nwarps) {
  const int L1 = g.L[1], L2 = g.L[2];
  const int half = lane >> 4, e = lane & 15;
  const int rows = g.L[0] * L1;
  const int step = 2 * nwarps;  // rows advance by `step` (< L1 is not assumed)
  const int g2 = wrap1(start[2] + e, g.Nt[2]);
  int r = 2 * warp + half;
  int r0 = r / L1, r1 = r - r0 * L1;
  const int s0 = step / L1, s1 = step - s0 * L1;
  if (e < L2) {
    for (; r < rows; r += step) {
      const int g0 = wrap1(start[0] + r0, g.Nt[0]);
      const int g1 = wrap1(start[1] + r1, g.Nt[1]);
      cp_async8(tile + (r0 * L1 + r1) * kPitch + e, grid + ((int64_t)g0 * g.Nt[1] + g1) * g.Nt[2] + g2);
      r0 += s0;
      r1 += s1;
      if (r1 >= L1) {
        r1 -= L1;
        ++r0;
      }
    }
  }
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(32 * kGatherWarps)
    gather3d_m4_kernel(Geometry g, const float2* __restrict__ grid, NodeArrays na,
                       const float* __restrict__ poly, float2* __restrict__ fhat) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  NodeStage& ns = *reinterpret_cast<NodeStage*>(smem_raw);
  float2* tile = reinterpret_cast<float2*>(smem_raw + sizeof(NodeStage));
  const int L1 = g.L[1];
  const int plane = L1 * kPitch;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int half = lane >> 4, lane16 = lane & 15;
  const int grp = lane16 >> 3, i2 = lane & 7;
  const int hbase = 16 * half;
  // lane evaluates tap i2 of dimension grp (weights wA) and of dimension 2 (wB)
  float cA[kCoef], cB[kCoef];
  load_coef(poly, grp, i2, cA);
  load_coef(poly, 2, i2, cB);
  const int nitems = *na.n_items;

  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int4 item = na.items[it];
    int tc[3], start[3];
    tile_origin(g, item.x, tc);
#pragma unroll
    for (int d = 0; d < 3; ++d) start[d] = tc[d] * g.T[d] + g.off;

    __syncthreads();
    load_tile(g, start, grid, tile, warp, lane, kGatherWarps);
    stage_nodes(g, na, item, tc, ns, nullptr, threadIdx.x, blockDim.x);
    cp_async_wait_all();
    __syncthreads();

    for (int s0 = 2 * warp; s0 < item.z; s0 += 2 * kGatherWarps) {
      const int s = min(s0 + half, item.z - 1);  // a half without a node repeats the last one
      const float4 rc = ns.rec[s];
      const float wA = horner(cA, (grp == 0 ? rc.x : rc.y) - 0.5f);
      const float wB = horner(cB, rc.z - 0.5f);
      const int pk = __float_as_int(rc.w);
      const int a0 = pk & 0xff, a1 = (pk >> 8) & 0xff, a2 = pk >> 16;
      f32x2 w12[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float w = __shfl_sync(0xffffffffu, wA, hbase + 8 + j + 4 * grp) * wB;
        w12[j] = pack2(w, w);
      }
      const f32x2* p = reinterpret_cast<const f32x2*>(tile + (a0 * L1 + a1 + 4 * grp) * kPitch + a2 + i2);
      f32x2 acc = pack2(0.f, 0.f);
#pragma unroll
      for (int i0 = 0; i0 < kTaps; ++i0) {
        const float w0 = __shfl_sync(0xffffffffu, wA, hbase + i0);
        const f32x2* q = p + i0 * plane;
        f32x2 sum = mul2(q[0], w12[0]);
        sum = fma2(q[kPitch], w12[1], sum);
        sum = fma2(q[2 * kPitch], w12[2], sum);
        sum = fma2(q[3 * kPitch], w12[3], sum);
        acc = fma2(sum, pack2(w0, w0), acc);
      }
      float2 r = unpack2(acc);
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        r.x += __shfl_xor_sync(0xffffffffu, r.x, o);
        r.y += __shfl_xor_sync(0xffffffffu, r.y, o);
      }
      if (lane16 == 0 && s0 + half < item.z) fhat[ns.perm[s]] = r;
    }
  }
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(32 * kScatterWarps)
    scatter3d_m4_kernel(Geometry g, float2* __restrict__ grid, NodeArrays na,
                        const float* __restrict__ poly, const float2* __restrict__ fhat) {
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
      const float4 rc = ns.rec[s];
      const float w = horner(c, (dl == 0 ? rc.x : (dl == 1 ? rc.y : rc.z)) - 0.5f);
      const int pk = __float_as_int(rc.w);
      const int a0 = pk & 0xff, a1 = (pk >> 8) & 0xff, a2 = pk >> 16;
      const int i0a = (warp - a0) & (kScatterWarps - 1);  // planes i0a, i0a + 4 are this warp's
      const float w2 = __shfl_sync(0xffffffffu, w, 16 + i2);
      const float wa = __shfl_sync(0xffffffffu, w, 8 + ra) * w2;
      const float wb = __shfl_sync(0xffffffffu, w, 8 + rb) * w2;
      const float w0a = __shfl_sync(0xffffffffu, w, i0a);
      const float w0b = __shfl_sync(0xffffffffu, w, i0a + 4);
      const float2 v = ns.v[s];
      const f32x2 vv = pack2(v.x, v.y);
      f32x2* pa = reinterpret_cast<f32x2*>(acc + ((a0 + i0a) * L1 + a1 + ra) * kPitch + a2 + i2);
      f32x2* pb = pa + 2 * kPitch;
      const f32x2 t0 = pa[0], t1 = pb[0], t2 = pa[4 * plane], t3 = pb[4 * plane];
      pa[0] = fma2(vv, pack2(wa * w0a, wa * w0a), t0);
      pb[0] = fma2(vv, pack2(wb * w0a, wb * w0a), t1);
      pa[4 * plane] = fma2(vv, pack2(wa * w0b, wa * w0b), t2);
      pb[4 * plane] = fma2(vv, pack2(wb * w0b, wb * w0b), t3);
      __syncwarp();
    }
    __syncthreads();

    // add block + halo back to the grid (periodic wrap only here)
    {
      const int half = lane >> 4, e = lane & 15;
      const int rows = L0 * L1;
      const int g2 = wrap1(start[2] + e, g.Nt[2]);
      for (int r = 2 * warp + half; r < rows; r += 2 * kScatterWarps) {
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

template <typename K>
cudaError_t set_smem(K kern, size_t smem) {
  if (smem > 48 * 1024)
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaSuccess;
}

}  // namespace

bool fast3d_supported(const Geometry& g, int cmax) {
  if (g.D != 3 || g.K != kTaps || g.closed || g.off != -3) return false;
  if (g.T[2] > kMaxTile2 || cmax > kItemCap) return false;
  for (int d = 0; d < 3; ++d)
    if (g.T[d] > g.Nt[d] - kTaps + 1 || g.L[d] > 255) return false;
  return smem_bytes(g) <= 200 * 1024;
}

int fast3d_ctas_per_sm(const Geometry& g, int kind) {
  const size_t smem = smem_bytes(g);
  void* k = kind == 0 ? (void*)gather3d_m4_kernel : (void*)scatter3d_m4_kernel;
  const int threads = kind == 0 ? 32 * kGatherWarps : 32 * kScatterWarps;
  if (set_smem(k, smem) != cudaSuccess) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, smem) != cudaSuccess) return 0;
  return n;
}

cudaError_t launch_gather3d_fast(const Geometry& g, const void* grid, const NodeArrays& na,
                                 const float* poly, void* fhat, int ctas, cudaStream_t s) {
  const size_t smem = smem_bytes(g);
  cudaError_t e = set_smem(gather3d_m4_kernel, smem);
  if (e != cudaSuccess) return e;
  gather3d_m4_kernel<<<ctas, 32 * kGatherWarps, smem, s>>>(g, (const float2*)grid, na, poly,
                                                          (float2*)fhat);
  return cudaGetLastError();
}

cudaError_t launch_scatter3d_fast(const Geometry& g, void* grid, const NodeArrays& na,
                                  const float* poly, const void* fhat, int ctas, cudaStream_t s) {
  const size_t smem = smem_bytes(g);
  cudaError_t e = set_smem(scatter3d_m4_kernel, smem);
  if (e != cudaSuccess) return e;
  scatter3d_m4_kernel<<<ctas, 32 * kScatterWarps, smem, s>>>(g, (float2*)grid, na, poly,
                                                            (const float2*)fhat);
  return cudaGetLastError();
}

}  // namespace nfftgb
