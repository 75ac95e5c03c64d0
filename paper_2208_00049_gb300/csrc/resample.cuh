// Block-partitioned resampling kernels (gather, scatter, node-gradient gather).
//
// arXiv 2208.00049:
//   * Eq. SumOverNode / Eq. SumOverNodeAdjoint: the direct resampling sums
//     ghat_l psi~(k_j - l/N~) over the footprint I_{N~,m}(k_j); the adjoint
//     adds fhat_j psi~(k_j - l/N~) into it.
//   * Eq. InnerTensorStructure: the footprint sum is evaluated as nested
//     one-dimensional sums with per-node local weight vectors psi^local_{d,j}
//     (2m window values per dimension), so a node costs O(mD) window
//     evaluations and O((2m)^D) multiply-adds.
//   * Algorithm 3 / Algorithm 4 (Sec. 3.7.3): nodes are grouped by grid block
//     R_p; the block plus its halo (Q + 2m cells per dimension) is copied to a
//     local cache, resampled there, and for the adjoint added back to the grid.
//     The index wrap is handled only when copying in / adding back.
//
// GB300 realisation: one CTA per work item (a tile and a slice of its sorted
// nodes).  The tile plus halo lives in shared memory; one thread evaluates one
// node's local weights and its nested tensor sum.  The adjoint accumulates in
// shared memory with shared atomics (optionally TwoSum-compensated) and adds
// the tile back to the grid with vector global atomics -- the mutex of
// Algorithm 4 becomes per-element atomic reductions in L2.
#pragma once

#include "nfft_internal.cuh"

namespace nfftgb {

template <typename R>
struct CplxT;
template <>
struct CplxT<float> {
  using type = float2;
};
template <>
struct CplxT<double> {
  using type = double2;
};

// Periodic wrap of a grid coordinate.  Region coordinates lie in
// [-m, 2 N~ + m) (a partial last tile plus its halo can pass N~ by more than
// one period's worth of halo), so a full modulo is used.
__device__ __forceinline__ int wrap_mod(int x, int n) {
  x %= n;
  return x < 0 ? x + n : x;
}

template <int D>
__device__ __forceinline__ void tile_coords(const Geometry& g, int t, int* tc) {
#pragma unroll
  for (int d = D - 1; d >= 0; --d) {
    tc[d] = t % g.ntile[d];
    t /= g.ntile[d];
  }
}

template <int D>
__device__ __forceinline__ int region_size(const Geometry& g) {
  int r = 1;
#pragma unroll
  for (int d = 0; d < D; ++d) r *= g.L[d];
  return r;
}

// Global linear index of region element e of the tile whose region starts at
// `start` (periodic wrap applied per dimension).
template <int D>
__device__ __forceinline__ int64_t region_to_grid(const Geometry& g, const int* start, int e) {
  int a[kMaxD];
#pragma unroll
  for (int d = D - 1; d >= 0; --d) {
    a[d] = e % g.L[d];
    e /= g.L[d];
  }
  int64_t lin = 0;
#pragma unroll
  for (int d = 0; d < D; ++d) lin = lin * g.Nt[d] + wrap_mod(start[d] + a[d], g.Nt[d]);
  return lin;
}

// LINEAR window (Sec. 3.7.4, Eq. linInterp): kappa = |u| (S - 2)/m, s =
// floor(kappa), alpha = kappa - s, w = tab[s] + alpha (tab[s + 1] - tab[s]);
// (S - 2)/m is a power of two, so kappa is |u| scaled exactly.  Also returns
// the slope of the segment in *slope (d w / d|u|).
template <typename R>
__device__ __forceinline__ R lut_window(const R* __restrict__ tab, int S, R scale, R u, R* slope) {
  const R kappa = fabs(u) * scale;
  int s = (int)kappa;
  s = s < S - 2 ? s : S - 2;
  const R alpha = kappa - R(s);
  const R lo = tab[s], hi = tab[s + 1];
  if (slope) *slope = (hi - lo) * scale;
  return lo + alpha * (hi - lo);
}

// Window values of the table modes (kWinLinear, kWinPoly) for the K taps of
// one dimension, and their derivatives d/dk if dw != nullptr.  Out of line:
// the modes share one copy instead of being inlined at every call site of
// the unrolled kernels.
template <int K, typename R>
__device__ __noinline__ void table_weights(const Geometry& g, int d, int mi, R t, R* w, R* dw) {
  if (g.wmode == kWinLinear) {
    const R* tab = (const R*)g.wtab + (int64_t)d * g.wS;
    const R scale = R(g.wS - 2) / R(mi);
    for (int i = 0; i < K; ++i) {
      const R u = R(-g.off - i) + t;
      R slope;
      R v = lut_window<R>(tab, g.wS, scale, u, &slope);
      R dv = (u < R(0) ? -slope : slope) * R(g.Nt[d]);
      if (g.closed && ((i == 0 && t != R(0)) || i == K - 1)) v = dv = R(0);
      w[i] = v;
      if (dw) dw[i] = dv;
    }
  } else {
    const int Z = g.wZ;
    const R* pc = (const R*)g.wtab + (int64_t)d * K * Z;
    const R zeta = t - R(0.5);
    for (int i = 0; i < K; ++i) {
      R v = pc[i * Z + Z - 1], dv = R(0);
      for (int z = Z - 2; z >= 0; --z) {
        dv = dv * zeta + v;
        v = v * zeta + pc[i * Z + z];
      }
      w[i] = v;
      if (dw) dw[i] = dv * R(g.Nt[d]);
    }
  }
}

// Local weight vector psi^local_{d,j} (Eq. InnerTensorStructure) for one
// dimension: tap i sits at l' = c + off + i, u = t - off - i.  The window
// values are evaluated (kWinDirect), looked up in the LINEAR table
// (kWinLinear) or taken from the POLYNOMIAL coefficients of tap i
// (kWinPoly, Horner in zeta = t - 1/2).
template <int K, typename R>
__device__ __forceinline__ void node_weights(const Geometry& g, int d, int mi, R t, R* w) {
  if (g.wmode != kWinDirect) {
    R tmp[K];
    table_weights<K, R>(g, d, mi, t, tmp, nullptr);
#pragma unroll
    for (int i = 0; i < K; ++i) w[i] = tmp[i];
    return;
  }
  const R b = R(g.b[d]), norm = R(g.norm[d]), mr = R(mi);
  const R normx = sizeof(R) == 4 ? kb_normx<R>(b, mr) : R(0);
#pragma unroll
  for (int i = 0; i < K; ++i) {
    R u = R(-g.off - i) + t;
    R mm_u = R(mi + g.off + i) - t;  // m - u
    R mp_u = R(mi - g.off - i) + t;  // m + u
    R v = kb_window<R>(u, mm_u, mp_u, b, norm, mr, normx);
    if (g.closed && ((i == 0 && t != R(0)) || i == K - 1)) v = R(0);
    w[i] = v;
  }
}

// d/dk of the local weights: N~_d * w'(u) (for the LINEAR window the slope
// of the interpolant's segment, for the POLYNOMIAL one the derivative of the
// polynomial, d/du = d/dzeta).
template <int K, typename R>
__device__ __forceinline__ void node_weight_derivs(const Geometry& g, int d, int mi, R t, R* dw) {
  if (g.wmode != kWinDirect) {
    R tmp[K], dtmp[K];
    table_weights<K, R>(g, d, mi, t, tmp, dtmp);
#pragma unroll
    for (int i = 0; i < K; ++i) dw[i] = dtmp[i];
    return;
  }
  const R b = R(g.b[d]), norm = R(g.norm[d]) * R(g.Nt[d]), mr = R(mi);
  const R normx = sizeof(R) == 4 ? kb_normx<R>(b, mr) * R(g.Nt[d]) : R(0);
  const R zsmall = sizeof(R) == 4 ? R(0.5) : R(0.05);
#pragma unroll
  for (int i = 0; i < K; ++i) {
    R u = R(-g.off - i) + t;
    R mm_u = R(mi + g.off + i) - t;
    R mp_u = R(mi - g.off - i) + t;
    R v = kb_window_deriv<R>(u, mm_u, mp_u, b, norm, zsmall, mr, normx);
    if (g.closed && ((i == 0 && t != R(0)) || i == K - 1)) v = R(0);
    dw[i] = v;
  }
}

// Window value of tap i alone (the tap-parallel 1D loops below): the same
// value node_weights gives for tap i.
template <int K, typename R>
__device__ __forceinline__ R node_weight_tap(const Geometry& g, int d, int mi, R t, int i) {
  if (g.wmode == kWinPoly) {  // tap i's polynomial alone
    const int Z = g.wZ;
    const R* pc = (const R*)g.wtab + ((int64_t)d * K + i) * Z;
    const R zeta = t - R(0.5);
    R v = pc[Z - 1];
    for (int z = Z - 2; z >= 0; --z) v = v * zeta + pc[z];
    return v;
  }
  if (g.wmode != kWinDirect) {
    R tmp[K];
    table_weights<K, R>(g, d, mi, t, tmp, nullptr);
    R v = R(0);
#pragma unroll
    for (int j = 0; j < K; ++j) v = (j == i) ? tmp[j] : v;
    return v;
  }
  const R b = R(g.b[d]), norm = R(g.norm[d]), mr = R(mi);
  const R normx = sizeof(R) == 4 ? kb_normx<R>(b, mr) : R(0);
  const R u = R(-g.off - i) + t;
  const R mm_u = R(mi + g.off + i) - t;
  const R mp_u = R(mi - g.off - i) + t;
  R v = kb_window<R>(u, mm_u, mp_u, b, norm, mr, normx);
  if (g.closed && ((i == 0 && t != R(0)) || i == K - 1)) v = R(0);
  return v;
}

// 1D items run tap-parallel: a group of KP >= K consecutive threads (a
// power of two) takes one node, thread i of the group its tap i.  A node
// costs K window evaluations, and in double precision those dominate: GB300
// issues FP64 arithmetic at a small fraction of the FP32 rate, so one node
// per thread leaves the FP64 units waiting on a few long dependent chains.
template <int K>
struct TapGroup {
  static constexpr int KP = K <= 2 ? 2 : K <= 4 ? 4 : K <= 8 ? 8 : K <= 16 ? 16 : 32;
  static_assert(K <= 32, "tap groups fit a warp");
};

// ---------------------------------------------------------------------------
// Direct resampling (Algorithm 3)
// ---------------------------------------------------------------------------
// One work item (tile + a slice of its sorted nodes) of the direct resampling.
template <int D, int K, typename R>
__device__ __forceinline__ void gather_item(const Geometry& g, const typename CplxT<R>::type* __restrict__ grid,
                                            const NodeArrays& na, const int4 item,
                                            typename CplxT<R>::type* __restrict__ fhat,
                                            typename CplxT<R>::type* tile) {
  using C = typename CplxT<R>::type;
  const R* __restrict__ frac = reinterpret_cast<const R*>(na.frac);
  const int region = region_size<D>(g);
  const int mi = (int)g.m;
  const int64_t M = g.M;
  int tc[kMaxD], start[kMaxD];
  tile_coords<D>(g, item.x, tc);
#pragma unroll
  for (int d = 0; d < D; ++d) start[d] = tc[d] * g.T[d] + g.off;

  __syncthreads();  // the previous item's nodes are done with the tile
  for (int e = threadIdx.x; e < region; e += blockDim.x) tile[e] = grid[region_to_grid<D>(g, start, e)];
  __syncthreads();

  if constexpr (D == 1) {
    constexpr int KP = TapGroup<K>::KP;
    const int per = blockDim.x / KP, jn = threadIdx.x / KP, i = threadIdx.x % KP;
    const int end = item.y + item.z;
    for (int q0 = item.y; q0 < end; q0 += per) {  // uniform over the CTA: the shuffles need whole warps
      const int q = q0 + jn;
      R re = R(0), im = R(0);
      if (q < end && i < K) {
        const int a0 = na.cell[q] - tc[0] * g.T[0];
        const R w = node_weight_tap<K, R>(g, 0, mi, frac[q], i);
        const C v = tile[a0 + i];
        re = w * v.x;
        im = w * v.y;
      }
#pragma unroll
      for (int o = KP / 2; o >= 1; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
      }
      if (q < end && i == 0) {
        C out;
        out.x = re;
        out.y = im;
        fhat[na.perm[q]] = out;
      }
    }
    return;
  }
  for (int q = item.y + threadIdx.x; q < item.y + item.z; q += blockDim.x) {
    R w[D][K];
    int a[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      a[d] = na.cell[d * M + q] - tc[d] * g.T[d];
      node_weights<K, R>(g, d, mi, frac[d * M + q], w[d]);
    }
    R re = R(0), im = R(0);
    if constexpr (D == 2) {
#pragma unroll
      for (int i0 = 0; i0 < K; ++i0) {
        const C* row = tile + (a[0] + i0) * g.L[1] + a[1];
        R sr = R(0), si = R(0);
#pragma unroll
        for (int i1 = 0; i1 < K; ++i1) {
          C v = row[i1];
          sr += w[1][i1] * v.x;
          si += w[1][i1] * v.y;
        }
        re += w[0][i0] * sr;
        im += w[0][i0] * si;
      }
    } else if constexpr (D == 3) {
#pragma unroll 1
      for (int i0 = 0; i0 < K; ++i0) {
        const C* plane = tile + ((a[0] + i0) * g.L[1] + a[1]) * g.L[2] + a[2];
        R s1r = R(0), s1i = R(0);
#pragma unroll
        for (int i1 = 0; i1 < K; ++i1) {
          const C* row = plane + i1 * g.L[2];
          R s2r = R(0), s2i = R(0);
#pragma unroll
          for (int i2 = 0; i2 < K; ++i2) {
            C v = row[i2];
            s2r += w[2][i2] * v.x;
            s2i += w[2][i2] * v.y;
          }
          s1r += w[1][i1] * s2r;
          s1i += w[1][i1] * s2i;
        }
        // w[0] is indexed by a rolled loop: keep the select explicit so the
        // array stays in registers.
        R w0 = R(0);
#pragma unroll
        for (int i = 0; i < K; ++i) w0 = (i == i0) ? w[0][i] : w0;
        re += w0 * s1r;
        im += w0 * s1i;
      }
    }
    C out;
    out.x = re;
    out.y = im;
    fhat[na.perm[q]] = out;
  }
}

template <int D, int K, typename R>
__global__ void __launch_bounds__(kResampleThreads)
    gather_kernel(Geometry g, const typename CplxT<R>::type* __restrict__ grid, NodeArrays na,
                  typename CplxT<R>::type* __restrict__ fhat) {
  using C = typename CplxT<R>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tile = reinterpret_cast<C*>(smem_raw);
  const int nitems = *na.n_items;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x)
    gather_item<D, K, R>(g, grid, na, na.items[it], fhat, tile);
}

// Batched: one persistent launch over the work items of many problems; item.w
// names the problem, whose geometry and buffer offsets come from `probs`.
template <int D, int K, typename R>
__global__ void __launch_bounds__(kResampleThreads)
    gather_batch_kernel(const BatchProblem* __restrict__ probs, const typename CplxT<R>::type* __restrict__ grid,
                        BatchNodes nb, typename CplxT<R>::type* __restrict__ fhat) {
  using C = typename CplxT<R>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tile = reinterpret_cast<C*>(smem_raw);
  const int nitems = *nb.n_items;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int4 item = nb.items[it];
    const BatchProblem& P = probs[item.w];
    const Geometry g = P.g;
    NodeArrays na;
    na.cell = nb.cell + D * P.node_off;
    na.frac = reinterpret_cast<const R*>(nb.frac) + D * P.node_off;
    na.perm = nb.perm + P.node_off;
    gather_item<D, K, R>(g, grid + P.grid_off, na, item, fhat + P.out_off, tile);
  }
}

// ---------------------------------------------------------------------------
// Adjoint resampling (Algorithm 4)
// ---------------------------------------------------------------------------
template <typename R, bool COMP>
__device__ __forceinline__ void smem_add(R* acc, R* comp, int idx, R x) {
  if constexpr (!COMP) {
    atomicAdd(acc + idx, x);
  } else {
    // TwoSum of (old, x): s = old + x as the atomic stored it, err exact.
    R old = atomicAdd(acc + idx, x);
    R s = old + x;
    R bp = s - old;
    R err = (old - (s - bp)) + (x - bp);
    atomicAdd(comp + idx, err);
  }
}

__device__ __forceinline__ void grid_add(float2* p, float re, float im) {
  atomicAdd(p, make_float2(re, im));  // vector red.global.add (sm_90+)
}
__device__ __forceinline__ void grid_add(double2* p, double re, double im) {
  atomicAdd(&p->x, re);
  atomicAdd(&p->y, im);
}

template <int D, int K, typename R, bool COMP>
__device__ __forceinline__ void scatter_item(const Geometry& g, typename CplxT<R>::type* __restrict__ grid,
                                             const NodeArrays& na, const int4 item,
                                             const typename CplxT<R>::type* __restrict__ fhat, R* acc) {
  using C = typename CplxT<R>::type;
  const int region = region_size<D>(g);
  R* comp = acc + (COMP ? 2 * region : 0);  // TwoSum error terms
  const R* __restrict__ frac = reinterpret_cast<const R*>(na.frac);
  const int mi = (int)g.m;
  const int64_t M = g.M;
  int tc[kMaxD], start[kMaxD];
  tile_coords<D>(g, item.x, tc);
#pragma unroll
  for (int d = 0; d < D; ++d) start[d] = tc[d] * g.T[d] + g.off;

  __syncthreads();  // previous flush finished reading the tile
  for (int e = threadIdx.x; e < 2 * region * (COMP ? 2 : 1); e += blockDim.x) acc[e] = R(0);
  __syncthreads();

  if constexpr (D == 1) {
    constexpr int KP = TapGroup<K>::KP;
    const int per = blockDim.x / KP, jn = threadIdx.x / KP, i = threadIdx.x % KP;
    for (int q = item.y + jn; q < item.y + item.z; q += per) {
      if (i < K) {
        const int a0 = na.cell[q] - tc[0] * g.T[0];
        const R w = node_weight_tap<K, R>(g, 0, mi, frac[q], i);
        const C v = fhat[na.perm[q]];
        const int idx = 2 * (a0 + i);
        smem_add<R, COMP>(acc, comp, idx, v.x * w);
        smem_add<R, COMP>(acc, comp, idx + 1, v.y * w);
      }
    }
  }
  for (int q = item.y + threadIdx.x; D > 1 && q < item.y + item.z; q += blockDim.x) {
    R w[D][K];
    int a[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      a[d] = na.cell[d * M + q] - tc[d] * g.T[d];
      node_weights<K, R>(g, d, mi, frac[d * M + q], w[d]);
    }
    const C v = fhat[na.perm[q]];
    if constexpr (D == 2) {
#pragma unroll
      for (int i0 = 0; i0 < K; ++i0) {
        const R vr = v.x * w[0][i0], vi = v.y * w[0][i0];
        const int rowi = (a[0] + i0) * g.L[1] + a[1];
#pragma unroll
        for (int i1 = 0; i1 < K; ++i1) {
          const int idx = 2 * (rowi + i1);
          smem_add<R, COMP>(acc, comp, idx, vr * w[1][i1]);
          smem_add<R, COMP>(acc, comp, idx + 1, vi * w[1][i1]);
        }
      }
    } else if constexpr (D == 3) {
#pragma unroll 1
      for (int i0 = 0; i0 < K; ++i0) {
        R w0 = R(0);
#pragma unroll
        for (int i = 0; i < K; ++i) w0 = (i == i0) ? w[0][i] : w0;
        const R v0r = v.x * w0, v0i = v.y * w0;
        const int planei = ((a[0] + i0) * g.L[1] + a[1]) * g.L[2] + a[2];
#pragma unroll
        for (int i1 = 0; i1 < K; ++i1) {
          const R vr = v0r * w[1][i1], vi = v0i * w[1][i1];
          const int rowi = planei + i1 * g.L[2];
#pragma unroll
          for (int i2 = 0; i2 < K; ++i2) {
            const int idx = 2 * (rowi + i2);
            smem_add<R, COMP>(acc, comp, idx, vr * w[2][i2]);
            smem_add<R, COMP>(acc, comp, idx + 1, vi * w[2][i2]);
          }
        }
      }
    }
  }
  __syncthreads();

  // Add the tile (block plus halo) back to the grid; wrap applied here only.
  for (int e = threadIdx.x; e < region; e += blockDim.x) {
    R re = acc[2 * e], im = acc[2 * e + 1];
    if constexpr (COMP) {
      re += comp[2 * e];
      im += comp[2 * e + 1];
    }
    if (re != R(0) || im != R(0)) grid_add(grid + region_to_grid<D>(g, start, e), re, im);
  }
}

template <int D, int K, typename R, bool COMP>
__global__ void __launch_bounds__(kResampleThreads)
    scatter_kernel(Geometry g, typename CplxT<R>::type* __restrict__ grid, NodeArrays na,
                   const typename CplxT<R>::type* __restrict__ fhat) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* acc = reinterpret_cast<R*>(smem_raw);  // interleaved re, im
  const int nitems = *na.n_items;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x)
    scatter_item<D, K, R, COMP>(g, grid, na, na.items[it], fhat, acc);
}

template <int D, int K, typename R>
__global__ void __launch_bounds__(kResampleThreads)
    scatter_batch_kernel(const BatchProblem* __restrict__ probs, typename CplxT<R>::type* __restrict__ grid,
                         BatchNodes nb, const typename CplxT<R>::type* __restrict__ fhat) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* acc = reinterpret_cast<R*>(smem_raw);
  const int nitems = *nb.n_items;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int4 item = nb.items[it];
    const BatchProblem& P = probs[item.w];
    const Geometry g = P.g;
    NodeArrays na;
    na.cell = nb.cell + D * P.node_off;
    na.frac = reinterpret_cast<const R*>(nb.frac) + D * P.node_off;
    na.perm = nb.perm + P.node_off;
    scatter_item<D, K, R, false>(g, grid + P.grid_off, na, item, fhat + P.out_off, acc);
  }
}

// ---------------------------------------------------------------------------
// Node-gradient gather: d fhat_j / d k_{j,d}, contracted with conj(cot_j)
// ---------------------------------------------------------------------------
template <int D, int K, typename R>
__global__ void __launch_bounds__(kResampleThreads)
    grad_kernel(Geometry g, const typename CplxT<R>::type* __restrict__ grid, NodeArrays na,
                const typename CplxT<R>::type* __restrict__ cot, R* __restrict__ gk) {
  using C = typename CplxT<R>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tile = reinterpret_cast<C*>(smem_raw);
  const R* __restrict__ frac = reinterpret_cast<const R*>(na.frac);
  const int nitems = *na.n_items;
  const int region = region_size<D>(g);
  const int mi = (int)g.m;
  const int64_t M = g.M;

  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int4 item = na.items[it];
    int tc[kMaxD], start[kMaxD];
    tile_coords<D>(g, item.x, tc);
#pragma unroll
    for (int d = 0; d < D; ++d) start[d] = tc[d] * g.T[d] + g.off;
    __syncthreads();
    for (int e = threadIdx.x; e < region; e += blockDim.x)
      tile[e] = grid[region_to_grid<D>(g, start, e)];
    __syncthreads();

    for (int q = item.y + threadIdx.x; q < item.y + item.z; q += blockDim.x) {
      R w[D][K], dw[D][K];
      int a[D];
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const R t = frac[d * M + q];
        a[d] = na.cell[d * M + q] - tc[d] * g.T[d];
        node_weights<K, R>(g, d, mi, t, w[d]);
        node_weight_derivs<K, R>(g, d, mi, t, dw[d]);
      }
      R dr[D], di[D];
#pragma unroll
      for (int d = 0; d < D; ++d) dr[d] = di[d] = R(0);
      if constexpr (D == 1) {
#pragma unroll
        for (int i = 0; i < K; ++i) {
          C v = tile[a[0] + i];
          dr[0] += dw[0][i] * v.x;
          di[0] += dw[0][i] * v.y;
        }
      } else if constexpr (D == 2) {
#pragma unroll
        for (int i0 = 0; i0 < K; ++i0) {
          const C* row = tile + (a[0] + i0) * g.L[1] + a[1];
          R sr = 0, si = 0, sdr = 0, sdi = 0;
#pragma unroll
          for (int i1 = 0; i1 < K; ++i1) {
            C v = row[i1];
            sr += w[1][i1] * v.x;
            si += w[1][i1] * v.y;
            sdr += dw[1][i1] * v.x;
            sdi += dw[1][i1] * v.y;
          }
          dr[0] += dw[0][i0] * sr;
          di[0] += dw[0][i0] * si;
          dr[1] += w[0][i0] * sdr;
          di[1] += w[0][i0] * sdi;
        }
      } else {
#pragma unroll 1
        for (int i0 = 0; i0 < K; ++i0) {
          const C* plane = tile + ((a[0] + i0) * g.L[1] + a[1]) * g.L[2] + a[2];
          R s1r = 0, s1i = 0, s1dr = 0, s1di = 0, s2dr = 0, s2di = 0;
#pragma unroll
          for (int i1 = 0; i1 < K; ++i1) {
            const C* row = plane + i1 * g.L[2];
            R sr = 0, si = 0, sdr = 0, sdi = 0;
#pragma unroll
            for (int i2 = 0; i2 < K; ++i2) {
              C v = row[i2];
              sr += w[2][i2] * v.x;
              si += w[2][i2] * v.y;
              sdr += dw[2][i2] * v.x;
              sdi += dw[2][i2] * v.y;
            }
            s1r += w[1][i1] * sr;
            s1i += w[1][i1] * si;
            s1dr += dw[1][i1] * sr;
            s1di += dw[1][i1] * si;
            s2dr += w[1][i1] * sdr;
            s2di += w[1][i1] * sdi;
          }
          R w0 = 0, dw0 = 0;
#pragma unroll
          for (int i = 0; i < K; ++i) {
            w0 = (i == i0) ? w[0][i] : w0;
            dw0 = (i == i0) ? dw[0][i] : dw0;
          }
          dr[0] += dw0 * s1r;
          di[0] += dw0 * s1i;
          dr[1] += w0 * s1dr;
          di[1] += w0 * s1di;
          dr[2] += w0 * s2dr;
          di[2] += w0 * s2di;
        }
      }
      const int j = na.perm[q];
      const C c = cot[j];
#pragma unroll
      for (int d = 0; d < D; ++d) gk[(int64_t)j * D + d] = c.x * dr[d] + c.y * di[d];
    }
  }
}

// ---------------------------------------------------------------------------
// Kernel selection on (D, K); K = taps per dimension (2m, or 2m+2 closed).
// Each kind is instantiated in its own translation unit.
// ---------------------------------------------------------------------------
#define NFFTGB_FOR_EACH_DK(X) \
  X(1, 2) X(1, 4) X(1, 6) X(1, 8) X(1, 10) X(1, 12) X(1, 14) X(1, 16) X(1, 18) \
  X(2, 2) X(2, 4) X(2, 6) X(2, 8) X(2, 10) X(2, 12) X(2, 14) X(2, 16) X(2, 18) \
  X(3, 2) X(3, 4) X(3, 6) X(3, 8) X(3, 10) X(3, 12) X(3, 14) X(3, 16) X(3, 18)
// m = 9, 10 (K = 20, 22) for the plain gather and scatter in 1D and 2D only,
// where the paper's accuracy study runs: instantiating every kind and 3D as
// well would triple the build time.
#define NFFTGB_FOR_EACH_DK_HIGH_M(X) X(1, 20) X(1, 22) X(2, 20) X(2, 22)

template <typename R>
void* pick_gather(int D, int K) {
#define NFFTGB_PICK(DD, KK) \
  if (D == DD && K == KK) return (void*)gather_kernel<DD, KK, R>;
  NFFTGB_FOR_EACH_DK(NFFTGB_PICK)
  NFFTGB_FOR_EACH_DK_HIGH_M(NFFTGB_PICK)
#undef NFFTGB_PICK
  return nullptr;
}

template <typename R>
void* pick_scatter(int D, int K, int compensated) {
#define NFFTGB_PICK(DD, KK)                                                  \
  if (D == DD && K == KK) {                                                  \
    if constexpr (sizeof(R) == 4) {                                          \
      if (compensated) return (void*)scatter_kernel<DD, KK, R, true>;        \
    }                                                                        \
    return compensated ? nullptr : (void*)scatter_kernel<DD, KK, R, false>;  \
  }
  NFFTGB_FOR_EACH_DK(NFFTGB_PICK)
#undef NFFTGB_PICK
#define NFFTGB_PICK(DD, KK) \
  if (D == DD && K == KK && !compensated) return (void*)scatter_kernel<DD, KK, R, false>;
  NFFTGB_FOR_EACH_DK_HIGH_M(NFFTGB_PICK)
#undef NFFTGB_PICK
  return nullptr;
}

template <typename R>
void* pick_gather_batch(int D, int K) {
#define NFFTGB_PICK(DD, KK) \
  if (D == DD && K == KK) return (void*)gather_batch_kernel<DD, KK, R>;
  NFFTGB_FOR_EACH_DK(NFFTGB_PICK)
#undef NFFTGB_PICK
  return nullptr;
}

template <typename R>
void* pick_scatter_batch(int D, int K) {
#define NFFTGB_PICK(DD, KK) \
  if (D == DD && K == KK) return (void*)scatter_batch_kernel<DD, KK, R>;
  NFFTGB_FOR_EACH_DK(NFFTGB_PICK)
#undef NFFTGB_PICK
  return nullptr;
}

template <typename R>
void* pick_grad(int D, int K) {
#define NFFTGB_PICK(DD, KK) \
  if (D == DD && K == KK) return (void*)grad_kernel<DD, KK, R>;
  NFFTGB_FOR_EACH_DK(NFFTGB_PICK)
#undef NFFTGB_PICK
  return nullptr;
}

}  // namespace nfftgb
