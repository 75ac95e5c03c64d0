// 2D complex128 scatter (Eq. SumOverNodeAdjoint, Algorithm 4) for K = 2m <= 16
// taps per dimension, without shared-memory atomics.
//
// GB300 issues FP64 arithmetic at about 1/64 of its FP32 rate (1.25 against
// 80 TFLOP/s nominal), so FP64 operations are the scarce resource.  The
// generic scatter adds each of a node's 2 K^2 real terms to shared memory
// with an FP64 atomic from the node's thread; here the accumulation needs no
// atomics and the FP64 pipe does little beyond the method's arithmetic:
//
//  * one CTA of 4 warps per work item, the region (tile + halo, L0 x L1
//    complex) in shared memory; nodes staged 32 at a time;
//  * window values: each of the 32 taps of a node (16 per dimension) is
//    evaluated once, thread t always taking tap t & 31 (the POLYNOMIAL form
//    from coefficients held in registers, or the LINEAR / direct forms), then
//    v w1 once per node and column residue mod 16;
//  * accumulation with exclusive ownership: lane (c, h) = (l & 15, l >> 4) of
//    warp w owns the region columns congruent to c mod 16 in the rows
//    congruent to 2w + h mod 8.  A node's K <= 16 consecutive columns hold
//    each residue mod 16 at most once and its K consecutive rows K/8 rows of
//    each residue mod 8, so a thread adds K/8 terms (v w1) w0 per node (two
//    at m = 8), and no two threads ever touch the same element: plain
//    read-modify-writes in program order per thread, whatever the nodes;
//  * the region is added to the grid with FP64 global reductions (performed
//    in L2), wrapped per dimension.
#include <stdlib.h>
#include <string.h>

#include "resample.cuh"

namespace nfftgb {
namespace {

constexpr int kF64Warps = 4;                 // warps per CTA, one work item per CTA
constexpr int kF64Threads = 32 * kF64Warps;
constexpr int kF64Rows = 2 * kF64Warps;      // row residues: (warp, lane >> 4)
constexpr int kF64Batch = 32;                // nodes staged per batch
constexpr int kF64Z = 17;                    // POLYNOMIAL coefficients per tap held (zero above the table's)

struct F64Stage {
  double t[kF64Batch][2];      // fractional positions
  double2 v[kF64Batch];        // input values
  int a[kF64Batch][2];         // cell offsets in the tile
  double w[kF64Batch][32];     // window values: [i] tap i of dimension 0, [16 + i] of dimension 1
  double2 vw[kF64Batch][16];   // v w1 at the column congruent to c mod 16 (zero off the footprint)
};

size_t f64_cta_bytes(const Geometry& g) {
  return sizeof(F64Stage) + (size_t)g.L[0] * g.L[1] * sizeof(double2);
}

// Window value of tap i of dimension d (u = t - off - i), in the plan's
// window form; coef: the tap's POLYNOMIAL coefficients, zero above the
// table's degree (kWinPoly only).
__device__ __forceinline__ double tap_value(const Geometry& g, int d, int mi, double t, int i,
                                            const double (&coef)[kF64Z]) {
  if (g.wmode == kWinPoly) {
    const double zeta = t - 0.5;
    double v = coef[kF64Z - 1];
#pragma unroll
    for (int z = kF64Z - 2; z >= 0; --z) v = v * zeta + coef[z];
    return v;
  }
  const double u = double(-g.off - i) + t;
  if (g.wmode == kWinLinear) {
    const double* tab = (const double*)g.wtab + (int64_t)d * g.wS;
    double slope;
    return lut_window<double>(tab, g.wS, double(g.wS - 2) / double(mi), u, &slope);
  }
  const double mm_u = double(mi + g.off + i) - t;  // m - u
  const double mp_u = double(mi - g.off - i) + t;  // m + u
  return kb_window<double>(u, mm_u, mp_u, g.b[d], g.norm[d], double(mi), 0.0);
}

template <int K>
__global__ void __launch_bounds__(kF64Threads)
    scatter2d_f64_kernel(Geometry g, double2* __restrict__ grid, NodeArrays na, const double2* __restrict__ fhat) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  F64Stage& st = *reinterpret_cast<F64Stage*>(smem_raw);
  double2* acc = reinterpret_cast<double2*>(smem_raw + sizeof(F64Stage));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int L0 = g.L[0], L1 = g.L[1], region = L0 * L1;
  const int c16 = lane & 15, h = lane >> 4;
  const int rres = 2 * warp + h;  // this thread's row residue mod kF64Rows
  const int mi = (int)g.m;
  const int64_t M = g.M;
  const double* frac = reinterpret_cast<const double*>(na.frac);
  // this thread's window tap: tap c16 of dimension h; coefficients in registers
  double coef[kF64Z];
#pragma unroll
  for (int z = 0; z < kF64Z; ++z)
    coef[z] = (g.wmode == kWinPoly && c16 < K && z < g.wZ) ? ((const double*)g.wtab)[((int64_t)h * K + c16) * g.wZ + z]
                                                           : 0.0;
  const int nitems = *na.n_items;

  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int4 item = na.items[it];
    int tc[2], start[2];
    tile_coords<2>(g, item.x, tc);
#pragma unroll
    for (int d = 0; d < 2; ++d) start[d] = tc[d] * g.T[d] + g.off;
    for (int e = tid; e < region; e += kF64Threads) acc[e] = make_double2(0.0, 0.0);

    for (int b = 0; b < item.z; b += kF64Batch) {
      const int nb = min(kF64Batch, item.z - b);
      __syncthreads();  // the previous batch is done with the stage; the region is cleared
      if (tid < nb) {
        const int q = item.y + b + tid;
        st.a[tid][0] = na.cell[q] - tc[0] * g.T[0];
        st.a[tid][1] = na.cell[M + q] - tc[1] * g.T[1];
        st.t[tid][0] = frac[q];
        st.t[tid][1] = frac[M + q];
        st.v[tid] = fhat[na.perm[q]];
      }
      __syncthreads();
      // tap (h, c16) of nodes warp, warp + 4, ...
#pragma unroll 2
      for (int n = warp; n < nb; n += kF64Warps)
        st.w[n][lane] = c16 < K ? tap_value(g, h, mi, st.t[n][h], c16, coef) : 0.0;
      __syncthreads();
      // v w1 per node and column residue
      for (int e = tid; e < nb * 16; e += kF64Threads) {
        const int n = e >> 4, c = e & 15;
        const int j1 = (c - st.a[n][1]) & 15;
        const double w1 = j1 < K ? st.w[n][16 + j1] : 0.0;
        const double2 v = st.v[n];
        st.vw[n][c] = make_double2(v.x * w1, v.y * w1);
      }
      __syncthreads();
      for (int n = 0; n < nb; ++n) {
        const int a0 = st.a[n][0], a1 = st.a[n][1];
        const int j1 = (c16 - a1) & 15;  // tap of dimension 1 at this thread's column
        if (j1 < K) {
          const double2 vw = st.vw[n][c16];
          const int i0s = (rres - a0) & (kF64Rows - 1);  // first tap whose row has this residue
          double2* p = acc + a1 + j1;
#pragma unroll
          for (int k = 0; k < (K + kF64Rows - 1) / kF64Rows; ++k) {
            const int i0 = i0s + kF64Rows * k;
            if (i0 < K) {
              const double w0 = st.w[n][i0];
              double2* q = p + (a0 + i0) * L1;
              double2 x = *q;
              x.x = fma(vw.x, w0, x.x);
              x.y = fma(vw.y, w0, x.y);
              *q = x;
            }
          }
        }
      }
    }
    __syncthreads();
    // add the region to the grid (wrap applied here only); the next item
    // clears the elements each thread has just read
    for (int e = tid; e < region; e += kF64Threads) {
      const double2 x = acc[e];
      if (x.x != 0.0 || x.y != 0.0) {
        double2* dst = grid + region_to_grid<2>(g, start, e);
        atomicAdd(&dst->x, x.x);
        atomicAdd(&dst->y, x.y);
      }
    }
  }
}

void* f64_kernel(int K) {
  switch (K) {
    case 2: return (void*)scatter2d_f64_kernel<2>;
    case 4: return (void*)scatter2d_f64_kernel<4>;
    case 6: return (void*)scatter2d_f64_kernel<6>;
    case 8: return (void*)scatter2d_f64_kernel<8>;
    case 10: return (void*)scatter2d_f64_kernel<10>;
    case 12: return (void*)scatter2d_f64_kernel<12>;
    case 14: return (void*)scatter2d_f64_kernel<14>;
    case 16: return (void*)scatter2d_f64_kernel<16>;
  }
  return nullptr;
}

cudaError_t f64_prepare(void* k, size_t smem) {
  if (smem > 48 * 1024) return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaSuccess;
}

}  // namespace

// NFFT_GB300_F64_SCATTER=generic keeps complex128 2D plans on the generic
// shared-atomic scatter (read at each call, so that the two forms can be
// compared in one process).
bool scatter2d_f64_supported(const Geometry& g) {
  const char* e = getenv("NFFT_GB300_F64_SCATTER");
  if (e && strcmp(e, "generic") == 0) return false;
  if (g.D != 2 || g.closed || g.K % 2 != 0 || g.K > 16 || g.K != 2 * (int)g.m || g.off != 1 - g.K / 2) return false;
  if (g.wmode == kWinPoly && g.wZ > kF64Z) return false;
  return f64_cta_bytes(g) <= 200 * 1024;
}

int scatter2d_f64_ctas_per_sm(const Geometry& g) {
  void* k = f64_kernel(g.K);
  if (!k) return 0;
  const size_t smem = f64_cta_bytes(g);
  if (f64_prepare(k, smem) != cudaSuccess) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kF64Threads, smem) != cudaSuccess) return 0;
  return n;
}

int scatter2d_f64_items_per_cta() { return 1; }

cudaError_t launch_scatter2d_f64(const Geometry& g, void* grid, const NodeArrays& na, const void* fhat, int ctas,
                                 cudaStream_t s) {
  void* k = f64_kernel(g.K);
  if (!k) return cudaErrorInvalidValue;
  const size_t smem = f64_cta_bytes(g);
  cudaError_t e = f64_prepare(k, smem);
  if (e != cudaSuccess) return e;
  auto kern = reinterpret_cast<void (*)(Geometry, double2*, NodeArrays, const double2*)>(k);
  kern<<<ctas, kF64Threads, smem, s>>>(g, (double2*)grid, na, (const double2*)fhat);
  return cudaGetLastError();
}

}  // namespace nfftgb
