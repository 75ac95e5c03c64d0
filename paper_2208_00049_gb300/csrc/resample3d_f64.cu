// 3D complex128 scatter (Eq. SumOverNodeAdjoint, Algorithm 4) for K = 2m <= 8
// taps per dimension, without shared-memory atomics: the residue-class
// ownership of the 2D complex128 scatter (resample2d_f64.cu) in three
// dimensions.
//
//  * one CTA of 128 threads per work item, the region (tile + halo,
//    L0 x L1 x L2 complex) in shared memory; nodes staged 16 at a time;
//  * window values: each of a node's 3K taps is evaluated once (the
//    POLYNOMIAL coefficients staged in shared memory, or the LINEAR / direct
//    forms); then per node the K x K table w0[i0] w1[i1] and v w2 per column
//    residue mod 8, so that each term costs one complex-by-real FMA;
//  * accumulation with exclusive ownership: thread (r0, r1, c) =
//    (tid >> 5, (tid >> 3) & 3, tid & 7) owns the region points whose
//    coordinates are congruent to (r0, r1, c) mod (4, 4, 8).  A node's K <= 8
//    consecutive points per dimension hold each residue mod 8 at most once
//    and each residue mod 4 at most twice, so a thread adds at most 4 terms
//    per node (exactly 4 at m = 4) to points no other thread touches: plain
//    read-modify-writes in program order per thread, whatever the nodes;
//  * the region is added to the grid with FP64 global reductions (performed
//    in L2), wrapped per dimension.
//
// FP64 work per node at m = 4: 24 Horner chains (of 16 steps in the complex128
// POLYNOMIAL table, degree 16 at m <= 8; or the direct form), 64 + 16 table
// products and 1024 multiply-adds for the 512 complex terms, about 1500
// operations, where the generic kernel adds each of the 1024 real terms
// with a shared-memory FP64 atomic.
#include <stdlib.h>
#include <string.h>

#include "resample.cuh"

namespace nfftgb {
namespace {

constexpr int kS3Threads = 128;
constexpr int kS3Batch = 16;  // nodes staged per batch
constexpr int kS3MaxK = 8;
constexpr int kS3Z = 17;      // POLYNOMIAL coefficients per tap held (zero above the table's)

template <int K>
struct S3Stage {
  double coef[3][K][kS3Z];         // POLYNOMIAL coefficients of every tap, zero above the table's
  double t[kS3Batch][3];           // fractional positions
  double2 v[kS3Batch];             // input values
  int a[kS3Batch][4];              // cell offsets in the tile
  double w[kS3Batch][3][K];        // window values per dimension and tap
  double w01[kS3Batch][K][K];      // w0[i0] w1[i1]
  double2 vw2[kS3Batch][8];        // v w2 at the column congruent to c mod 8 (zero off the footprint)
};

template <int K>
size_t s3_bytes(const Geometry& g) {
  return sizeof(S3Stage<K>) + (size_t)g.L[0] * g.L[1] * g.L[2] * sizeof(double2);
}

// Window value of tap i of dimension d (u = t - off - i), in the plan's
// window form; pc: the tap's kS3Z POLYNOMIAL coefficients (kWinPoly only).
__device__ __forceinline__ double tap_value3(const Geometry& g, int d, int mi, double t, int i, const double* pc) {
  if (g.wmode == kWinPoly) {
    const double zeta = t - 0.5;
    double v = pc[kS3Z - 1];
#pragma unroll
    for (int z = kS3Z - 2; z >= 0; --z) v = v * zeta + pc[z];
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
__global__ void __launch_bounds__(kS3Threads)
    scatter3d_f64_kernel(Geometry g, double2* __restrict__ grid, NodeArrays na, const double2* __restrict__ fhat) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  S3Stage<K>& st = *reinterpret_cast<S3Stage<K>*>(smem_raw);
  double2* acc = reinterpret_cast<double2*>(smem_raw + sizeof(S3Stage<K>));
  const int tid = threadIdx.x;
  const int r0 = tid >> 5, r1 = (tid >> 3) & 3, c2 = tid & 7;
  const int L0 = g.L[0], L1 = g.L[1], L2 = g.L[2], region = L0 * L1 * L2;
  const int mi = (int)g.m;
  const int64_t M = g.M;
  const double* frac = reinterpret_cast<const double*>(na.frac);
  if (g.wmode == kWinPoly)
    for (int e = tid; e < 3 * K * kS3Z; e += kS3Threads) {
      const int tap = e / kS3Z, z = e - tap * kS3Z;  // tap = d K + i
      (&st.coef[0][0][0])[e] = z < g.wZ ? ((const double*)g.wtab)[(int64_t)tap * g.wZ + z] : 0.0;
    }
  const int nitems = *na.n_items;

  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int4 item = na.items[it];
    int tc[3], start[3];
    tile_coords<3>(g, item.x, tc);
#pragma unroll
    for (int d = 0; d < 3; ++d) start[d] = tc[d] * g.T[d] + g.off;
    for (int e = tid; e < region; e += kS3Threads) acc[e] = make_double2(0.0, 0.0);

    for (int b = 0; b < item.z; b += kS3Batch) {
      const int nb = min(kS3Batch, item.z - b);
      __syncthreads();  // the previous batch is done with the stage; the region is cleared
      if (tid < nb) {
        const int q = item.y + b + tid;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          st.a[tid][d] = na.cell[d * M + q] - tc[d] * g.T[d];
          st.t[tid][d] = frac[d * M + q];
        }
        st.v[tid] = fhat[na.perm[q]];
      }
      __syncthreads();
      for (int e = tid; e < nb * 3 * K; e += kS3Threads) {
        const int n = e / (3 * K), j = e - n * 3 * K, d = j / K, i = j - d * K;
        st.w[n][d][i] = tap_value3(g, d, mi, st.t[n][d], i, &st.coef[d][i][0]);
      }
      __syncthreads();
      for (int e = tid; e < nb * K * K; e += kS3Threads) {
        const int n = e / (K * K), j = e - n * K * K, i0 = j / K, i1 = j - i0 * K;
        st.w01[n][i0][i1] = st.w[n][0][i0] * st.w[n][1][i1];
      }
      for (int e = tid; e < nb * 8; e += kS3Threads) {
        const int n = e >> 3, c = e & 7;
        const int j2 = (c - st.a[n][2]) & 7;
        const double w2 = j2 < K ? st.w[n][2][j2] : 0.0;
        const double2 v = st.v[n];
        st.vw2[n][c] = make_double2(v.x * w2, v.y * w2);
      }
      __syncthreads();
      for (int n = 0; n < nb; ++n) {
        const int a0 = st.a[n][0], a1 = st.a[n][1], a2 = st.a[n][2];
        const int j2 = (c2 - a2) & 7;  // tap of dimension 2 at this thread's column
        if (j2 < K) {
          const double2 vw = st.vw2[n][c2];
          const int i0s = (r0 - a0) & 3, i1s = (r1 - a1) & 3;  // first taps with this thread's residues
          double2* p = acc + ((a0 + i0s) * L1 + a1 + i1s) * L2 + a2 + j2;
#pragma unroll
          for (int k0 = 0; k0 < (K + 3) / 4; ++k0) {
#pragma unroll
            for (int k1 = 0; k1 < (K + 3) / 4; ++k1) {
              const int i0 = i0s + 4 * k0, i1 = i1s + 4 * k1;
              if (i0 < K && i1 < K) {
                const double w = st.w01[n][i0][i1];
                double2* q = p + (4 * k0 * L1 + 4 * k1) * L2;
                double2 x = *q;
                x.x = fma(vw.x, w, x.x);
                x.y = fma(vw.y, w, x.y);
                *q = x;
              }
            }
          }
        }
      }
    }
    __syncthreads();
    // add the region to the grid (wrap applied here only); the next item
    // clears the elements each thread has just read
    for (int e = tid; e < region; e += kS3Threads) {
      const double2 x = acc[e];
      if (x.x != 0.0 || x.y != 0.0) {
        double2* dst = grid + region_to_grid<3>(g, start, e);
        atomicAdd(&dst->x, x.x);
        atomicAdd(&dst->y, x.y);
      }
    }
  }
}

void* s3_kernel(int K) {
  switch (K) {
    case 2: return (void*)scatter3d_f64_kernel<2>;
    case 4: return (void*)scatter3d_f64_kernel<4>;
    case 6: return (void*)scatter3d_f64_kernel<6>;
    case 8: return (void*)scatter3d_f64_kernel<8>;
  }
  return nullptr;
}

size_t s3_smem(const Geometry& g) {
  switch (g.K) {
    case 2: return s3_bytes<2>(g);
    case 4: return s3_bytes<4>(g);
    case 6: return s3_bytes<6>(g);
    case 8: return s3_bytes<8>(g);
  }
  return 0;
}

cudaError_t s3_prepare(void* k, size_t smem) {
  if (smem > 48 * 1024) return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaSuccess;
}

}  // namespace

// NFFT_GB300_F64_SCATTER=generic keeps complex128 3D plans on the generic
// shared-atomic scatter as well (read at each call).
bool scatter3d_f64_supported(const Geometry& g) {
  const char* e = getenv("NFFT_GB300_F64_SCATTER");
  if (e && strcmp(e, "generic") == 0) return false;
  if (g.D != 3 || g.closed || g.K % 2 != 0 || g.K > kS3MaxK || g.K != 2 * (int)g.m || g.off != 1 - g.K / 2)
    return false;
  if (g.wmode == kWinPoly && g.wZ > kS3Z) return false;
  return s3_smem(g) <= 200 * 1024;
}

int scatter3d_f64_ctas_per_sm(const Geometry& g) {
  void* k = s3_kernel(g.K);
  if (!k) return 0;
  const size_t smem = s3_smem(g);
  if (s3_prepare(k, smem) != cudaSuccess) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kS3Threads, smem) != cudaSuccess) return 0;
  return n;
}

cudaError_t launch_scatter3d_f64(const Geometry& g, void* grid, const NodeArrays& na, const void* fhat, int ctas,
                                 cudaStream_t s) {
  void* k = s3_kernel(g.K);
  if (!k) return cudaErrorInvalidValue;
  const size_t smem = s3_smem(g);
  cudaError_t e = s3_prepare(k, smem);
  if (e != cudaSuccess) return e;
  auto kern = reinterpret_cast<void (*)(Geometry, double2*, NodeArrays, const double2*)>(k);
  kern<<<ctas, kS3Threads, smem, s>>>(g, (double2*)grid, na, (const double2*)fhat);
  return cudaGetLastError();
}

}  // namespace nfftgb
