// Deconvolution (resampling correction), plan-time tables and node bin-sort.
//
// arXiv 2208.00049:
//  * Algorithm 1 (correction and zero-pad step) and Algorithm 2 (crop and
//    correction step): the resampling correction 1/(|I_N~| phi(n)) with zero
//    pad (direct) or crop (adjoint);
//    Sec. 3.5 folds the fftshift into the index map and factorises the
//    correction into per-dimension vectors beta_d (O(sum N_d) memory).
//  * Sec. 3.7.3: nodes are grouped by the grid block they fall in (the sets
//    Gamma_p); here by a device counting sort over tiles, with tiles holding
//    more than `cmax` nodes split into several work items (fixed number of
//    points per block, Sec. 3.7.2).
#include "nfft_internal.cuh"

namespace nfftgb {

template <typename R>
struct Cplx;
template <>
struct Cplx<float> {
  using type = float2;
};
template <>
struct Cplx<double> {
  using type = double2;
};

static int launch_blocks(int64_t work, int threads) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t want = (work + threads - 1) / threads;
  int64_t cap = (int64_t)sms * 16;
  if (want > cap) want = cap;
  if (want < 1) want = 1;
  return (int)want;
}

// ---------------------------------------------------------------------------
// beta_d(n_d) = W_d(0) / I0(m sqrt(b_d^2 - (2 pi n_d / N~_d)^2)), n_d in I_{N_d},
// in FP64 on the device.  W_d(0) = sinh(b_d m)/(pi m) is the peak of the
// window, which the resampling kernels divide out of their weights; the
// product over d of these factors is 1/(|I_N~| phi(n)) times that peak.
// ---------------------------------------------------------------------------
struct BetaArgs {
  int D;
  int N[kMaxD];
  int Nt[kMaxD];
  int offset[kMaxD];
  double b[kMaxD];
  int m;
};

__global__ void build_beta_kernel(BetaArgs a, double* beta64, float* beta32) {
  int total = a.offset[a.D - 1] + a.N[a.D - 1];
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    int d = 0;
    while (d + 1 < a.D && idx >= a.offset[d + 1]) ++d;
    int i = idx - a.offset[d];
    double n = (double)(i - a.N[d] / 2);
    double w = 2.0 * M_PI * n / (double)a.Nt[d];
    double bb = a.b[d];
    double arg = (double)a.m * sqrt(bb * bb - w * w);
    double peak = sinh(bb * (double)a.m) / (M_PI * (double)a.m);
    double v = peak / cyl_bessel_i0(arg);
    beta64[idx] = v;
    beta32[idx] = (float)v;
  }
}

cudaError_t launch_build_beta(int D, const int* N, const int* Nt, int m, const double* b,
                              double* beta64, float* beta32, cudaStream_t s) {
  BetaArgs a{};
  a.D = D;
  a.m = m;
  int off = 0;
  for (int d = 0; d < D; ++d) {
    a.N[d] = N[d];
    a.Nt[d] = Nt[d];
    a.b[d] = b[d];
    a.offset[d] = off;
    off += N[d];
  }
  build_beta_kernel<<<launch_blocks(off, 256), 256, 0, s>>>(a, beta64, beta32);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// POLYNOMIAL window precomputation (Sec. 3.7.4, item 5): the window is split
// into the K unit intervals of its taps; on each, with zeta = t - 1/2 in
// [-1/2, 1/2] (t the node's fraction), the tap value is a polynomial of degree
// `deg` in zeta.  Coefficients: interpolation at the deg + 1 Chebyshev points
// of [-1/2, 1/2] (instead of the paper's least squares on 2(deg + 1)
// equispaced samples), solved in FP64 by Gaussian elimination with partial
// pivoting, one thread per (dimension, tap).  Stored as FP32 in
// coef[(d * K + i) * (deg + 1) + z], for the scaled window w(u)/w(0).
// ---------------------------------------------------------------------------
constexpr int kMaxPolyCoef = 2 * kMaxM + 1;

__global__ void build_poly_kernel(PolyArgs a, float* coef, double* coef64) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= a.D * a.K) return;
  const int d = idx / a.K, i = idx % a.K;
  const int Z = a.deg + 1;
  double V[kMaxPolyCoef][kMaxPolyCoef + 1];
  const double center = 0.5 - (double)a.off - (double)i;  // u = zeta + center
  const double m = (double)a.m, b = a.b[d];
  const double norm = m / sinh(b * m);
  for (int j = 0; j < Z; ++j) {
    const double zeta = 0.5 * cos(M_PI * (j + 0.5) / Z);
    const double u = center + zeta;
    const double s2 = (m - u) * (m + u);
    const double s = sqrt(s2 > 0.0 ? s2 : -s2);
    const double val = (s == 0.0) ? b * norm : (s2 > 0.0 ? sinh(b * s) : sin(b * s)) / s * norm;
    double p = 1.0;
    for (int z = 0; z < Z; ++z) {
      V[j][z] = p;
      p *= zeta;
    }
    V[j][Z] = val;
  }
  for (int col = 0; col < Z; ++col) {
    int piv = col;
    for (int r = col + 1; r < Z; ++r)
      if (fabs(V[r][col]) > fabs(V[piv][col])) piv = r;
    if (piv != col)
      for (int c = col; c <= Z; ++c) {
        double tmp = V[col][c];
        V[col][c] = V[piv][c];
        V[piv][c] = tmp;
      }
    for (int r = col + 1; r < Z; ++r) {
      const double f = V[r][col] / V[col][col];
      for (int c = col; c <= Z; ++c) V[r][c] -= f * V[col][c];
    }
  }
  for (int r = Z - 1; r >= 0; --r) {
    double acc = V[r][Z];
    for (int c = r + 1; c < Z; ++c) acc -= V[r][c] * V[c][Z];
    V[r][Z] = acc / V[r][r];
  }
  for (int z = 0; z < Z; ++z) {
    if (coef) coef[(d * a.K + i) * Z + z] = (float)V[z][Z];
    if (coef64) coef64[(d * a.K + i) * Z + z] = V[z][Z];
  }
}

cudaError_t launch_build_poly(const PolyArgs& a, float* coef, cudaStream_t s, double* coef64) {
  if (a.deg + 1 > kMaxPolyCoef) return cudaErrorInvalidValue;
  build_poly_kernel<<<1, 64, 0, s>>>(a, coef, coef64);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// LINEAR window tables (Sec. 3.7.4): psi_s = psi_Base(s / (S - 2)), i.e. the
// window (scaled to 1 at u = 0) at u = m s / (S - 2) in grid units, on the
// closed support [-m, m] (entry S - 2 is the edge value read by the tap at
// u = -m) and 0 beyond it (entry S - 1), S = m 2^{c_min(m, 8)} + 2 with NFFT3's
// exponents C = (3, 7, 9, 14, 17, 20, 23, 24).  FP64 arithmetic.
// ---------------------------------------------------------------------------
int64_t lut_table_size(int m) {
  static const int C[8] = {3, 7, 9, 14, 17, 20, 23, 24};
  if (m < 1) return 0;
  return (int64_t)m * ((int64_t)1 << C[(m < 8 ? m : 8) - 1]) + 2;
}

struct LutArgs {
  int D;
  int m;
  int64_t S;
  double b[kMaxD];
};

__global__ void build_lut_kernel(LutArgs a, float* lut32, double* lut64) {
  const int64_t n = (int64_t)a.D * a.S;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int d = (int)(e / a.S);
    const int64_t sidx = e - (int64_t)d * a.S;
    const double m = (double)a.m, b = a.b[d];
    double v = 0.0;
    if (sidx <= a.S - 2) {
      const double u = m * (double)sidx / (double)(a.S - 2);
      const double s2 = (m - u) * (m + u);
      const double sq = sqrt(s2 > 0.0 ? s2 : 0.0);
      const double z = b * sq;
      v = (z < 1e-4 ? b * (1.0 + z * z / 6.0) : sinh(z) / sq) * (m / sinh(b * m));
    }
    if (lut32) lut32[e] = (float)v;
    if (lut64) lut64[e] = v;
  }
}

cudaError_t launch_build_lut(int D, int m, const double* b, int64_t S, float* lut32, double* lut64, cudaStream_t s) {
  LutArgs a{};
  a.D = D;
  a.m = m;
  a.S = S;
  for (int d = 0; d < D; ++d) a.b[d] = b[d];
  build_lut_kernel<<<launch_blocks((int64_t)D * S, 256), 256, 0, s>>>(a, lut32, lut64);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Algorithm 1, correction and zero-pad step: g[p] = f_n * prod_d beta_d(n_d)
// where the grid position p_d = n_d mod N~_d, zero at every other position.  One thread
// writes two adjacent grid points (16 B for complex64) of the last dimension.
// ---------------------------------------------------------------------------
template <int D, typename R>
__device__ __forceinline__ void deconv_pad_body(const DeconvArgs& a, const typename Cplx<R>::type* __restrict__ f,
                                                typename Cplx<R>::type* __restrict__ grid, int64_t first,
                                                int64_t stride) {
  using C = typename Cplx<R>::type;
  const R* __restrict__ beta0 = (const R*)a.beta[0];
  const R* __restrict__ beta1 = (const R*)a.beta[D > 1 ? 1 : 0];
  const R* __restrict__ beta2 = (const R*)a.beta[D > 2 ? 2 : 0];
  const int last = D - 1;
  const int half_last = a.Nt[last] / 2;  // pairs per row
  int64_t rows = 1;
  for (int d = 0; d < last; ++d) rows *= a.Nt[d];
  const int64_t total = rows * half_last;
  for (int64_t t = first; t < total; t += stride) {
    const int pair = (int)(t % half_last);
    int64_t row = t / half_last;
    // index into f of the outer dimensions; -1 if outside I_N
    int64_t frow = 0;
    R scale = R(1);
    bool inside = true;
    if constexpr (D == 3) {
      int p1 = (int)(row % a.Nt[1]);
      int p0 = (int)(row / a.Nt[1]);
      int l0 = p0 < a.Nt[0] / 2 ? p0 : p0 - a.Nt[0];
      int l1 = p1 < a.Nt[1] / 2 ? p1 : p1 - a.Nt[1];
      int i0 = l0 + a.N[0] / 2, i1 = l1 + a.N[1] / 2;
      inside = (i0 >= 0 && i0 < a.N[0] && i1 >= 0 && i1 < a.N[1]);
      if (inside) {
        frow = (int64_t)i0 * a.N[1] + i1;
        scale = beta0[i0] * beta1[i1];
      }
    } else if constexpr (D == 2) {
      int p0 = (int)row;
      int l0 = p0 < a.Nt[0] / 2 ? p0 : p0 - a.Nt[0];
      int i0 = l0 + a.N[0] / 2;
      inside = (i0 >= 0 && i0 < a.N[0]);
      if (inside) {
        frow = i0;
        scale = beta0[i0];
      }
    }
    C out[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int p = 2 * pair + h;
      const int l = p < a.Nt[last] / 2 ? p : p - a.Nt[last];
      const int i = l + a.N[last] / 2;
      C v;
      v.x = R(0);
      v.y = R(0);
      if (inside && i >= 0 && i < a.N[last]) {
        const R* bl = (D == 1) ? beta0 : (D == 2 ? beta1 : beta2);
        const C x = f[frow * a.N[last] + i];
        const R s = scale * bl[i];
        v.x = x.x * s;
        v.y = x.y * s;
      }
      out[h] = v;
    }
    C* dst = grid + row * a.Nt[last] + 2 * pair;
    dst[0] = out[0];
    dst[1] = out[1];
  }
}

template <int D, typename R>
__global__ void deconv_pad_kernel(DeconvArgs a, const typename Cplx<R>::type* __restrict__ f,
                                  typename Cplx<R>::type* __restrict__ grid) {
  deconv_pad_body<D, R>(a, f, grid, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

// Batched: one 1D grid over all problems, problem p owning the blocks
// [block_start[p], block_start[p + 1]) (in proportion to its size, set at
// batch creation), so that small problems do not launch the blocks of the
// largest; sizes and offsets from the problem table.
__device__ __forceinline__ int batch_problem_of_block(const int* __restrict__ block_start, int B) {
  int lo = 0, hi = B;  // block_start[0] = 0 <= blockIdx.x < block_start[B]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (block_start[mid] <= (int)blockIdx.x) lo = mid;
    else hi = mid;
  }
  return lo;
}

template <int D, typename R>
__device__ __forceinline__ DeconvArgs batch_deconv_args(const BatchProblem& P, const R* beta_all) {
  DeconvArgs a{};
  a.D = D;
  int64_t off = P.beta_off;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    a.N[d] = P.N[d];
    a.Nt[d] = P.g.Nt[d];
    a.beta[d] = beta_all + off;
    off += P.N[d];
  }
  return a;
}

template <int D, typename R>
__global__ void deconv_pad_batch_kernel(const BatchProblem* __restrict__ probs, const int* __restrict__ block_start,
                                        int B, const R* __restrict__ beta_all,
                                        const typename Cplx<R>::type* __restrict__ f,
                                        typename Cplx<R>::type* __restrict__ grid) {
  const int p = batch_problem_of_block(block_start, B);
  const BatchProblem& P = probs[p];
  const DeconvArgs a = batch_deconv_args<D, R>(P, beta_all);
  const int b0 = block_start[p], nb = block_start[p + 1] - b0;
  deconv_pad_body<D, R>(a, f + P.in_off, grid + P.grid_off, (blockIdx.x - b0) * (int64_t)blockDim.x + threadIdx.x,
                        (int64_t)nb * blockDim.x);
}

// Algorithm 2, crop and correction step: y_n = g[n mod N~] * prod_d beta_d(n_d),
// n in I_N.
template <int D, typename R>
__device__ __forceinline__ void crop_deconv_body(const DeconvArgs& a, const typename Cplx<R>::type* __restrict__ grid,
                                                 typename Cplx<R>::type* __restrict__ y, int64_t first,
                                                 int64_t stride) {
  using C = typename Cplx<R>::type;
  const R* __restrict__ beta0 = (const R*)a.beta[0];
  const R* __restrict__ beta1 = (const R*)a.beta[D > 1 ? 1 : 0];
  const R* __restrict__ beta2 = (const R*)a.beta[D > 2 ? 2 : 0];
  int64_t total = 1;
  for (int d = 0; d < D; ++d) total *= a.N[d];
  for (int64_t t = first; t < total; t += stride) {
    int64_t rem = t;
    int i[kMaxD];
#pragma unroll
    for (int d = D - 1; d >= 0; --d) {
      i[d] = (int)(rem % a.N[d]);
      rem /= a.N[d];
    }
    int64_t lin = 0;
    R s = R(1);
#pragma unroll
    for (int d = 0; d < D; ++d) {
      int n = i[d] - a.N[d] / 2;
      int p = n < 0 ? n + a.Nt[d] : n;
      lin = lin * a.Nt[d] + p;
      const R* bd = d == 0 ? beta0 : (d == 1 ? beta1 : beta2);
      s *= bd[i[d]];
    }
    C g = grid[lin];
    C out;
    out.x = g.x * s;
    out.y = g.y * s;
    y[t] = out;
  }
}

template <int D, typename R>
__global__ void crop_deconv_kernel(DeconvArgs a, const typename Cplx<R>::type* __restrict__ grid,
                                   typename Cplx<R>::type* __restrict__ y) {
  crop_deconv_body<D, R>(a, grid, y, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

template <int D, typename R>
__global__ void crop_deconv_batch_kernel(const BatchProblem* __restrict__ probs, const int* __restrict__ block_start,
                                         int B, const R* __restrict__ beta_all,
                                         const typename Cplx<R>::type* __restrict__ grid,
                                         typename Cplx<R>::type* __restrict__ y) {
  const int p = batch_problem_of_block(block_start, B);
  const BatchProblem& P = probs[p];
  const DeconvArgs a = batch_deconv_args<D, R>(P, beta_all);
  const int b0 = block_start[p], nb = block_start[p + 1] - b0;
  crop_deconv_body<D, R>(a, grid + P.grid_off, y + P.in_off, (blockIdx.x - b0) * (int64_t)blockDim.x + threadIdx.x,
                         (int64_t)nb * blockDim.x);
}

template <typename R>
cudaError_t launch_deconv_pad(const DeconvArgs& a, const void* f, void* grid, cudaStream_t s) {
  using C = typename Cplx<R>::type;
  int64_t total = 1;
  for (int d = 0; d < a.D; ++d) total *= a.Nt[d];
  int blocks = launch_blocks(total / 2, 256);
  if (a.D == 1)
    deconv_pad_kernel<1, R><<<blocks, 256, 0, s>>>(a, (const C*)f, (C*)grid);
  else if (a.D == 2)
    deconv_pad_kernel<2, R><<<blocks, 256, 0, s>>>(a, (const C*)f, (C*)grid);
  else
    deconv_pad_kernel<3, R><<<blocks, 256, 0, s>>>(a, (const C*)f, (C*)grid);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_crop_deconv(const DeconvArgs& a, const void* grid, void* y, cudaStream_t s) {
  using C = typename Cplx<R>::type;
  int64_t total = 1;
  for (int d = 0; d < a.D; ++d) total *= a.N[d];
  int blocks = launch_blocks(total, 256);
  if (a.D == 1)
    crop_deconv_kernel<1, R><<<blocks, 256, 0, s>>>(a, (const C*)grid, (C*)y);
  else if (a.D == 2)
    crop_deconv_kernel<2, R><<<blocks, 256, 0, s>>>(a, (const C*)grid, (C*)y);
  else
    crop_deconv_kernel<3, R><<<blocks, 256, 0, s>>>(a, (const C*)grid, (C*)y);
  return cudaGetLastError();
}


template <typename R>
cudaError_t launch_deconv_pad_batch(int D, int B, const int* block_start, int blocks, const BatchProblem* probs,
                                    const void* beta_all, const void* f, void* grid, cudaStream_t s) {
  using C = typename Cplx<R>::type;
  const R* beta = (const R*)beta_all;
  if (D == 1)
    deconv_pad_batch_kernel<1, R><<<blocks, kBatchDeconvThreads, 0, s>>>(probs, block_start, B, beta, (const C*)f,
                                                                         (C*)grid);
  else if (D == 2)
    deconv_pad_batch_kernel<2, R><<<blocks, kBatchDeconvThreads, 0, s>>>(probs, block_start, B, beta, (const C*)f,
                                                                         (C*)grid);
  else
    deconv_pad_batch_kernel<3, R><<<blocks, kBatchDeconvThreads, 0, s>>>(probs, block_start, B, beta, (const C*)f,
                                                                         (C*)grid);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_crop_deconv_batch(int D, int B, const int* block_start, int blocks, const BatchProblem* probs,
                                     const void* beta_all, const void* grid, void* y, cudaStream_t s) {
  using C = typename Cplx<R>::type;
  const R* beta = (const R*)beta_all;
  if (D == 1)
    crop_deconv_batch_kernel<1, R><<<blocks, kBatchDeconvThreads, 0, s>>>(probs, block_start, B, beta,
                                                                          (const C*)grid, (C*)y);
  else if (D == 2)
    crop_deconv_batch_kernel<2, R><<<blocks, kBatchDeconvThreads, 0, s>>>(probs, block_start, B, beta,
                                                                          (const C*)grid, (C*)y);
  else
    crop_deconv_batch_kernel<3, R><<<blocks, kBatchDeconvThreads, 0, s>>>(probs, block_start, B, beta,
                                                                          (const C*)grid, (C*)y);
  return cudaGetLastError();
}

template cudaError_t launch_deconv_pad_batch<float>(int, int, const int*, int, const BatchProblem*, const void*,
                                                    const void*, void*, cudaStream_t);
template cudaError_t launch_deconv_pad_batch<double>(int, int, const int*, int, const BatchProblem*, const void*,
                                                     const void*, void*, cudaStream_t);
template cudaError_t launch_crop_deconv_batch<float>(int, int, const int*, int, const BatchProblem*, const void*,
                                                     const void*, void*, cudaStream_t);
template cudaError_t launch_crop_deconv_batch<double>(int, int, const int*, int, const BatchProblem*, const void*,
                                                      const void*, void*, cudaStream_t);

template cudaError_t launch_deconv_pad<float>(const DeconvArgs&, const void*, void*, cudaStream_t);
template cudaError_t launch_deconv_pad<double>(const DeconvArgs&, const void*, void*, cudaStream_t);
template cudaError_t launch_crop_deconv<float>(const DeconvArgs&, const void*, void*, cudaStream_t);
template cudaError_t launch_crop_deconv<double>(const DeconvArgs&, const void*, void*, cudaStream_t);

// ---------------------------------------------------------------------------
// Node bin-sort (set_nodes).
// x = N~_d k_{j,d} in FP64; cell c = floor(x) mod N~_d; fraction t = x - floor(x).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double load_k(const void* k, int k_is_fp64, int64_t idx) {
  return k_is_fp64 ? ((const double*)k)[idx] : (double)((const float*)k)[idx];
}

__device__ __forceinline__ void split_coord(double kv, int Nt, int& cell, double& t) {
  double x = (double)Nt * kv;
  double fl = floor(x);
  t = x - fl;
  long long c = (long long)fl % (long long)Nt;
  if (c < 0) c += Nt;
  cell = (int)c;
}

__global__ void node_count_kernel(SortArgs a, const void* k, int k_is_fp64, int* tile_count,
                                  int* key, int* rank) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < a.M; j += gridDim.x * blockDim.x) {
    int lin = 0;
    for (int d = 0; d < a.D; ++d) {
      int c;
      double t;
      split_coord(load_k(k, k_is_fp64, (int64_t)j * a.D + d), a.Nt[d], c, t);
      lin = lin * a.ntile[d] + c / a.T[d];
    }
    key[j] = lin;
    rank[j] = atomicAdd(tile_count + lin, 1);
  }
}

cudaError_t launch_node_count(const SortArgs& a, const void* k, int k_is_fp64, int* tile_count,
                              int* key, int* rank, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(tile_count, 0, sizeof(int) * (size_t)a.n_tiles, s);
  if (e != cudaSuccess) return e;
  if (a.M == 0) return cudaSuccess;
  node_count_kernel<<<launch_blocks(a.M, 256), 256, 0, s>>>(a, k, k_is_fp64, tile_count, key, rank);
  return cudaGetLastError();
}

// One CTA: exclusive scan of the tile counts and of the per-tile work-item
// counts ceil(count / cmax); then every non-empty tile writes its items.
constexpr int kScanThreads = 1024;

__device__ __forceinline__ int2 block_exclusive_scan2(int2 v, int2* total) {
  __shared__ int2 warp_sums[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int2 incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int x = __shfl_up_sync(0xffffffffu, incl.x, o);
    int y = __shfl_up_sync(0xffffffffu, incl.y, o);
    if (lane >= o) {
      incl.x += x;
      incl.y += y;
    }
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int2 ws = lane < kScanThreads / 32 ? warp_sums[lane] : make_int2(0, 0);
    int2 wi = ws;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int x = __shfl_up_sync(0xffffffffu, wi.x, o);
      int y = __shfl_up_sync(0xffffffffu, wi.y, o);
      if (lane >= o) {
        wi.x += x;
        wi.y += y;
      }
    }
    if (lane < kScanThreads / 32) warp_sums[lane] = make_int2(wi.x - ws.x, wi.y - ws.y);
    if (lane == kScanThreads / 32 - 1) *total = wi;
  }
  __syncthreads();
  int2 base = warp_sums[warp];
  int2 out = make_int2(base.x + incl.x - v.x, base.y + incl.y - v.y);
  __syncthreads();
  return out;
}

__global__ void __launch_bounds__(kScanThreads)
    tile_scan_kernel(SortArgs a, const int* tile_count, int* tile_offset, int4* items, int* n_items) {
  __shared__ int2 total;
  int2 carry = make_int2(0, 0);
  for (int base = 0; base < a.n_tiles; base += kScanThreads) {
    const int t = base + threadIdx.x;
    const int cnt = t < a.n_tiles ? tile_count[t] : 0;
    const int nit = (cnt + a.cmax - 1) / a.cmax;
    int2 ex = block_exclusive_scan2(make_int2(cnt, nit), &total);
    __syncthreads();
    if (t < a.n_tiles) {
      const int off = carry.x + ex.x;
      const int ioff = carry.y + ex.y;
      tile_offset[t] = off;
      for (int r = 0; r < nit && ioff + r < a.max_items; ++r) {
        const int first = r * a.cmax;
        const int c = min(a.cmax, cnt - first);
        items[ioff + r] = make_int4(t, off + first, c, 0);
      }
    }
    carry.x += total.x;
    carry.y += total.y;
    __syncthreads();
  }
  if (threadIdx.x == 0) *n_items = min(carry.y, a.max_items);
}

cudaError_t launch_tile_scan(const SortArgs& a, const int* tile_count, int* tile_offset, int4* items,
                             int* n_items, cudaStream_t s) {
  tile_scan_kernel<<<1, kScanThreads, 0, s>>>(a, tile_count, tile_offset, items, n_items);
  return cudaGetLastError();
}

__global__ void node_place_kernel(SortArgs a, const void* k, int k_is_fp64, const int* key,
                                  const int* rank, const int* tile_offset, int* cell, void* frac,
                                  int frac_is_fp64, int* perm) {
  const int64_t M = a.M;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < a.M; j += gridDim.x * blockDim.x) {
    const int pos = tile_offset[key[j]] + rank[j];
    for (int d = 0; d < a.D; ++d) {
      int c;
      double t;
      split_coord(load_k(k, k_is_fp64, (int64_t)j * a.D + d), a.Nt[d], c, t);
      cell[d * M + pos] = c;
      if (frac_is_fp64) {
        ((double*)frac)[d * M + pos] = t;
      } else {
        // round to FP32, keeping t < 1
        float tf = (float)t;
        if (tf >= 1.0f) tf = 0.99999994f;
        ((float*)frac)[d * M + pos] = tf;
      }
    }
    perm[pos] = j;
  }
}

cudaError_t launch_node_place(const SortArgs& a, const void* k, int k_is_fp64, const int* key,
                              const int* rank, const int* tile_offset, int* cell, void* frac,
                              int frac_is_fp64, int* perm, cudaStream_t s) {
  if (a.M == 0) return cudaSuccess;
  node_place_kernel<<<launch_blocks(a.M, 256), 256, 0, s>>>(a, k, k_is_fp64, key, rank, tile_offset,
                                                            cell, frac, frac_is_fp64, perm);
  return cudaGetLastError();
}

// Copy a node set's work items into the batch list, tagging them with problem p.
__global__ void items_expand_kernel(const int4* src, const int* n_src, int4* dst, const int* dst_off, int p) {
  const int n = *n_src;
  const int base = *dst_off;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int4 v = src[i];
    v.w = p;
    dst[base + i] = v;
  }
}

cudaError_t launch_items_expand(const int4* src, const int* n_src, int max_n, int4* dst, const int* dst_off, int p,
                                cudaStream_t s) {
  items_expand_kernel<<<launch_blocks(max_n, 256), 256, 0, s>>>(src, n_src, dst, dst_off, p);
  return cudaGetLastError();
}

}  // namespace nfftgb
