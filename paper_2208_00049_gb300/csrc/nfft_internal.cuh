// Internal declarations shared by the translation units of libnfft_gb300.
//
// Layout in HBM (see nfft_plan.cu for allocation):
//   grid   : N~_0 x ... x N~_{D-1} complex, row-major, natural FFT order
//            (grid index l lives at position l mod N~_d).
//   cell   : D planes of M int32, the sorted nodes' cells floor(N~_d k) mod N~_d
//   frac   : D planes of M reals, the sorted nodes' fractions N~_d k - floor(.)
//   perm   : M int32, sorted position -> caller's node index
//   items  : work items {tile, first sorted node, node count, 0}
//   beta   : sum_d N_d reals, the scaled deconvolution vectors
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>
#include <stdint.h>

#include "nfft_gb300.h"

namespace nfftgb {

constexpr int kMaxD = 3;
constexpr int kResampleThreads = 128;
constexpr int kMaxM = 10;

// How the generic resampling kernels obtain window values (Sec. 3.7.4):
// evaluated (sinh, sqrt), looked up in the LINEAR table with linear
// interpolation, or from the POLYNOMIAL coefficients (Horner).
constexpr int kWinDirect = 0;
constexpr int kWinLinear = 1;
constexpr int kWinPoly = 2;

// Everything a resampling kernel needs about the plan, passed by value.
// Dimension d = D-1 is the contiguous one.
struct Geometry {
  int D;
  int Nt[kMaxD];     // oversampled sizes
  int T[kMaxD];      // tile extent in grid cells
  int ntile[kMaxD];  // tiles per dimension
  int L[kMaxD];      // shared-memory region extent = T + K - 1
  int K;             // taps per dimension held by the kernel template
  int off;           // footprint start relative to the cell: -m+1 (or -m closed)
  int closed;        // support [-m, m] instead of [-m, m)
  int M;             // number of nodes
  double m;          // window half-width
  double b[kMaxD];   // Kaiser-Bessel shape per dimension
  double norm[kMaxD];  // m / sinh(b m): scales the window to 1 at u = 0
  // window values of the generic kernels: kWinDirect (wtab unused),
  // kWinLinear (wtab = D tables of wS entries of the scaled window in the
  // plan's real type, table d at d * wS), kWinPoly (wtab = [D][K][wZ]
  // coefficients in the plan's real type, increasing powers of zeta)
  int wmode;
  int wS;
  const void* wtab;
  int wZ;            // kWinPoly: coefficients per tap (degree + 1; 2m + 1, or more for complex128)
};

// Kaiser-Bessel window in grid units, scaled to 1 at u = 0:
//   w(u) = [sinh(b s)/s] * m/sinh(b m),  s = sqrt(m^2 - u^2)     (|u| <= m)
//   w(u) = [sin(b s')/s'] * m/sinh(b m), s' = sqrt(u^2 - m^2)    (|u| > m)
// (the second line is the untruncated window past the support, used by the
// (2m+2)-point footprint).  s^2 is formed as (m - u)(m + u) from the integer
// and fractional parts of u so that it stays accurate near the support
// edges.  At s = 0 both forms tend to b * m/sinh(b m).
//
// In single precision the ratio sinh(b s)/sinh(b m) loses about b m ulps
// (the rounding of the argument b s, up to b m ~ 47 at m = 10, is amplified
// by the exponential), and it loses them at the largest taps.  There the
// same value is taken as
//   w(u) = exp(b (s - m)) (1 - exp(-2 b s)) / s * m/(1 - exp(-2 b m)),
//   b (s - m) = -b u^2 / (s + m),
// whose exponent is small where the window is large, so the error of each
// tap scales with its own size.
template <typename R>
__device__ __forceinline__ R kb_window(R u, R mm_u, R mp_u, R b, R norm, R m, R normx) {
  const R s2 = mm_u * mp_u;
  const R s = sqrt(s2 > R(0) ? s2 : -s2);
  const R z = b * s;
  R r;
  if (s2 >= R(0)) {
    if (z < R(1e-3))
      r = b * (R(1) + z * z * R(1.0 / 6.0));
    else if (sizeof(R) == 4)
      return exp(-b * (u * u) / (s + m)) * (-expm1(R(-2) * z)) / s * normx;
    else
      r = sinh(z) / s;
  } else {
    r = (z < R(1e-3)) ? b * (R(1) - z * z * R(1.0 / 6.0)) : sin(z) / s;
  }
  return r * norm;
}

// m/(1 - exp(-2 b m)): the scale of the single-precision form above.
template <typename R>
__device__ __forceinline__ R kb_normx(R b, R m) {
  return m / (-expm1(R(-2) * b * m));
}

// Derivative of the scaled window with respect to u:
//   |u| <= m: w'(u) = -u (b s cosh(b s) - sinh(b s)) / s^3 * m/sinh(b m)
//   |u| > m:  w'(u) = +u (b s' cos(b s') - sin(b s')) / s'^3 * m/sinh(b m)
// with the series b^3 (1/3 + z^2/30 + z^4/840 + z^6/45360) inside and
// b^3 (-1/3 + z^2/30 - z^4/840 + z^6/45360) outside for small z = b s.
// Single precision takes z cosh z - sinh z = e^z ((z - 1) + (z + 1) e^{-2z}) / 2
// inside, scaled as in kb_window (normx carries the factor N~ of norm).
template <typename R>
__device__ __forceinline__ R kb_window_deriv(R u, R mm_u, R mp_u, R b, R norm, R zsmall, R m, R normx) {
  const R s2 = mm_u * mp_u;
  const R s = sqrt(s2 > R(0) ? s2 : -s2);
  const R z = b * s;
  const R z2 = z * z;
  R h;
  if (s2 >= R(0)) {
    if (z < zsmall) {
      h = b * b * b * (R(1.0 / 3.0) + z2 * (R(1.0 / 30.0) + z2 * (R(1.0 / 840.0) + z2 * R(1.0 / 45360.0))));
    } else if (sizeof(R) == 4) {
      const R e = -b * (u * u) / (s + m);
      const R g = (z - R(1)) + (z + R(1)) * exp(R(-2) * z);
      return -u * exp(e) * g / (s * s * s) * normx;
    } else {
      h = (z * cosh(z) - sinh(z)) / (s * s * s);
    }
    return -u * h * norm;
  }
  if (z < zsmall)
    h = b * b * b * (R(-1.0 / 3.0) + z2 * (R(1.0 / 30.0) + z2 * (R(-1.0 / 840.0) + z2 * R(1.0 / 45360.0))));
  else
    h = (z * cos(z) - sin(z)) / (s * s * s);
  return u * h * norm;
}

// ---- launchers (one per translation unit) ------------------------------
struct NodeArrays {
  const int* cell;   // D planes of M
  const void* frac;  // D planes of M reals
  const int* perm;   // M
  const int4* items;
  const int* n_items;
};

// Batched execution: one problem of a batch (geometry and buffer offsets).
struct BatchProblem {
  Geometry g;        // g.M = the problem's node count
  int N[kMaxD];      // coefficient sizes
  int64_t grid_off;  // complex elements into the batch grid buffer
  int64_t node_off;  // node-set offset: cell / frac planes start at D * node_off, perm at node_off
  int64_t out_off;   // offset of this problem's fhat in the concatenated fhat buffer
  int64_t in_off;    // offset of this problem's f / y in the concatenated coefficient buffer
  int64_t beta_off;  // offset of this problem's deconvolution vectors
  int64_t poly_off;  // offset of this problem's POLYNOMIAL coefficients
};
struct BatchNodes {
  const int* cell;
  const void* frac;
  const int* perm;   // node-set-local indices
  const int4* items; // {tile, first sorted node (set-local), count, problem}
  const int* n_items;
};
template <typename R>
cudaError_t launch_gather_batch(const BatchProblem* probs_dev, const Geometry& gmax, const void* grid,
                                const BatchNodes& nb, void* fhat, int ctas, cudaStream_t s);
template <typename R>
cudaError_t launch_scatter_batch(const BatchProblem* probs_dev, const Geometry& gmax, void* grid,
                                 const BatchNodes& nb, const void* fhat, int ctas, cudaStream_t s);
template <typename R>
int resample_batch_ctas_per_sm(const Geometry& gmax, int kind);  // kind 0 gather, 1 scatter

template <typename R>
cudaError_t launch_gather(const Geometry& g, const void* grid, const NodeArrays& na,
                          void* fhat, int grid_ctas, cudaStream_t s);
template <typename R>
cudaError_t launch_scatter(const Geometry& g, void* grid, const NodeArrays& na,
                           const void* fhat, int compensated, int grid_ctas, cudaStream_t s);
template <typename R>
cudaError_t launch_grad_gather(const Geometry& g, const void* grid, const NodeArrays& na,
                               const void* cot, void* gk, int grid_ctas, cudaStream_t s);
template <typename R>
size_t resample_smem_bytes(const Geometry& g, int kind);  // kind 0 gather, 1 scatter, 2 scatter+comp
template <typename R>
int resample_ctas_per_sm(const Geometry& g, int kind);

// 3D, m = 4, complex64 warp-per-node kernels (resample3d.cu); `poly` holds
// the FP32 polynomial window coefficients [3][8][9] (launch_build_poly).
bool fast3d_supported(const Geometry& g, int cmax);
// 3D m = 4 complex64 node gradient with the gather's layout (resample3d.cu)
int grad3d_ctas_per_sm(const Geometry& g);
cudaError_t launch_grad3d_fast(const Geometry& g, const void* grid, const NodeArrays& na, const float* poly,
                               const void* cot, void* gk, int ctas, cudaStream_t s);
// 3D complex64 register-accumulating scatter, m = 4 or 6 (any tile of at
// most 17 - 2m cells per dimension); kind 1 of the two functions below.
bool fast_scatter_supported(const Geometry& g, int cmax);
int fast3d_ctas_per_sm(const Geometry& g, int kind);  // kind 0 gather, 1 scatter, 2 compensated scatter
// 1 if a CTA of the 3D gather / node gradient gave up its bounded wait for a
// region copy since the last call (the flag is cleared), 0 if not, -1 if the
// flag could not be read.  Synchronous; call with the plan's device current.
int fast3d_take_wait_timeout();
cudaError_t launch_gather3d_fast(const Geometry& g, const void* grid, const NodeArrays& na,
                                 const float* poly, void* fhat, int ctas, cudaStream_t s);
// compensated != 0: TwoSum-compensated accumulation (NFFT_FLAG_COMPENSATED)
cudaError_t launch_scatter3d_fast(const Geometry& g, void* grid, const NodeArrays& na,
                                  const float* poly, const void* fhat, int compensated, int ctas, cudaStream_t s);

// Pruned FFT with the resampling correction fused in, complex64
// (fft_pruned.cu): 3D with N~_d = 2 N_d = 256 or N~_d = 160, N_d = 128, and
// 2D with N~_d = 2 N_d = 512 (len = N~_0).  `tw` holds the inter-stage
// twiddles (and phases) of that form (build_fft_twiddles, at most
// kPrunedFftTwiddles); beta[d] are the FP32 correction vectors.
constexpr int kPrunedFftTwiddles = 1024;
bool pruned_fft_supported(int D, const int* N, const int* Nt);
cudaError_t build_fft_twiddles(int D, int len, float2* tw, cudaStream_t s);
cudaError_t launch_pruned_forward(int D, int len, const void* f, const float* const* beta, const float2* tw,
                                  void* grid, cudaStream_t s);
cudaError_t launch_pruned_adjoint(int D, int len, void* grid, const float* const* beta, const float2* tw, void* y,
                                  cudaStream_t s);

// Small 1D complex128 plans (dft1d.cu): correction + pad + FFT and inverse
// FFT + crop + correction as direct sums spread over every SM; `tw` holds
// the N~ roots of unity e^{-2 pi i k / N~} in FP64.
bool dft1d_supported(int D, int N, int Nt);
cudaError_t launch_dft_twiddles(double2* tw, int Nt, cudaStream_t s);
cudaError_t launch_dft1d_forward(int N, int Nt, const void* f, const double* beta, const double2* tw, void* grid,
                                 int sms, cudaStream_t s);
cudaError_t launch_dft1d_adjoint(int N, int Nt, const void* grid, const double* beta, const double2* tw, void* y,
                                 int sms, cudaStream_t s);

// 2D, m = 4, complex64 register-accumulating scatter and warp-per-item
// gather (resample2d.cu): tiles of at most 9 cells in dimension 0 and
// regions of at most 32 in dimension 1.
bool scatter2d_supported(const Geometry& g);
int scatter2d_ctas_per_sm(int compensated = 0);
int gather2d_ctas_per_sm();
// poly: POLYNOMIAL coefficients [D][K][2m + 1] of the plan, or of all
// problems of a batch (problem p's table at poly + probs[p].poly_off).
cudaError_t launch_gather2d_fast(const Geometry& g, const void* grid, const NodeArrays& na, const float* poly,
                                 void* fhat, int ctas, cudaStream_t s);
cudaError_t launch_gather2d_fast_batch(const BatchProblem* probs, const void* grid, const BatchNodes& nb,
                                       const float* poly, void* fhat, int ctas, cudaStream_t s);
cudaError_t launch_scatter2d_fast(const Geometry& g, void* grid, const NodeArrays& na, const float* poly,
                                  const void* fhat, int compensated, int ctas, cudaStream_t s);
cudaError_t launch_scatter2d_fast_batch(const BatchProblem* probs, void* grid, const BatchNodes& nb,
                                        const float* poly, const void* fhat, int ctas, cudaStream_t s);

// 2D complex128 scatter without shared-memory atomics (resample2d_f64.cu):
// even K = 2m <= 16 taps, half-open support, any window form; one work item
// per CTA (scatter2d_f64_items_per_cta()).
bool scatter2d_f64_supported(const Geometry& g);
int scatter2d_f64_ctas_per_sm(const Geometry& g);
int scatter2d_f64_items_per_cta();
cudaError_t launch_scatter2d_f64(const Geometry& g, void* grid, const NodeArrays& na, const void* fhat, int ctas,
                                 cudaStream_t s);
// 3D counterpart (resample3d_f64.cu): even K = 2m <= 8, one work item per CTA.
bool scatter3d_f64_supported(const Geometry& g);
int scatter3d_f64_ctas_per_sm(const Geometry& g);
cudaError_t launch_scatter3d_f64(const Geometry& g, void* grid, const NodeArrays& na, const void* fhat, int ctas,
                                 cudaStream_t s);

// FULL precomputation: B as a CSR matrix, applied with cuSPARSE (nfft_full.cu)
struct FullMatrix;
int full_build(FullMatrix** out, const Geometry& g, int dtype, const NodeArrays& na, cudaStream_t s);
int full_forward(FullMatrix* F, const void* grid, void* fhat, cudaStream_t s);
int full_adjoint(FullMatrix* F, const void* fhat, void* grid, cudaStream_t s);
void full_destroy(FullMatrix* F);

// deconvolution, tables, sorting (nfft_kernels.cu)
struct DeconvArgs {
  int D;
  int N[kMaxD];
  int Nt[kMaxD];
  const void* beta[kMaxD];  // per-dimension beta vectors (plan real type)
};
template <typename R>
cudaError_t launch_deconv_pad(const DeconvArgs& a, const void* f, void* grid, cudaStream_t s);
template <typename R>
cudaError_t launch_crop_deconv(const DeconvArgs& a, const void* grid, void* y, cudaStream_t s);

struct PolyArgs {
  int D;
  int K;     // taps per dimension
  int off;   // first tap offset (-m + 1)
  int deg;   // polynomial degree (2m)
  int m;
  double b[kMaxD];
};
// coef and coef64 (either may be null) receive the FP32 and FP64
// coefficients [D][K][deg + 1].
cudaError_t launch_build_poly(const PolyArgs& a, float* coef, cudaStream_t s, double* coef64 = nullptr);

// LINEAR window tables (Sec. 3.7.4): for each dimension d, entries
// s = 0 .. S - 1 of the window scaled to 1 at u = 0, at u = m s / (S - 2) on
// its closed support and 0 beyond (entry S - 1), S = m 2^{c_min(m,8)} + 2;
// computed in FP64, stored in FP32 (lut32) and/or FP64 (lut64).
int64_t lut_table_size(int m);
cudaError_t launch_build_lut(int D, int m, const double* b, int64_t S, float* lut32, double* lut64, cudaStream_t s);

// Batched correction kernels: one 1D grid of `blocks` blocks of
// kBatchDeconvThreads threads, problem p owning blocks
// [block_start[p], block_start[p + 1]) (device array of B + 1 entries).
constexpr int kBatchDeconvThreads = 256;
template <typename R>
cudaError_t launch_deconv_pad_batch(int D, int B, const int* block_start, int blocks, const BatchProblem* probs,
                                    const void* beta_all, const void* f, void* grid, cudaStream_t s);
template <typename R>
cudaError_t launch_crop_deconv_batch(int D, int B, const int* block_start, int blocks, const BatchProblem* probs,
                                     const void* beta_all, const void* grid, void* y, cudaStream_t s);
cudaError_t launch_items_expand(const int4* src, const int* n_src, int max_n, int4* dst, const int* dst_off, int p,
                                cudaStream_t s);

cudaError_t launch_build_beta(int D, const int* N, const int* Nt, int m, const double* b,
                              double* beta64, float* beta32, cudaStream_t s);

struct SortArgs {
  int D;
  int M;
  int Nt[kMaxD];
  int T[kMaxD];
  int ntile[kMaxD];
  int n_tiles;
  int cmax;
  int max_items;
};
cudaError_t launch_node_count(const SortArgs& a, const void* k, int k_is_fp64, int* tile_count,
                              int* key, int* rank, cudaStream_t s);
cudaError_t launch_tile_scan(const SortArgs& a, const int* tile_count, int* tile_offset,
                             int4* items, int* n_items, cudaStream_t s);
cudaError_t launch_node_place(const SortArgs& a, const void* k, int k_is_fp64, const int* key,
                              const int* rank, const int* tile_offset, int* cell, void* frac,
                              int frac_is_fp64, int* perm, cudaStream_t s);

}  // namespace nfftgb
