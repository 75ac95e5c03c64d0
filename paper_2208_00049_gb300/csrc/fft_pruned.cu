// Pruned 3D FFT with the resampling correction fused in, for N~ = 2N = 256 per
// dimension (complex64): the correction + zero-pad + FFT steps of Algorithm 1
// and the inverse FFT + crop + correction steps of Algorithm 2 in three
// one-dimensional passes each.
//
// Forward.  g is non-zero only on I_N (after the zero pad), so the 3D DFT of
// the FFT step factorises into passes that each touch only non-zero data:
//   A: rows (i0, i1) in [0,N)^2:   read f * beta, DFT along dim 2   -> N x N x N~
//   B: lines (i0, l2), i0 < N:     DFT along dim 1                  -> N x N~ x N~
//   C: lines (l1, l2):             DFT along dim 0                  -> N~ x N~ x N~
// Each line holds its N inputs at array index i = n + N/2; the fftshift of
// Sec. 3.5 becomes the exact post-phase exp(i pi N l / N~) = i^l (N~ = 2N).
// Adjoint (inverse FFT, crop, correction): the same passes in reverse keep
// only the N outputs of each inverse DFT, with the pre-phase (-i)^l, and the
// last pass multiplies by the correction and writes y.  HBM traffic: 352 MB per direction at N = 128
// against about 950 MB for a separate correction pass plus a full 3D FFT.
//
// A 256-point line DFT is 16 x 16: thread r of the line's 16 takes the
// 16-point DFT over n1 of x[16 n1 + r], multiplies by exp(-2 pi i r k1/256),
// and after a transpose in shared memory thread k1 takes the 16-point DFT
// over n2, giving X[k1 + 16 k2].  The 16-point DFTs are 4 x 4 in registers
// with constant twiddles.
//
// Thread layouts make every global access coalesced without staging: in a row
// pass (line contiguous) thread (line, r) loads x[16 n1 + r], 16 lanes reading
// 128 consecutive bytes; in a column pass 16 adjacent lines (columns) are
// handled together and thread (line, r) loads row 16 n1 + r of its column, a
// half-warp again reading 128 consecutive bytes.  Stage-2 thread k1 holds
// X[k1 + 16 k2], k2 = 0..15, and stores them in the same pattern.  One
// shared-memory transpose and one barrier per pass.
//
// The phases fold into the inter-stage twiddles: output n = k1 + 16 k2 has
// i^n = i^k1 (constant per stage-2 thread) and input n = 16 n1 + r has
// (-i)^n = (-i)^r (constant per stage-1 thread), so the tables are
//   forward  W256^(r k1) i^k1,   inverse  conj(W256^(r k1)) (-i)^r,
// built in FP64 on the device.
#include "nfft_internal.cuh"

namespace nfftgb {
namespace {

constexpr int kLen = 256;
constexpr int kHalf = 128;
#ifndef NFFT_PRUNED_LINES
#define NFFT_PRUNED_LINES 16
#endif
#ifndef NFFT_PRUNED_MIN_CTAS
#define NFFT_PRUNED_MIN_CTAS 4
#endif
constexpr int kLines = NFFT_PRUNED_LINES;     // lines per CTA
constexpr int kThreads = 16 * kLines;         // 16 threads per line
constexpr int kMinCtas = NFFT_PRUNED_MIN_CTAS;  // CTAs per SM the register cap allows
static_assert(kLines == 8 || kLines == 16, "lines per CTA");

// Transpose buffers.  Row passes: [line][a][b], pitch 17 along a.  Column
// passes: [a][b][line] (lines fastest, 8 complex of padding per a when
// kLines = 8 so that the two r of a half-warp fall in different banks).
constexpr int kRowT = kLines * 16 * 17;
constexpr int kColPad = kLines == 8 ? 8 : 0;
constexpr int kColT = 16 * (16 * kLines + kColPad);
constexpr int kTSize = kRowT > kColT ? kRowT : kColT;
static_assert(kTSize * 8 <= 48 * 1024, "static shared-memory launch");

__device__ __forceinline__ int row_t(int line, int a, int b) { return line * (16 * 17) + a * 17 + b; }
__device__ __forceinline__ int col_t(int line, int a, int b) { return a * (16 * kLines + kColPad) + b * kLines + line; }

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 conj_if(float2 w, bool c) { return c ? make_float2(w.x, -w.y) : w; }
__device__ __forceinline__ float2 cscale(float2 a, float b) { return make_float2(a.x * b, a.y * b); }

// W16^k = exp(-2 pi i k/16) for the products n2 k1 of the 4 x 4 split
// (k in {1, 2, 3, 4, 6, 9}); cos(pi/8), sin(pi/8) and sqrt(1/2).
constexpr float kC8 = 0.92387953251128674f;
constexpr float kS8 = 0.38268343236508977f;
constexpr float kR2 = 0.70710678118654752f;
template <int K>
__device__ __forceinline__ float2 w16() {
  static_assert(K == 1 || K == 2 || K == 3 || K == 4 || K == 6 || K == 9, "W16 power");
  if constexpr (K == 1) return make_float2(kC8, -kS8);
  if constexpr (K == 2) return make_float2(kR2, -kR2);
  if constexpr (K == 3) return make_float2(kS8, -kC8);
  if constexpr (K == 4) return make_float2(0.f, -1.f);
  if constexpr (K == 6) return make_float2(-kR2, -kR2);
  return make_float2(-kC8, kS8);  // K == 9
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  const float2 s02 = cadd(a0, a2), d02 = csub(a0, a2), s13 = cadd(a1, a3), d13 = csub(a1, a3);
  // forward W4 = -i: -i d13 = (d13.y, -d13.x); inverse W4 = +i
  const float2 j13 = INV ? make_float2(-d13.y, d13.x) : make_float2(d13.y, -d13.x);
  a0 = cadd(s02, s13);
  a2 = csub(s02, s13);
  a1 = cadd(d02, j13);
  a3 = csub(d02, j13);
}

template <bool INV, int K>
__device__ __forceinline__ void tw16(float2& a) {
  if constexpr (K == 4) {
    a = INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);  // * -+i
  } else {
    a = cmul(a, conj_if(w16<K>(), INV));
  }
}

// 16-point DFT in registers, in place with the output permuted:
// on return x[4 k1 + k2] = X[k1 + 4 k2] = sum_n x[n] W16^(n k),
// n = 4 n1 + n2 (W16 = exp(-+2 pi i/16)).
template <bool INV>
__device__ __forceinline__ void dft16(float2* x) {
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4<INV>(x[n2], x[4 + n2], x[8 + n2], x[12 + n2]);
  // x[4 k1 + n2] = A[n2][k1]; twiddle W16^(n2 k1)
  tw16<INV, 1>(x[5]);
  tw16<INV, 2>(x[6]);
  tw16<INV, 3>(x[7]);
  tw16<INV, 2>(x[9]);
  tw16<INV, 4>(x[10]);
  tw16<INV, 6>(x[11]);
  tw16<INV, 3>(x[13]);
  tw16<INV, 6>(x[14]);
  tw16<INV, 9>(x[15]);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4<INV>(x[4 * k1], x[4 * k1 + 1], x[4 * k1 + 2], x[4 * k1 + 3]);
}

// X[k] of dft16's output: x[4 (k & 3) + (k >> 2)]
__device__ __forceinline__ constexpr int perm16(int k) { return 4 * (k & 3) + (k >> 2); }

// The 256-point line DFT around the loads and stores: on entry x[n1] =
// x_line[16 n1 + r] (thread (line, r)), on return x[perm16(k2)] =
// X_line[r + 16 k2] (thread (line, k1 = r)), phases included.  COL selects
// the transpose layout.  One barrier.
template <bool INV, bool COL>
__device__ __forceinline__ void line_dft256(float2* x, float2* T, const float2* __restrict__ tw, int line, int r) {
  dft16<INV>(x);
  const float2* twr = tw + (INV ? kLen : 0) + r;
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) {
    const float2 v = cmul(x[perm16(k1)], __ldg(twr + 16 * k1));
    T[COL ? col_t(line, k1, r) : row_t(line, k1, r)] = v;
  }
  __syncthreads();
#pragma unroll
  for (int n2 = 0; n2 < 16; ++n2) x[n2] = T[COL ? col_t(line, r, n2) : row_t(line, r, n2)];
  dft16<INV>(x);
}

// Pass A (forward): rows (i0, i1) of f times the correction, DFT along dim 2,
// into the grid rows (i0, i1, :).
__global__ void __launch_bounds__(kThreads, kMinCtas)
    fwd_rows_kernel(const float2* __restrict__ f, const float* __restrict__ beta0, const float* __restrict__ beta1,
                    const float* __restrict__ beta2, const float2* __restrict__ tw, float2* __restrict__ grid) {
  __shared__ float2 T[kTSize];
  const int t = threadIdx.x, line = t >> 4, r = t & 15;
  const int row = blockIdx.x * kLines + line, i0 = row / kHalf, i1 = row - i0 * kHalf;
  const float2* src = f + (int64_t)row * kHalf + r;
  float2 x[16];
#pragma unroll
  for (int n1 = 0; n1 < 8; ++n1) x[n1] = src[16 * n1];
  const float b01 = beta0[i0] * beta1[i1];
#pragma unroll
  for (int n1 = 0; n1 < 8; ++n1) x[n1] = cscale(x[n1], b01 * beta2[16 * n1 + r]);
#pragma unroll
  for (int n1 = 8; n1 < 16; ++n1) x[n1] = make_float2(0.f, 0.f);
  line_dft256<false, false>(x, T, tw, line, r);
  float2* dst = grid + ((int64_t)i0 * kLen + i1) * kLen + r;
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) dst[16 * k2] = x[perm16(k2)];
}

// Passes B and C (forward): kLines adjacent columns (element stride S, first
// element at base + line) read N inputs, write N~ outputs in place.  Passes
// C' and B' (adjoint): read N~ inputs, write the N outputs of the inverse DFT
// in place.
template <bool INV>
__global__ void __launch_bounds__(kThreads, kMinCtas)
    cols_kernel(float2* __restrict__ grid, int64_t outer_stride, int64_t S, const float2* __restrict__ tw) {
  __shared__ float2 T[kTSize];
  constexpr int NIN1 = (INV ? kLen : kHalf) / 16;   // stage-1 inputs per thread
  constexpr int NOUT2 = (INV ? kHalf : kLen) / 16;  // stage-2 outputs per thread
  const int t = threadIdx.x, line = t % kLines, r = t / kLines;
  constexpr int blocks_per_outer = kLen / kLines;
  const int outer = blockIdx.x / blocks_per_outer;
  const int jb = (blockIdx.x - outer * blocks_per_outer) * kLines;
  float2* col = grid + outer * outer_stride + jb + line;
  float2 x[16];
#pragma unroll
  for (int n1 = 0; n1 < 16; ++n1) x[n1] = n1 < NIN1 ? col[(16 * n1 + r) * S] : make_float2(0.f, 0.f);
  line_dft256<INV, true>(x, T, tw, line, r);
#pragma unroll
  for (int k2 = 0; k2 < NOUT2; ++k2) col[(r + 16 * k2) * S] = x[perm16(k2)];
}

// Pass A' (adjoint): rows (i0, i1) of the grid, inverse DFT along dim 2, the
// N outputs times the correction into y.
__global__ void __launch_bounds__(kThreads, kMinCtas)
    adj_rows_kernel(const float2* __restrict__ grid, const float* __restrict__ beta0, const float* __restrict__ beta1,
                    const float* __restrict__ beta2, const float2* __restrict__ tw, float2* __restrict__ y) {
  __shared__ float2 T[kTSize];
  const int t = threadIdx.x, line = t >> 4, r = t & 15;
  const int row = blockIdx.x * kLines + line, i0 = row / kHalf, i1 = row - i0 * kHalf;
  const float2* src = grid + ((int64_t)i0 * kLen + i1) * kLen + r;
  float2 x[16];
#pragma unroll
  for (int n1 = 0; n1 < 16; ++n1) x[n1] = src[16 * n1];
  line_dft256<true, false>(x, T, tw, line, r);
  const float b01 = beta0[i0] * beta1[i1];
  float2* dst = y + (int64_t)row * kHalf + r;
#pragma unroll
  for (int k2 = 0; k2 < 8; ++k2) dst[16 * k2] = cscale(x[perm16(k2)], b01 * beta2[r + 16 * k2]);
}

// tw[16 k1 + r]       = exp(-2 pi i r k1/256) i^k1      (forward)
// tw[256 + 16 k1 + r] = exp(+2 pi i r k1/256) (-i)^r    (inverse)
// in FP64, then rounded.
__global__ void build_twiddles_kernel(float2* tw) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < 2 * kLen) {
    const int inv = j >= kLen, e = j & (kLen - 1), k1 = e >> 4, r = e & 15;
    const double turn = 2.0 * M_PI / (double)kLen;
    const double a = inv ? turn * (double)(r * k1) - 0.5 * M_PI * (double)r
                         : -turn * (double)(r * k1) + 0.5 * M_PI * (double)k1;
    tw[j] = make_float2((float)cos(a), (float)sin(a));
  }
}

// ---------------------------------------------------------------------------
// The 2D form, N~_d = 2 N_d = 512 (N = 256^2, complex64): passes A (rows
// i0 < N: correction, DFT along dim 1) and B (columns: DFT along dim 0) for
// the forward, B' and A' for the adjoint.  A 512-point line DFT is 32 x 16:
// thread r of the line's 16 holds x[16 n1 + r], n1 = 0..31, and takes the
// 32-point DFT over n1 (two 16-point DFTs and a radix-2 step), multiplies by
// the twiddle, and after a transpose in shared memory takes the 16-point
// DFTs over r of k1 = r and k1 = r + 16, giving X[k1 + 32 k2].  The fftshift
// phases fold into the twiddles as in 3D: i^l = i^k1 for l = k1 + 32 k2 and
// (-i)^n = (-i)^r for n = 16 n1 + r, so
//   forward  W512^(r k1) i^k1,   inverse  conj(W512^(r k1)) (-i)^r.
constexpr int kLen2 = 512;
constexpr int kHalf2 = 256;
constexpr int kLines2 = 4;                 // lines per CTA
constexpr int kThreads2 = 16 * kLines2;
constexpr int kColPad2 = 4;                // complex of padding per k1 block (column passes)
constexpr int kT2 = kLines2 * 32 * 17 > 32 * (16 * kLines2 + kColPad2) ? kLines2 * 32 * 17
                                                                        : 32 * (16 * kLines2 + kColPad2);

__device__ __forceinline__ int row_t2(int line, int k1, int r) { return line * (32 * 17) + k1 * 17 + r; }
__device__ __forceinline__ int col_t2(int line, int k1, int r) {
  return k1 * (16 * kLines2 + kColPad2) + r * kLines2 + line;
}

// exp(-2 pi i k/32) = (cos(pi k/16), -sin(pi k/16)), k = 0..15
__constant__ float2 kW32[16] = {
    {1.00000000000000000f, 0.00000000000000000f},  {0.98078528040323043f, 0.19509032201612825f},
    {0.92387953251128674f, 0.38268343236508978f},  {0.83146961230254524f, 0.55557023301960218f},
    {0.70710678118654757f, 0.70710678118654746f},  {0.55557023301960229f, 0.83146961230254524f},
    {0.38268343236508984f, 0.92387953251128674f},  {0.19509032201612833f, 0.98078528040323043f},
    {0.00000000000000006f, 1.00000000000000000f},  {-0.19509032201612819f, 0.98078528040323043f},
    {-0.38268343236508973f, 0.92387953251128674f}, {-0.55557023301960196f, 0.83146961230254546f},
    {-0.70710678118654746f, 0.70710678118654757f}, {-0.83146961230254535f, 0.55557023301960218f},
    {-0.92387953251128674f, 0.38268343236508989f}, {-0.98078528040323043f, 0.19509032201612861f}};

// 32-point DFT of x[n], n = 0..31 (W32 = exp(-+2 pi i/32)), natural order
// out: y[k].  Even and odd halves by dft16, then y[k], y[k + 16] = E[k] +- W32^k O[k].
template <bool INV>
__device__ __forceinline__ void dft32(const float2* x, float2* y) {
  float2 e[16], o[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    e[j] = x[2 * j];
    o[j] = x[2 * j + 1];
  }
  dft16<INV>(e);
  dft16<INV>(o);
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const float2 c = kW32[k];
    const float2 w = INV ? c : make_float2(c.x, -c.y);
    const float2 t = cmul(o[perm16(k)], w);
    y[k] = cadd(e[perm16(k)], t);
    y[k + 16] = csub(e[perm16(k)], t);
  }
}

// The 512-point line DFT: on entry x[n1] = x_line[16 n1 + r], on return
// x[perm16(k2)] = X_line[r + 32 k2] and x[16 + perm16(k2)] = X_line[r + 16 + 32 k2]
// (phases included).  One barrier.
template <bool INV, bool COL>
__device__ __forceinline__ void line_dft512(float2* x, float2* T, const float2* __restrict__ tw, int line, int r) {
  float2 y[32];
  dft32<INV>(x, y);
  const float2* twr = tw + (INV ? kLen2 : 0) + r;
#pragma unroll
  for (int k1 = 0; k1 < 32; ++k1) {
    const float2 v = cmul(y[k1], __ldg(twr + 16 * k1));
    T[COL ? col_t2(line, k1, r) : row_t2(line, k1, r)] = v;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    x[q] = T[COL ? col_t2(line, r, q) : row_t2(line, r, q)];
    x[16 + q] = T[COL ? col_t2(line, r + 16, q) : row_t2(line, r + 16, q)];
  }
  dft16<INV>(x);
  dft16<INV>(x + 16);
}

// Pass A (forward): rows i0 < N of f times the correction, DFT along dim 1,
// into grid rows i0.
__global__ void __launch_bounds__(kThreads2)
    fwd_rows2d_kernel(const float2* __restrict__ f, const float* __restrict__ beta0, const float* __restrict__ beta1,
                      const float2* __restrict__ tw, float2* __restrict__ grid) {
  __shared__ float2 T[kT2];
  const int t = threadIdx.x, line = t >> 4, r = t & 15;
  const int i0 = blockIdx.x * kLines2 + line;
  const float2* src = f + (int64_t)i0 * kHalf2 + r;
  const float b0 = beta0[i0];
  float2 x[32];
#pragma unroll
  for (int n1 = 0; n1 < 16; ++n1) x[n1] = cscale(src[16 * n1], b0 * beta1[16 * n1 + r]);
#pragma unroll
  for (int n1 = 16; n1 < 32; ++n1) x[n1] = make_float2(0.f, 0.f);
  line_dft512<false, false>(x, T, tw, line, r);
  float2* dst = grid + (int64_t)i0 * kLen2 + r;
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) {
    dst[32 * k2] = x[perm16(k2)];
    dst[32 * k2 + 16] = x[16 + perm16(k2)];
  }
}

// Pass B (forward: rows < N in, all N~ rows out) and B' (adjoint: all N~
// rows in, rows < N out) over kLines2 adjacent columns, in place.
template <bool INV>
__global__ void __launch_bounds__(kThreads2)
    cols2d_kernel(float2* __restrict__ grid, const float2* __restrict__ tw) {
  __shared__ float2 T[kT2];
  constexpr int NIN1 = INV ? 32 : 16;   // stage-1 inputs per thread
  constexpr int NOUT2 = INV ? 8 : 16;   // stage-2 outputs per thread and k1 half
  const int t = threadIdx.x, line = t % kLines2, r = t / kLines2;
  float2* col = grid + blockIdx.x * kLines2 + line;
  float2 x[32];
#pragma unroll
  for (int n1 = 0; n1 < 32; ++n1) x[n1] = n1 < NIN1 ? col[(int64_t)(16 * n1 + r) * kLen2] : make_float2(0.f, 0.f);
  line_dft512<INV, true>(x, T, tw, line, r);
#pragma unroll
  for (int k2 = 0; k2 < NOUT2; ++k2) {
    col[(int64_t)(r + 32 * k2) * kLen2] = x[perm16(k2)];
    col[(int64_t)(r + 16 + 32 * k2) * kLen2] = x[16 + perm16(k2)];
  }
}

// Pass A' (adjoint): rows i0 < N of the grid, inverse DFT along dim 1, the
// N outputs times the correction into y.
__global__ void __launch_bounds__(kThreads2)
    adj_rows2d_kernel(const float2* __restrict__ grid, const float* __restrict__ beta0,
                      const float* __restrict__ beta1, const float2* __restrict__ tw, float2* __restrict__ y) {
  __shared__ float2 T[kT2];
  const int t = threadIdx.x, line = t >> 4, r = t & 15;
  const int i0 = blockIdx.x * kLines2 + line;
  const float2* src = grid + (int64_t)i0 * kLen2 + r;
  float2 x[32];
#pragma unroll
  for (int n1 = 0; n1 < 32; ++n1) x[n1] = src[16 * n1];
  line_dft512<true, false>(x, T, tw, line, r);
  const float b0 = beta0[i0];
  float2* dst = y + (int64_t)i0 * kHalf2 + r;
#pragma unroll
  for (int k2 = 0; k2 < 8; ++k2) {
    dst[32 * k2] = cscale(x[perm16(k2)], b0 * beta1[r + 32 * k2]);
    dst[32 * k2 + 16] = cscale(x[16 + perm16(k2)], b0 * beta1[r + 16 + 32 * k2]);
  }
}

// tw[16 k1 + r]       = exp(-2 pi i r k1/512) i^k1      (forward)
// tw[512 + 16 k1 + r] = exp(+2 pi i r k1/512) (-i)^r    (inverse)
// in FP64, then rounded.
__global__ void build_twiddles2d_kernel(float2* tw) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < 2 * kLen2) {
    const int inv = j >= kLen2, e = j & (kLen2 - 1), k1 = e >> 4, r = e & 15;
    const double turn = 2.0 * M_PI / (double)kLen2;
    const double a = inv ? turn * (double)(r * k1) - 0.5 * M_PI * (double)r
                         : -turn * (double)(r * k1) + 0.5 * M_PI * (double)k1;
    tw[j] = make_float2((float)cos(a), (float)sin(a));
  }
}

// ---------------------------------------------------------------------------
// The 3D form at sigma = 1.25: N~_d = 160, N_d = 128 (complex64).  The same
// three passes per direction with 160-point line DFTs, 10 x 16: thread r of
// the line's 16 holds x[16 n1 + r], n1 = 0..9, takes the 10-point DFT over
// n1 (two 5-point DFTs and a radix-2 step), multiplies by W160^(r k1), and
// after a transpose threads k1 < 10 take the 16-point DFT over r, giving
// X[k1 + 10 k2].  N~ is not 2N here, so the fftshift of Sec. 3.5 is the
// phase exp(2 pi i (N/2) l / N~) on output l (forward) and its conjugate on
// input l (adjoint), applied per element from a table.
constexpr int kLen3 = 160;
constexpr int kHalf3 = 128;
constexpr int kLines3 = 16;
constexpr int kThreads3 = 16 * kLines3;
constexpr int kT3 = kLines3 * 10 * 17 > 10 * 16 * kLines3 ? kLines3 * 10 * 17 : 10 * 16 * kLines3;
static_assert(kT3 * 8 <= 48 * 1024, "static shared-memory launch");
constexpr int kTw3Inv = kLen3;       // inverse twiddles at tw[160 + 16 k1 + r]
constexpr int kTw3Phase = 2 * kLen3;  // phases at tw[320 + l]

__device__ __forceinline__ int row_t3(int line, int k1, int r) { return line * (10 * 17) + k1 * 17 + r; }
__device__ __forceinline__ int col_t3(int line, int k1, int r) { return k1 * (16 * kLines3) + r * kLines3 + line; }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// 5-point DFT (W5 = exp(-+2 pi i/5)) in place.
template <bool INV>
__device__ __forceinline__ void dft5(float2& x0, float2& x1, float2& x2, float2& x3, float2& x4) {
  constexpr float c1 = 0.30901699437494745f, c2 = -0.80901699437494734f;
  constexpr float s1 = 0.95105651629515353f, s2 = 0.58778525229247325f;
  const float2 t1 = cadd(x1, x4), t2 = cadd(x2, x3), d1 = csub(x1, x4), d2 = csub(x2, x3);
  const float2 a1 = make_float2(x0.x + c1 * t1.x + c2 * t2.x, x0.y + c1 * t1.y + c2 * t2.y);
  const float2 a2 = make_float2(x0.x + c2 * t1.x + c1 * t2.x, x0.y + c2 * t1.y + c1 * t2.y);
  const float2 e1 = make_float2(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y);
  const float2 e2 = make_float2(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y);
  // b = -+ i e
  const float2 b1 = INV ? make_float2(-e1.y, e1.x) : make_float2(e1.y, -e1.x);
  const float2 b2 = INV ? make_float2(-e2.y, e2.x) : make_float2(e2.y, -e2.x);
  x0 = cadd(x0, cadd(t1, t2));
  x1 = cadd(a1, b1);
  x4 = csub(a1, b1);
  x2 = cadd(a2, b2);
  x3 = csub(a2, b2);
}

// 10-point DFT of x[n] (n = 0..9) into y[k], natural order: 5-point DFTs of
// the even and odd elements, then y[k], y[k + 5] = E[k] +- W10^k O[k].
template <bool INV>
__device__ __forceinline__ void dft10(const float2* x, float2* y) {
  constexpr float wc[5] = {1.0f, 0.80901699437494742f, 0.30901699437494745f, -0.30901699437494734f,
                           -0.80901699437494734f};
  constexpr float ws[5] = {0.0f, 0.58778525229247314f, 0.95105651629515353f, 0.95105651629515364f,
                           0.58778525229247325f};
  float2 e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6], e4 = x[8];
  float2 o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7], o4 = x[9];
  dft5<INV>(e0, e1, e2, e3, e4);
  dft5<INV>(o0, o1, o2, o3, o4);
  const float2 E[5] = {e0, e1, e2, e3, e4}, O[5] = {o0, o1, o2, o3, o4};
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const float2 w = make_float2(wc[k], INV ? ws[k] : -ws[k]);
    const float2 t = cmul(O[k], w);
    y[k] = cadd(E[k], t);
    y[k + 5] = csub(E[k], t);
  }
}

// The 160-point line DFT: on entry x[n1] = x_line[16 n1 + r] (n1 < 10, the
// adjoint's input phase already applied), on return, for threads r < 10,
// x[perm16(k2)] = X_line[r + 10 k2].  One barrier.
template <bool INV, bool COL>
__device__ __forceinline__ void line_dft160(float2* x, float2* T, const float2* __restrict__ tw, int line, int r) {
  float2 y[10];
  dft10<INV>(x, y);
  const float2* twr = tw + (INV ? kTw3Inv : 0) + r;
#pragma unroll
  for (int k1 = 0; k1 < 10; ++k1) {
    const float2 v = cmul(y[k1], __ldg(twr + 16 * k1));
    T[COL ? col_t3(line, k1, r) : row_t3(line, k1, r)] = v;
  }
  __syncthreads();
  if (r < 10) {
#pragma unroll
    for (int q = 0; q < 16; ++q) x[q] = T[COL ? col_t3(line, r, q) : row_t3(line, r, q)];
    dft16<INV>(x);
  }
}

// Pass A (forward): rows (i0, i1) of f times the correction, DFT along dim 2,
// with the output phase, into grid rows (i0, i1, :).
__global__ void __launch_bounds__(kThreads3)
    fwd_rows160_kernel(const float2* __restrict__ f, const float* __restrict__ beta0,
                       const float* __restrict__ beta1, const float* __restrict__ beta2,
                       const float2* __restrict__ tw, float2* __restrict__ grid) {
  __shared__ float2 T[kT3];
  const int t = threadIdx.x, line = t >> 4, r = t & 15;
  const int row = blockIdx.x * kLines3 + line, i0 = row / kHalf3, i1 = row - i0 * kHalf3;
  const float2* src = f + (int64_t)row * kHalf3 + r;
  const float b01 = beta0[i0] * beta1[i1];
  float2 x[16];
#pragma unroll
  for (int n1 = 0; n1 < 8; ++n1) x[n1] = cscale(src[16 * n1], b01 * beta2[16 * n1 + r]);
  x[8] = x[9] = make_float2(0.f, 0.f);
  line_dft160<false, false>(x, T, tw, line, r);
  if (r < 10) {
    float2* dst = grid + ((int64_t)i0 * kLen3 + i1) * kLen3;
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) {
      const int l = r + 10 * k2;
      dst[l] = cmul(x[perm16(k2)], __ldg(tw + kTw3Phase + l));
    }
  }
}

// Passes B, C (forward: N inputs, N~ outputs with the output phase) and C',
// B' (adjoint: N~ inputs with the input phase, the N outputs kept) over
// kLines3 adjacent columns, in place.
template <bool INV>
__global__ void __launch_bounds__(kThreads3)
    cols160_kernel(float2* __restrict__ grid, int64_t outer_stride, int64_t S, const float2* __restrict__ tw) {
  __shared__ float2 T[kT3];
  constexpr int NIN1 = INV ? 10 : 8;
  const int t = threadIdx.x, line = t % kLines3, r = t / kLines3;
  constexpr int blocks_per_outer = kLen3 / kLines3;
  const int outer = blockIdx.x / blocks_per_outer;
  const int jb = (blockIdx.x - outer * blocks_per_outer) * kLines3;
  float2* col = grid + outer * outer_stride + jb + line;
  float2 x[16];
#pragma unroll
  for (int n1 = 0; n1 < 10; ++n1) {
    if (n1 < NIN1) {
      const float2 v = col[(16 * n1 + r) * S];
      x[n1] = INV ? cmul(v, cconj(__ldg(tw + kTw3Phase + 16 * n1 + r))) : v;
    } else {
      x[n1] = make_float2(0.f, 0.f);
    }
  }
  line_dft160<INV, true>(x, T, tw, line, r);
  if (r < 10) {
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) {
      const int l = r + 10 * k2;
      if (!INV)
        col[l * S] = cmul(x[perm16(k2)], __ldg(tw + kTw3Phase + l));
      else if (l < kHalf3)
        col[l * S] = x[perm16(k2)];
    }
  }
}

// Pass A' (adjoint): rows (i0, i1) of the grid with the input phase, inverse
// DFT along dim 2, the N outputs times the correction into y.
__global__ void __launch_bounds__(kThreads3)
    adj_rows160_kernel(const float2* __restrict__ grid, const float* __restrict__ beta0,
                       const float* __restrict__ beta1, const float* __restrict__ beta2,
                       const float2* __restrict__ tw, float2* __restrict__ y) {
  __shared__ float2 T[kT3];
  const int t = threadIdx.x, line = t >> 4, r = t & 15;
  const int row = blockIdx.x * kLines3 + line, i0 = row / kHalf3, i1 = row - i0 * kHalf3;
  const float2* src = grid + ((int64_t)i0 * kLen3 + i1) * kLen3 + r;
  float2 x[16];
#pragma unroll
  for (int n1 = 0; n1 < 10; ++n1) x[n1] = cmul(src[16 * n1], cconj(__ldg(tw + kTw3Phase + 16 * n1 + r)));
  line_dft160<true, false>(x, T, tw, line, r);
  if (r < 10) {
    const float b01 = beta0[i0] * beta1[i1];
    float2* dst = y + (int64_t)row * kHalf3;
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) {
      const int i = r + 10 * k2;
      if (i < kHalf3) dst[i] = cscale(x[perm16(k2)], b01 * beta2[i]);
    }
  }
}

// tw[16 k1 + r]        = exp(-2 pi i r k1/160)   (forward, k1 < 10)
// tw[160 + 16 k1 + r]  = exp(+2 pi i r k1/160)   (inverse)
// tw[320 + l]          = exp(+2 pi i (N/2) l/160), N/2 = 64 (the fftshift phase)
// in FP64, then rounded.
__global__ void build_twiddles160_kernel(float2* tw) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < 3 * kLen3) {
    const double turn = 2.0 * M_PI / (double)kLen3;
    double a;
    if (j < 2 * kLen3) {
      const int e = j % kLen3, k1 = e >> 4, r = e & 15;
      a = (j < kLen3 ? -turn : turn) * (double)(r * k1);
    } else {
      a = turn * (double)(kHalf3 / 2) * (double)(j - 2 * kLen3);
    }
    tw[j] = make_float2((float)cos(a), (float)sin(a));
  }
}

}  // namespace

bool pruned_fft_supported(int D, const int* N, const int* Nt) {
  if (D == 2) return N[0] == kHalf2 && N[1] == kHalf2 && Nt[0] == kLen2 && Nt[1] == kLen2;
  if (D != 3) return false;
  const bool is256 = N[0] == kHalf && Nt[0] == kLen, is160 = N[0] == kHalf3 && Nt[0] == kLen3;
  if (!is256 && !is160) return false;
  for (int d = 1; d < 3; ++d)
    if (N[d] != N[0] || Nt[d] != Nt[0]) return false;
  return true;
}

cudaError_t build_fft_twiddles(int D, int len, float2* tw, cudaStream_t s) {
  static_assert(kPrunedFftTwiddles >= 2 * kLen && kPrunedFftTwiddles >= 2 * kLen2 &&
                    kPrunedFftTwiddles >= 3 * kLen3, "twiddle table size");
  if (D == 2)
    build_twiddles2d_kernel<<<4, kLen2 / 2, 0, s>>>(tw);
  else if (len == kLen3)
    build_twiddles160_kernel<<<3, kLen3, 0, s>>>(tw);
  else
    build_twiddles_kernel<<<2, kLen, 0, s>>>(tw);
  return cudaGetLastError();
}

cudaError_t launch_pruned_forward(int D, int len, const void* f, const float* const* beta, const float2* tw,
                                  void* grid, cudaStream_t s) {
  float2* g = (float2*)grid;
  if (D == 2) {
    fwd_rows2d_kernel<<<kHalf2 / kLines2, kThreads2, 0, s>>>((const float2*)f, beta[0], beta[1], tw, g);
    cols2d_kernel<false><<<kLen2 / kLines2, kThreads2, 0, s>>>(g, tw);
    return cudaGetLastError();
  }
  if (len == kLen3) {
    fwd_rows160_kernel<<<kHalf3 * kHalf3 / kLines3, kThreads3, 0, s>>>((const float2*)f, beta[0], beta[1], beta[2],
                                                                       tw, g);
    // B: lines (i0 < N, l2), element stride N~ (dim 1)
    cols160_kernel<false><<<kHalf3 * (kLen3 / kLines3), kThreads3, 0, s>>>(g, (int64_t)kLen3 * kLen3, kLen3, tw);
    // C: lines (l1, l2), element stride N~^2 (dim 0)
    cols160_kernel<false><<<kLen3 * (kLen3 / kLines3), kThreads3, 0, s>>>(g, kLen3, (int64_t)kLen3 * kLen3, tw);
    return cudaGetLastError();
  }
  fwd_rows_kernel<<<kHalf * kHalf / kLines, kThreads, 0, s>>>((const float2*)f, beta[0], beta[1], beta[2], tw, g);
  // B: lines (i0 < N, l2), element stride N~ (dim 1)
  cols_kernel<false><<<kHalf * (kLen / kLines), kThreads, 0, s>>>(g, (int64_t)kLen * kLen, kLen, tw);
  // C: lines (l1, l2), element stride N~^2 (dim 0)
  cols_kernel<false><<<kLen * (kLen / kLines), kThreads, 0, s>>>(g, kLen, (int64_t)kLen * kLen, tw);
  return cudaGetLastError();
}

cudaError_t launch_pruned_adjoint(int D, int len, void* grid, const float* const* beta, const float2* tw, void* y,
                                  cudaStream_t s) {
  float2* g = (float2*)grid;
  if (D == 2) {
    cols2d_kernel<true><<<kLen2 / kLines2, kThreads2, 0, s>>>(g, tw);
    adj_rows2d_kernel<<<kHalf2 / kLines2, kThreads2, 0, s>>>(g, beta[0], beta[1], tw, (float2*)y);
    return cudaGetLastError();
  }
  if (len == kLen3) {
    // C': lines (l1, l2) along dim 0, keep i0 < N
    cols160_kernel<true><<<kLen3 * (kLen3 / kLines3), kThreads3, 0, s>>>(g, kLen3, (int64_t)kLen3 * kLen3, tw);
    // B': lines (i0 < N, l2) along dim 1, keep i1 < N
    cols160_kernel<true><<<kHalf3 * (kLen3 / kLines3), kThreads3, 0, s>>>(g, (int64_t)kLen3 * kLen3, kLen3, tw);
    adj_rows160_kernel<<<kHalf3 * kHalf3 / kLines3, kThreads3, 0, s>>>(g, beta[0], beta[1], beta[2], tw, (float2*)y);
    return cudaGetLastError();
  }
  // C': lines (l1, l2) along dim 0, keep i0 < N
  cols_kernel<true><<<kLen * (kLen / kLines), kThreads, 0, s>>>(g, kLen, (int64_t)kLen * kLen, tw);
  // B': lines (i0 < N, l2) along dim 1, keep i1 < N
  cols_kernel<true><<<kHalf * (kLen / kLines), kThreads, 0, s>>>(g, (int64_t)kLen * kLen, kLen, tw);
  adj_rows_kernel<<<kHalf * kHalf / kLines, kThreads, 0, s>>>(g, beta[0], beta[1], beta[2], tw, (float2*)y);
  return cudaGetLastError();
}

}  // namespace nfftgb
