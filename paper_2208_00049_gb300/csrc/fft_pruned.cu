// Pruned 3D FFT with the resampling correction fused in, for N~ = 2N = 256 per
// dimension (complex64): Algorithm 1 lines 1-6 and Algorithm 2 lines 4-10 in
// three one-dimensional passes each.
//
// Forward.  g is non-zero only on I_N (Algorithm 1 lines 1-3), so the 3D DFT
// (lines 4-6) factorises into passes that each touch only non-zero data:
//   A: rows (i0, i1) in [0,N)^2:   read f * beta, DFT along dim 2   -> N x N x N~
//   B: lines (i0, l2), i0 < N:     DFT along dim 1                  -> N x N~ x N~
//   C: lines (l1, l2):             DFT along dim 0                  -> N~ x N~ x N~
// Each line holds its N inputs at array index i = n + N/2; the fftshift of
// Sec. 3.5 becomes the exact post-phase exp(i pi N l / N~) = i^l (N~ = 2N).
// Adjoint (lines 4-10): the same passes in reverse keep only the N outputs of
// each inverse DFT, with the pre-phase (-i)^l, and the last pass multiplies by
// the correction and writes y.  HBM traffic: 352 MB per direction at N = 128
// against about 950 MB for a separate correction pass plus a full 3D FFT.
//
// A 256-point line DFT is 16 x 16: thread n2 of the line's 16 takes the
// 16-point DFT over n1 of x[16 n1 + n2], multiplies by exp(-2 pi i n2 k1/256),
// and after a transpose thread k1 takes the 16-point DFT over n2, giving
// X[k1 + 16 k2].  The 16-point DFTs are 4 x 4 in registers with constant
// twiddles; the 16 x 16 inter-stage twiddles come from a table built in FP64
// on the device.
//
// Latency, not bandwidth, limits passes like these: every pass loads all of a
// CTA's lines with fully unrolled loads before the first shared-memory store,
// the transpose buffer aliases the staging buffer (about 19 KB per CTA), and
// registers are capped so that 8 CTAs share an SM.
#include "nfft_internal.cuh"

namespace nfftgb {
namespace {

constexpr int kLen = 256;
constexpr int kHalf = 128;
constexpr int kLines = 8;                 // lines per CTA
constexpr int kThreads = 16 * kLines;     // 16 threads per line
constexpr int kSweep = kThreads / kLines; // rows of the column block per CTA-wide load
constexpr int kBufPitch = kLen + 2;       // line pitch (complex): column staging conflict-free
constexpr int kTPitch = 17;               // padded pitch of the 16 x 16 transpose
constexpr int kMinCtas = 8;               // CTAs per SM the register cap allows

struct FftSmem {
  union {
    float2 buf[kLines][kBufPitch];        // the lines (staging, input and output)
    float2 T[kLines][16][kTPitch];        // the 16 x 16 transposes between the stages
  } u;
  float2 tw[16][16];                      // tw[k1][r] = W256^(r k1)
};
static_assert(sizeof(FftSmem) <= 48 * 1024, "static shared-memory launch");

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 conj_if(float2 w, bool c) { return c ? make_float2(w.x, -w.y) : w; }

// a * i^q, branch-free (q mod 4)
__device__ __forceinline__ float2 mul_ipow(float2 a, int q) {
  float2 v = (q & 1) ? make_float2(-a.y, a.x) : a;
  return (q & 2) ? make_float2(-v.x, -v.y) : v;
}

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
  a = cmul(a, conj_if(w16<K>(), INV));
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

// 256-point DFT of the kLines lines staged in s.u.buf, in place.  Thread
// (line, r): r = n2 in the first stage, r = k1 in the second.  NIN = number
// of leading inputs that can be non-zero (128 for the zero-padded forward).
template <bool INV, int NIN>
__device__ __forceinline__ void line_dft256(FftSmem& s, int line, int r) {
  float2 x[16];
#pragma unroll
  for (int n1 = 0; n1 < 16; ++n1) x[n1] = (16 * n1 < NIN) ? s.u.buf[line][16 * n1 + r] : make_float2(0.f, 0.f);
  dft16<INV>(x);
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) x[perm16(k1)] = cmul(x[perm16(k1)], conj_if(s.tw[k1][r], INV));
  __syncthreads();  // every line read before the transpose overwrites it
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) s.u.T[line][k1][r] = x[perm16(k1)];
  __syncthreads();
#pragma unroll
  for (int n2 = 0; n2 < 16; ++n2) x[n2] = s.u.T[line][r][n2];
  dft16<INV>(x);
  __syncthreads();  // every transpose read before the lines are written back
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) s.u.buf[line][r + 16 * k2] = x[perm16(k2)];
  __syncthreads();
}

__device__ __forceinline__ void load_twiddles(FftSmem& s, const float2* tw) {
  for (int j = threadIdx.x; j < kLen; j += blockDim.x) (&s.tw[0][0])[j] = tw[j];
}

// Pass A (forward): rows (i0, i1) of f times the correction, DFT along dim 2,
// post-phase i^l, into the grid rows (i0, i1, :).
__global__ void __launch_bounds__(kThreads, kMinCtas)
    fwd_rows_kernel(const float2* __restrict__ f, const float* __restrict__ beta0, const float* __restrict__ beta1,
                    const float* __restrict__ beta2, const float2* __restrict__ tw, float2* __restrict__ grid) {
  __shared__ FftSmem s;
  const int t = threadIdx.x;
  const int row0 = blockIdx.x * kLines;
  float2 v[kLines];
#pragma unroll
  for (int line = 0; line < kLines; ++line) v[line] = f[(int64_t)(row0 + line) * kHalf + t];
  load_twiddles(s, tw);
  const float b2 = beta2[t];
#pragma unroll
  for (int line = 0; line < kLines; ++line) {
    const int row = row0 + line, i0 = row / kHalf, i1 = row - i0 * kHalf;
    const float b = beta0[i0] * beta1[i1] * b2;
    s.u.buf[line][t] = make_float2(v[line].x * b, v[line].y * b);
  }
  __syncthreads();
  line_dft256<false, kHalf>(s, t >> 4, t & 15);
#pragma unroll
  for (int line = 0; line < kLines; ++line) {
    const int row = row0 + line, i0 = row / kHalf, i1 = row - i0 * kHalf;
    float2* dst = grid + ((int64_t)i0 * kLen + i1) * kLen;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int l = t + h * kThreads;
      dst[l] = mul_ipow(s.u.buf[line][l], l);
    }
  }
}

// Passes B and C (forward): kLines adjacent columns (element stride S, first
// element at base + j) read N inputs, write N~ outputs in place with the
// post-phase i^l.  Passes C' and B' (adjoint): read N~ inputs with the
// pre-phase (-i)^l, write the N outputs of the inverse DFT in place.
template <bool INV>
__global__ void __launch_bounds__(kThreads, kMinCtas)
    cols_kernel(float2* __restrict__ grid, int64_t outer_stride, int64_t S, const float2* __restrict__ tw) {
  __shared__ FftSmem s;
  constexpr int NIN = INV ? kLen : kHalf;
  constexpr int NOUT = INV ? kHalf : kLen;
  const int t = threadIdx.x;
  constexpr int blocks_per_outer = kLen / kLines;
  const int outer = blockIdx.x / blocks_per_outer;
  const int jb = (blockIdx.x - outer * blocks_per_outer) * kLines;
  float2* base = grid + outer * outer_stride + jb;
  const int j = t % kLines, n0 = t / kLines;
  float2 v[NIN / kSweep];
#pragma unroll
  for (int i = 0; i < NIN / kSweep; ++i) v[i] = base[(n0 + kSweep * i) * S + j];
  load_twiddles(s, tw);
#pragma unroll
  for (int i = 0; i < NIN / kSweep; ++i) {
    const int n = n0 + kSweep * i;
    s.u.buf[j][n] = INV ? mul_ipow(v[i], 3 * n) : v[i];  // (-i)^n = i^(3n)
  }
  __syncthreads();
  line_dft256<INV, NIN>(s, t >> 4, t & 15);
#pragma unroll
  for (int i = 0; i < NOUT / kSweep; ++i) {
    const int n = n0 + kSweep * i;
    const float2 o = s.u.buf[j][n];
    base[n * S + j] = INV ? o : mul_ipow(o, n);
  }
}

// Pass A' (adjoint): rows (i0, i1) of the grid, pre-phase, inverse DFT along
// dim 2, the N outputs times the correction into y.
__global__ void __launch_bounds__(kThreads, kMinCtas)
    adj_rows_kernel(const float2* __restrict__ grid, const float* __restrict__ beta0, const float* __restrict__ beta1,
                    const float* __restrict__ beta2, const float2* __restrict__ tw, float2* __restrict__ y) {
  __shared__ FftSmem s;
  const int t = threadIdx.x;
  const int row0 = blockIdx.x * kLines;
  float2 v[2 * kLines];
#pragma unroll
  for (int line = 0; line < kLines; ++line) {
    const int row = row0 + line, i0 = row / kHalf, i1 = row - i0 * kHalf;
    const float2* src = grid + ((int64_t)i0 * kLen + i1) * kLen;
    v[2 * line] = src[t];
    v[2 * line + 1] = src[t + kThreads];
  }
  load_twiddles(s, tw);
#pragma unroll
  for (int line = 0; line < kLines; ++line) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int l = t + h * kThreads;
      s.u.buf[line][l] = mul_ipow(v[2 * line + h], 3 * l);
    }
  }
  __syncthreads();
  line_dft256<true, kLen>(s, t >> 4, t & 15);
  const float b2 = beta2[t];
#pragma unroll
  for (int line = 0; line < kLines; ++line) {
    const int row = row0 + line, i0 = row / kHalf, i1 = row - i0 * kHalf;
    const float b = beta0[i0] * beta1[i1] * b2;
    const float2 o = s.u.buf[line][t];
    y[(int64_t)row * kHalf + t] = make_float2(o.x * b, o.y * b);
  }
}

// tw[16 k1 + r] = exp(-2 pi i r k1/256), in FP64 then rounded
__global__ void build_twiddles_kernel(float2* tw) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < kLen) {
    const int k1 = j >> 4, r = j & 15;
    const double a = 2.0 * M_PI * (double)(r * k1) / (double)kLen;
    tw[j] = make_float2((float)cos(a), (float)-sin(a));
  }
}

}  // namespace

bool pruned_fft_supported(int D, const int* N, const int* Nt) {
  if (D != 3) return false;
  for (int d = 0; d < 3; ++d)
    if (N[d] != kHalf || Nt[d] != kLen) return false;
  return true;
}

cudaError_t build_fft_twiddles(float2* tw, cudaStream_t s) {
  build_twiddles_kernel<<<1, kLen, 0, s>>>(tw);
  return cudaGetLastError();
}

cudaError_t launch_pruned_forward(const void* f, const float* const* beta, const float2* tw, void* grid,
                                  cudaStream_t s) {
  float2* g = (float2*)grid;
  fwd_rows_kernel<<<kHalf * kHalf / kLines, kThreads, 0, s>>>((const float2*)f, beta[0], beta[1], beta[2], tw, g);
  // B: lines (i0 < N, l2), element stride N~ (dim 1)
  cols_kernel<false><<<kHalf * (kLen / kLines), kThreads, 0, s>>>(g, (int64_t)kLen * kLen, kLen, tw);
  // C: lines (l1, l2), element stride N~^2 (dim 0)
  cols_kernel<false><<<kLen * (kLen / kLines), kThreads, 0, s>>>(g, kLen, (int64_t)kLen * kLen, tw);
  return cudaGetLastError();
}

cudaError_t launch_pruned_adjoint(void* grid, const float* const* beta, const float2* tw, void* y, cudaStream_t s) {
  float2* g = (float2*)grid;
  // C': lines (l1, l2) along dim 0, keep i0 < N
  cols_kernel<true><<<kLen * (kLen / kLines), kThreads, 0, s>>>(g, kLen, (int64_t)kLen * kLen, tw);
  // B': lines (i0 < N, l2) along dim 1, keep i1 < N
  cols_kernel<true><<<kHalf * (kLen / kLines), kThreads, 0, s>>>(g, (int64_t)kLen * kLen, kLen, tw);
  adj_rows_kernel<<<kHalf * kHalf / kLines, kThreads, 0, s>>>(g, beta[0], beta[1], beta[2], tw, (float2*)y);
  return cudaGetLastError();
}

}  // namespace nfftgb
