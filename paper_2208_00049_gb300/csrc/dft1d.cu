// Small one-dimensional complex128 transforms: the correction + zero-pad +
// FFT steps of Algorithm 1 and the inverse FFT + crop + correction steps of
// Algorithm 2 (Sec. 3.5) evaluated as direct sums,
//
//   forward:  g^_l = sum_{n in I_N} f_n beta(n) e^{-2 pi i n l / N~},  l = 0 .. N~-1
//   adjoint:  y_n  = beta(n) sum_{l=0}^{N~-1} g^_l e^{+2 pi i n l / N~},  n in I_N
//
// (the zero-padded entries contribute nothing and the cropped outputs are
// never formed).  GB300's FP64 units are narrow: a library FFT of 512 points
// runs on one SM for about 20 us, while these sums cost N N~ complex
// multiply-adds spread over every SM.  Each CTA takes a block of outputs and
// a chunk of the sum, and adds its partial sums to the zeroed output with
// FP64 atomics.  Twiddles come from an FP64 table of the N~-th roots of unity
// indexed by (n l) mod N~, so no rounding accumulates along a sum.
#include <cuda_runtime.h>

#include "nfft_internal.cuh"

namespace nfftgb {
namespace {

constexpr int kDftThreads = 128;

__global__ void dft_twiddle_kernel(double2* tw, int Nt) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < Nt; k += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(2.0 * (double)k / (double)Nt, &s, &c);
    tw[k] = make_double2(c, -s);  // e^{-2 pi i k / N~}
  }
}

// One thread per output l of the CTA's block, summing inputs [i0, i1) of f.
__global__ void __launch_bounds__(kDftThreads)
    dft_forward_kernel(int N, int Nt, int chunk, const double2* __restrict__ f, const double* __restrict__ beta,
                       const double2* __restrict__ tw, double2* __restrict__ grid) {
  __shared__ double2 fb[kDftThreads];
  const int l = blockIdx.x * kDftThreads + threadIdx.x;
  const int i0 = blockIdx.y * chunk, i1 = min(N, i0 + chunk);
  double re = 0.0, im = 0.0;
  for (int base = i0; base < i1; base += kDftThreads) {
    const int cnt = min(kDftThreads, i1 - base);
    __syncthreads();
    if (threadIdx.x < cnt) {
      const double2 v = f[base + threadIdx.x];
      const double bb = beta[base + threadIdx.x];
      fb[threadIdx.x] = make_double2(v.x * bb, v.y * bb);
    }
    __syncthreads();
    if (l < Nt) {
      // k = (n l) mod N~ for n = base - N/2, then + l per step
      const long long n0 = (long long)(base - N / 2);
      int k = (int)(((n0 % Nt + Nt) % Nt) * (long long)l % Nt);
      for (int j = 0; j < cnt; ++j) {
        const double2 w = tw[k];
        const double2 a = fb[j];
        re = fma(a.x, w.x, fma(-a.y, w.y, re));
        im = fma(a.x, w.y, fma(a.y, w.x, im));
        k += l;
        if (k >= Nt) k -= Nt;
      }
    }
  }
  if (l < Nt) {
    atomicAdd(&grid[l].x, re);
    atomicAdd(&grid[l].y, im);
  }
}

// One thread per output n = i - N/2 of the CTA's block, summing grid entries
// [l0, l1).
__global__ void __launch_bounds__(kDftThreads)
    dft_adjoint_kernel(int N, int Nt, int chunk, const double2* __restrict__ grid, const double* __restrict__ beta,
                       const double2* __restrict__ tw, double2* __restrict__ y) {
  __shared__ double2 gs[kDftThreads];
  const int i = blockIdx.x * kDftThreads + threadIdx.x;
  const int l0 = blockIdx.y * chunk, l1 = min(Nt, l0 + chunk);
  const int nm = i < N ? (((i - N / 2) % Nt) + Nt) % Nt : 0;  // n mod N~
  double re = 0.0, im = 0.0;
  for (int base = l0; base < l1; base += kDftThreads) {
    const int cnt = min(kDftThreads, l1 - base);
    __syncthreads();
    if (threadIdx.x < cnt) gs[threadIdx.x] = grid[base + threadIdx.x];
    __syncthreads();
    if (i < N) {
      int k = (int)((long long)nm * base % Nt);
      for (int j = 0; j < cnt; ++j) {
        const double2 w = tw[k];  // conj(w) = e^{+2 pi i k / N~}
        const double2 a = gs[j];
        re = fma(a.x, w.x, fma(a.y, w.y, re));
        im = fma(a.y, w.x, fma(-a.x, w.y, im));
        k += nm;
        if (k >= Nt) k -= Nt;
      }
    }
  }
  if (i < N) {
    const double bb = beta[i];
    atomicAdd(&y[i].x, re * bb);
    atomicAdd(&y[i].y, im * bb);
  }
}

// Sum chunk so that the launch has about one CTA per SM (at least 16 terms a
// thread, at most the whole sum).
int dft_chunk(int n_out, int n_sum, int sms) {
  const int blocks = (n_out + kDftThreads - 1) / kDftThreads;
  int chunks = sms / blocks;
  if (chunks < 1) chunks = 1;
  int chunk = (n_sum + chunks - 1) / chunks;
  if (chunk < 16) chunk = 16;
  return chunk < n_sum ? chunk : n_sum;
}

}  // namespace

bool dft1d_supported(int D, int N, int Nt) {
  return D == 1 && Nt <= 4096 && (long long)N * Nt <= (1ll << 20);
}

cudaError_t launch_dft_twiddles(double2* tw, int Nt, cudaStream_t s) {
  dft_twiddle_kernel<<<(Nt + 255) / 256, 256, 0, s>>>(tw, Nt);
  return cudaGetLastError();
}

cudaError_t launch_dft1d_forward(int N, int Nt, const void* f, const double* beta, const double2* tw, void* grid,
                                 int sms, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(grid, 0, sizeof(double2) * (size_t)Nt, s);
  if (e != cudaSuccess) return e;
  const int chunk = dft_chunk(Nt, N, sms);
  const dim3 grd((Nt + kDftThreads - 1) / kDftThreads, (N + chunk - 1) / chunk);
  dft_forward_kernel<<<grd, kDftThreads, 0, s>>>(N, Nt, chunk, (const double2*)f, beta, tw, (double2*)grid);
  return cudaGetLastError();
}

cudaError_t launch_dft1d_adjoint(int N, int Nt, const void* grid, const double* beta, const double2* tw, void* y,
                                 int sms, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(y, 0, sizeof(double2) * (size_t)N, s);
  if (e != cudaSuccess) return e;
  const int chunk = dft_chunk(N, Nt, sms);
  const dim3 grd((N + kDftThreads - 1) / kDftThreads, (Nt + chunk - 1) / chunk);
  dft_adjoint_kernel<<<grd, kDftThreads, 0, s>>>(N, Nt, chunk, (const double2*)grid, beta, tw, (double2*)y);
  return cudaGetLastError();
}

}  // namespace nfftgb
