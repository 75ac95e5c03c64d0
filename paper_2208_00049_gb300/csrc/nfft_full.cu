// FULL precomputation: the resampling as the sparse matrix B of Eq. Bmatrix.
//
// Sec. 3.7.4 (item 2, "full precomputation") stores every window value and
// applies the resampling as a sparse matrix-vector product; Sec. 6 describes
// the paper's GPU prototype (CuNFFT.jl) as exactly this, with B uploaded to
// the GPU.  This file builds B on the device with the plan's window (one row
// per node in the caller's order, (2m)^D entries per row in ascending column
// order) and applies B and B^T with cuSPARSE SpMM, treating the complex grid
// and fhat as real matrices with two columns (re, im).  It is the library
// comparison form for the tiled kernels; it moves (2m)^D (value + index)
// per node, far more than the grid itself (Table 1: (2m)^D J values).
#include <cusparse.h>

#include "nfft_internal.cuh"

namespace nfftgb {

struct FullMatrix {
  int64_t rows = 0, cols = 0, nnz = 0;
  int dtype = NFFT_C64;
  int* rowptr = nullptr;
  int* col = nullptr;
  void* val = nullptr;
  int* rowptrT = nullptr;
  int* colT = nullptr;
  void* valT = nullptr;
  cusparseHandle_t h = nullptr;
  void* buf_fwd = nullptr;
  void* buf_adj = nullptr;
  size_t buf_fwd_bytes = 0, buf_adj_bytes = 0;
};

namespace {

template <int D, int K, typename R>
__global__ void build_rows_kernel(Geometry g, NodeArrays na, int* __restrict__ col, R* __restrict__ val) {
  const R* __restrict__ frac = reinterpret_cast<const R*>(na.frac);
  const int64_t M = g.M;
  const int mi = (int)g.m;
  constexpr int nnz_row = D == 1 ? K : (D == 2 ? K * K : K * K * K);
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < g.M; q += gridDim.x * blockDim.x) {
    int pos[D][K];
    R w[D][K];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const R t = frac[d * M + q];
      const int c = na.cell[d * M + q];
      // taps i = 0..K-1 at l' = c + off + i, listed in ascending position
      // order: the wrapped ones (l' >= N~) first.
      int first = 0;
#pragma unroll
      for (int i = 0; i < K; ++i)
        if (c + g.off + i >= g.Nt[d]) {
          first = i;
          break;
        }
      int nwrap_hi = 0;
#pragma unroll
      for (int i = 0; i < K; ++i) nwrap_hi += (c + g.off + i >= g.Nt[d]) ? 1 : 0;
      const R b = R(g.b[d]), norm = R(g.norm[d]), mr = R(mi);
      const R normx = sizeof(R) == 4 ? kb_normx<R>(b, mr) : R(0);
#pragma unroll
      for (int s = 0; s < K; ++s) {
        // ascending order: taps with l' < 0 wrap to the top, l' >= N~ to the bottom
        int i;
        if (nwrap_hi > 0) {
          i = (first + s) % K;
        } else {
          int nneg = 0;
#pragma unroll
          for (int r = 0; r < K; ++r) nneg += (c + g.off + r < 0) ? 1 : 0;
          i = (s + nneg) % K;
        }
        int l = c + g.off + i;
        l = l < 0 ? l + g.Nt[d] : (l >= g.Nt[d] ? l - g.Nt[d] : l);
        const R u = R(-g.off - i) + t;
        const R mm_u = R(mi + g.off + i) - t;
        const R mp_u = R(mi - g.off - i) + t;
        R v = kb_window<R>(u, mm_u, mp_u, b, norm, mr, normx);
        if (g.closed && ((i == 0 && t != R(0)) || i == K - 1)) v = R(0);
        pos[d][s] = l;
        w[d][s] = v;
      }
    }
    const int64_t row = na.perm[q];
    int* cr = col + row * nnz_row;
    R* vr = val + row * nnz_row;
    int e = 0;
    if constexpr (D == 1) {
#pragma unroll
      for (int i = 0; i < K; ++i, ++e) {
        cr[e] = pos[0][i];
        vr[e] = w[0][i];
      }
    } else if constexpr (D == 2) {
#pragma unroll
      for (int i0 = 0; i0 < K; ++i0)
#pragma unroll
        for (int i1 = 0; i1 < K; ++i1, ++e) {
          cr[e] = pos[0][i0] * g.Nt[1] + pos[1][i1];
          vr[e] = w[0][i0] * w[1][i1];
        }
    } else {
#pragma unroll 1
      for (int i0 = 0; i0 < K; ++i0) {
        int p0 = 0;
        R w0 = 0;
#pragma unroll
        for (int i = 0; i < K; ++i) {
          p0 = (i == i0) ? pos[0][i] : p0;
          w0 = (i == i0) ? w[0][i] : w0;
        }
#pragma unroll
        for (int i1 = 0; i1 < K; ++i1)
#pragma unroll
          for (int i2 = 0; i2 < K; ++i2, ++e) {
            cr[(int64_t)i0 * K * K + i1 * K + i2] = (p0 * g.Nt[1] + pos[1][i1]) * g.Nt[2] + pos[2][i2];
            vr[(int64_t)i0 * K * K + i1 * K + i2] = w0 * w[1][i1] * w[2][i2];
          }
      }
    }
  }
}

__global__ void rowptr_kernel(int* rowptr, int64_t rows, int per_row) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= rows; i += (int64_t)gridDim.x * blockDim.x)
    rowptr[i] = (int)(i * per_row);
}

template <typename R>
cudaError_t launch_build_rows(const Geometry& g, const NodeArrays& na, int* col, void* val, cudaStream_t s) {
  const int blocks = (g.M + 127) / 128 > 0 ? (g.M + 127) / 128 : 1;
#define NFFTGB_ROWS(DD, KK)                                                                  \
  if (g.D == DD && g.K == KK) {                                                             \
    build_rows_kernel<DD, KK, R><<<blocks, 128, 0, s>>>(g, na, col, (R*)val);              \
    return cudaGetLastError();                                                              \
  }
  NFFTGB_ROWS(1, 2) NFFTGB_ROWS(1, 4) NFFTGB_ROWS(1, 6) NFFTGB_ROWS(1, 8) NFFTGB_ROWS(1, 10)
  NFFTGB_ROWS(1, 12) NFFTGB_ROWS(1, 14) NFFTGB_ROWS(1, 16) NFFTGB_ROWS(1, 18)
  NFFTGB_ROWS(2, 2) NFFTGB_ROWS(2, 4) NFFTGB_ROWS(2, 6) NFFTGB_ROWS(2, 8) NFFTGB_ROWS(2, 10)
  NFFTGB_ROWS(2, 12) NFFTGB_ROWS(2, 14) NFFTGB_ROWS(2, 16) NFFTGB_ROWS(2, 18)
  NFFTGB_ROWS(3, 2) NFFTGB_ROWS(3, 4) NFFTGB_ROWS(3, 6) NFFTGB_ROWS(3, 8) NFFTGB_ROWS(3, 10)
  NFFTGB_ROWS(3, 12)
#undef NFFTGB_ROWS
  return cudaErrorInvalidValue;
}

int cs(cusparseStatus_t st) { return st == CUSPARSE_STATUS_SUCCESS ? NFFT_OK : NFFT_ERR_CUDA; }

cudaDataType dtype_of(int dtype) { return dtype == NFFT_C128 ? CUDA_R_64F : CUDA_R_32F; }

// y (rows x 2) = op(A) x, A = CSR (rows x cols), x, y row-major with 2 columns
int spmm(FullMatrix* F, bool transposed, const void* x, void* y, cudaStream_t s, void** buf, size_t* buf_bytes) {
  const int64_t r = transposed ? F->cols : F->rows, c = transposed ? F->rows : F->cols;
  int* rp = transposed ? F->rowptrT : F->rowptr;
  int* ci = transposed ? F->colT : F->col;
  void* va = transposed ? F->valT : F->val;
  const cudaDataType dt = dtype_of(F->dtype);
  cusparseSpMatDescr_t A = nullptr;
  cusparseDnMatDescr_t X = nullptr, Y = nullptr;
  int st = cs(cusparseCreateCsr(&A, r, c, F->nnz, rp, ci, va, CUSPARSE_INDEX_32I, CUSPARSE_INDEX_32I,
                                CUSPARSE_INDEX_BASE_ZERO, dt));
  if (st == NFFT_OK) st = cs(cusparseCreateDnMat(&X, c, 2, 2, const_cast<void*>(x), dt, CUSPARSE_ORDER_ROW));
  if (st == NFFT_OK) st = cs(cusparseCreateDnMat(&Y, r, 2, 2, y, dt, CUSPARSE_ORDER_ROW));
  double one64 = 1.0, zero64 = 0.0;
  float one32 = 1.f, zero32 = 0.f;
  const void* alpha = F->dtype == NFFT_C128 ? (const void*)&one64 : (const void*)&one32;
  const void* beta = F->dtype == NFFT_C128 ? (const void*)&zero64 : (const void*)&zero32;
  if (st == NFFT_OK) st = cs(cusparseSetStream(F->h, s));
  size_t need = 0;
  if (st == NFFT_OK)
    st = cs(cusparseSpMM_bufferSize(F->h, CUSPARSE_OPERATION_NON_TRANSPOSE, CUSPARSE_OPERATION_NON_TRANSPOSE, alpha,
                                    A, X, beta, Y, dt, CUSPARSE_SPMM_CSR_ALG2, &need));
  if (st == NFFT_OK && need > *buf_bytes) {
    if (*buf) cudaFree(*buf);
    *buf = nullptr;
    *buf_bytes = 0;
    if (cudaMalloc(buf, need) != cudaSuccess) {
      cudaGetLastError();
      st = NFFT_ERR_OOM;
    } else {
      *buf_bytes = need;
    }
  }
  if (st == NFFT_OK)
    st = cs(cusparseSpMM(F->h, CUSPARSE_OPERATION_NON_TRANSPOSE, CUSPARSE_OPERATION_NON_TRANSPOSE, alpha, A, X, beta,
                         Y, dt, CUSPARSE_SPMM_CSR_ALG2, *buf));
  if (A) cusparseDestroySpMat(A);
  if (X) cusparseDestroyDnMat(X);
  if (Y) cusparseDestroyDnMat(Y);
  return st;
}

}  // namespace

void full_destroy(FullMatrix* F) {
  if (!F) return;
  void* bufs[] = {F->rowptr, F->col, F->val, F->rowptrT, F->colT, F->valT, F->buf_fwd, F->buf_adj};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (F->h) cusparseDestroy(F->h);
  delete F;
}

// Build B (rows = nodes in caller order) and B^T from the plan's sorted nodes.
int full_build(FullMatrix** out, const Geometry& g, int dtype, const NodeArrays& na, cudaStream_t s) {
  full_destroy(*out);
  *out = nullptr;
  int64_t per_row = 1, cols = 1;
  for (int d = 0; d < g.D; ++d) {
    per_row *= g.K;
    cols *= g.Nt[d];
  }
  const int64_t nnz = per_row * g.M;
  if (nnz >= ((int64_t)1 << 31) || cols >= ((int64_t)1 << 31)) return NFFT_ERR_UNSUPPORTED;
  if (g.D == 3 && g.K > 12) return NFFT_ERR_UNSUPPORTED;  // rows of 14^3+ entries: not instantiated
  FullMatrix* F = new FullMatrix();
  F->rows = g.M;
  F->cols = cols;
  F->nnz = nnz;
  F->dtype = dtype;
  const size_t rs = dtype == NFFT_C128 ? 8 : 4;
  int st = NFFT_OK;
  auto alloc = [&](void** p, size_t bytes) {
    if (st != NFFT_OK) return;
    if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) {
      cudaGetLastError();
      *p = nullptr;
      st = NFFT_ERR_OOM;
    }
  };
  alloc((void**)&F->rowptr, sizeof(int) * (g.M + 1));
  alloc((void**)&F->col, sizeof(int) * nnz);
  alloc(&F->val, rs * nnz);
  alloc((void**)&F->rowptrT, sizeof(int) * (cols + 1));
  alloc((void**)&F->colT, sizeof(int) * nnz);
  alloc(&F->valT, rs * nnz);
  if (st == NFFT_OK) st = cs(cusparseCreate(&F->h));
  if (st == NFFT_OK) st = cs(cusparseSetStream(F->h, s));
  if (st == NFFT_OK) {
    rowptr_kernel<<<256, 256, 0, s>>>(F->rowptr, g.M, (int)per_row);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && g.M > 0)
      e = dtype == NFFT_C128 ? launch_build_rows<double>(g, na, F->col, F->val, s)
                             : launch_build_rows<float>(g, na, F->col, F->val, s);
    if (e != cudaSuccess) st = NFFT_ERR_CUDA;
  }
  if (st == NFFT_OK) {  // B^T = CSC of B
    size_t need = 0;
    const cudaDataType dt = dtype_of(dtype);
    st = cs(cusparseCsr2cscEx2_bufferSize(F->h, g.M, cols, nnz, F->val, F->rowptr, F->col, F->valT, F->rowptrT,
                                          F->colT, dt, CUSPARSE_ACTION_NUMERIC, CUSPARSE_INDEX_BASE_ZERO,
                                          CUSPARSE_CSR2CSC_ALG1, &need));
    void* buf = nullptr;
    alloc(&buf, need);
    if (st == NFFT_OK)
      st = cs(cusparseCsr2cscEx2(F->h, g.M, cols, nnz, F->val, F->rowptr, F->col, F->valT, F->rowptrT, F->colT, dt,
                                 CUSPARSE_ACTION_NUMERIC, CUSPARSE_INDEX_BASE_ZERO, CUSPARSE_CSR2CSC_ALG1, buf));
    if (buf) {
      cudaStreamSynchronize(s);
      cudaFree(buf);
    }
  }
  if (st != NFFT_OK) {
    full_destroy(F);
    return st;
  }
  *out = F;
  return NFFT_OK;
}

int full_forward(FullMatrix* F, const void* grid, void* fhat, cudaStream_t s) {
  if (F->rows == 0) return NFFT_OK;
  return spmm(F, false, grid, fhat, s, &F->buf_fwd, &F->buf_fwd_bytes);
}

int full_adjoint(FullMatrix* F, const void* fhat, void* grid, cudaStream_t s) {
  if (F->rows == 0) {
    const size_t cs = F->dtype == NFFT_C128 ? 16 : 8;
    return cudaMemsetAsync(grid, 0, cs * F->cols, s) == cudaSuccess ? NFFT_OK : NFFT_ERR_CUDA;
  }
  return spmm(F, true, fhat, grid, s, &F->buf_adj, &F->buf_adj_bytes);
}

}  // namespace nfftgb
