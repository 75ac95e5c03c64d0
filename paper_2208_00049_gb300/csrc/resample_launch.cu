// Launchers and occupancy queries for the resampling kernels.  The kernels
// themselves are instantiated per kind and precision in resample_*.cu.
#include "nfft_internal.cuh"

namespace nfftgb {

template <typename R>
void* pick_gather(int D, int K);
template <typename R>
void* pick_scatter(int D, int K, int compensated);
template <typename R>
void* pick_grad(int D, int K);
template <typename R>
void* pick_gather_batch(int D, int K);
template <typename R>
void* pick_scatter_batch(int D, int K);

template <typename R>
struct CplxL;
template <>
struct CplxL<float> {
  using type = float2;
};
template <>
struct CplxL<double> {
  using type = double2;
};

// kind: 0 gather, 1 scatter, 2 compensated scatter, 3 node-gradient gather
template <typename R>
static void* pick(const Geometry& g, int kind) {
  switch (kind) {
    case 0: return pick_gather<R>(g.D, g.K);
    case 1: return pick_scatter<R>(g.D, g.K, 0);
    case 2: return pick_scatter<R>(g.D, g.K, 1);
    case 3: return pick_grad<R>(g.D, g.K);
  }
  return nullptr;
}

template <typename R>
size_t resample_smem_bytes(const Geometry& g, int kind) {
  size_t region = 1;
  for (int d = 0; d < g.D; ++d) region *= (size_t)g.L[d];
  return region * 2 * sizeof(R) * (kind == 2 ? 2 : 1);
}

static cudaError_t prepare_smem(void* kern, size_t smem) {
  if (smem > 48 * 1024)
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaSuccess;
}

template <typename R>
int resample_ctas_per_sm(const Geometry& g, int kind) {
  void* k = pick<R>(g, kind);
  if (!k) return sizeof(R) == 8 && kind == 2 ? 1 : 0;  // no FP64 compensated variant
  size_t smem = resample_smem_bytes<R>(g, kind == 3 ? 0 : kind);
  if (prepare_smem(k, smem) != cudaSuccess) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kResampleThreads, smem) != cudaSuccess)
    return 0;
  return n;
}

template <typename R>
cudaError_t launch_gather(const Geometry& g, const void* grid, const NodeArrays& na, void* fhat,
                          int ctas, cudaStream_t s) {
  using C = typename CplxL<R>::type;
  void* k = pick<R>(g, 0);
  if (!k) return cudaErrorInvalidValue;
  size_t smem = resample_smem_bytes<R>(g, 0);
  cudaError_t e = prepare_smem(k, smem);
  if (e != cudaSuccess) return e;
  auto kern = reinterpret_cast<void (*)(Geometry, const C*, NodeArrays, C*)>(k);
  kern<<<ctas, kResampleThreads, smem, s>>>(g, (const C*)grid, na, (C*)fhat);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_scatter(const Geometry& g, void* grid, const NodeArrays& na, const void* fhat,
                           int compensated, int ctas, cudaStream_t s) {
  using C = typename CplxL<R>::type;
  const int kind = compensated ? 2 : 1;
  void* k = pick<R>(g, kind);
  if (!k) return cudaErrorInvalidValue;
  size_t smem = resample_smem_bytes<R>(g, kind);
  cudaError_t e = prepare_smem(k, smem);
  if (e != cudaSuccess) return e;
  auto kern = reinterpret_cast<void (*)(Geometry, C*, NodeArrays, const C*)>(k);
  kern<<<ctas, kResampleThreads, smem, s>>>(g, (C*)grid, na, (const C*)fhat);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_grad_gather(const Geometry& g, const void* grid, const NodeArrays& na,
                               const void* cot, void* gk, int ctas, cudaStream_t s) {
  using C = typename CplxL<R>::type;
  void* k = pick<R>(g, 3);
  if (!k) return cudaErrorInvalidValue;
  size_t smem = resample_smem_bytes<R>(g, 0);
  cudaError_t e = prepare_smem(k, smem);
  if (e != cudaSuccess) return e;
  auto kern = reinterpret_cast<void (*)(Geometry, const C*, NodeArrays, const C*, R*)>(k);
  kern<<<ctas, kResampleThreads, smem, s>>>(g, (const C*)grid, na, (const C*)cot, (R*)gk);
  return cudaGetLastError();
}

template <typename R>
int resample_batch_ctas_per_sm(const Geometry& gmax, int kind) {
  void* k = kind == 0 ? pick_gather_batch<R>(gmax.D, gmax.K) : pick_scatter_batch<R>(gmax.D, gmax.K);
  if (!k) return 0;
  size_t smem = resample_smem_bytes<R>(gmax, kind == 0 ? 0 : 1);
  if (prepare_smem(k, smem) != cudaSuccess) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kResampleThreads, smem) != cudaSuccess)
    return 0;
  return n;
}

// gmax: a geometry whose region L is the largest of the batch (sizes the
// shared-memory tile); the kernels read each problem's own geometry.
template <typename R>
cudaError_t launch_gather_batch(const BatchProblem* probs, const Geometry& gmax, const void* grid,
                                const BatchNodes& nb, void* fhat, int ctas, cudaStream_t s) {
  using C = typename CplxL<R>::type;
  void* k = pick_gather_batch<R>(gmax.D, gmax.K);
  if (!k) return cudaErrorInvalidValue;
  size_t smem = resample_smem_bytes<R>(gmax, 0);
  cudaError_t e = prepare_smem(k, smem);
  if (e != cudaSuccess) return e;
  auto kern = reinterpret_cast<void (*)(const BatchProblem*, const C*, BatchNodes, C*)>(k);
  kern<<<ctas, kResampleThreads, smem, s>>>(probs, (const C*)grid, nb, (C*)fhat);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_scatter_batch(const BatchProblem* probs, const Geometry& gmax, void* grid,
                                 const BatchNodes& nb, const void* fhat, int ctas, cudaStream_t s) {
  using C = typename CplxL<R>::type;
  void* k = pick_scatter_batch<R>(gmax.D, gmax.K);
  if (!k) return cudaErrorInvalidValue;
  size_t smem = resample_smem_bytes<R>(gmax, 1);
  cudaError_t e = prepare_smem(k, smem);
  if (e != cudaSuccess) return e;
  auto kern = reinterpret_cast<void (*)(const BatchProblem*, C*, BatchNodes, const C*)>(k);
  kern<<<ctas, kResampleThreads, smem, s>>>(probs, (C*)grid, nb, (const C*)fhat);
  return cudaGetLastError();
}

#define NFFTGB_INSTANTIATE_LAUNCH(R)                                                             \
  template size_t resample_smem_bytes<R>(const Geometry&, int);                                 \
  template int resample_ctas_per_sm<R>(const Geometry&, int);                                   \
  template cudaError_t launch_gather<R>(const Geometry&, const void*, const NodeArrays&, void*, \
                                        int, cudaStream_t);                                     \
  template cudaError_t launch_scatter<R>(const Geometry&, void*, const NodeArrays&, const void*,\
                                         int, int, cudaStream_t);                               \
  template cudaError_t launch_grad_gather<R>(const Geometry&, const void*, const NodeArrays&,   \
                                             const void*, void*, int, cudaStream_t);            \
  template int resample_batch_ctas_per_sm<R>(const Geometry&, int);                             \
  template cudaError_t launch_gather_batch<R>(const BatchProblem*, const Geometry&, const void*, \
                                              const BatchNodes&, void*, int, cudaStream_t);     \
  template cudaError_t launch_scatter_batch<R>(const BatchProblem*, const Geometry&, void*,      \
                                               const BatchNodes&, const void*, int, cudaStream_t);
NFFTGB_INSTANTIATE_LAUNCH(float)
NFFTGB_INSTANTIATE_LAUNCH(double)

}  // namespace nfftgb
