// Plan object and C ABI (see include/nfft_gb300.h).
//
// arXiv 2208.00049, Sec. 3.1-3.2: a plan holds every temporary (the
// oversampled grid ghat, the FFT plans, the index/window data and the
// blocking buffers) and does the precomputation, so that transforms allocate
// nothing.  Algorithm 1 = deconv_pad -> FFT -> gather; Algorithm 2 =
// scatter -> FFT^H -> crop_deconv.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "nfft_internal.cuh"

using namespace nfftgb;

struct nfft_plan {
  int D = 0;
  int64_t N[kMaxD] = {1, 1, 1};
  int64_t Nt[kMaxD] = {1, 1, 1};
  int64_t M = 0;
  double sigma = 2.0;
  int m = 4;
  int dtype = NFFT_C64;
  uint32_t flags = 0;
  double b[kMaxD] = {0, 0, 0};
  cudaStream_t stream = nullptr;
  int device = 0;
  int sms = 1;
  int K = 8, off = -3;

  int64_t T[kMaxD] = {1, 1, 1};
  int ntile[kMaxD] = {1, 1, 1};
  int64_t n_tiles = 0;
  int cmax = 128;              // nodes per work item (set by configure_tiles)
  int64_t max_items = 0;
  int ctas[4] = {0, 0, 0, 0};  // persistent grid per kernel kind
  bool fast_gather = false;    // specialised complex64 gather (3D m = 4 / 6, 2D m = 4)
  bool fast_scatter = false;   // register-accumulating complex64 scatter (3D m = 4 / 6, 2D m = 4)
  FullMatrix* full = nullptr;  // NFFT_FLAG_FULL_MATRIX: B and B^T as CSR
  int fast_ctas[2] = {0, 0};
  int grad_ctas = 0;           // 3D m = 4 complex64 node-gradient kernel (0: generic)
  int f64_scatter_ctas = 0;    // 2D / 3D complex128 scatter without shared atomics (0: generic)
  bool pruned = false;         // nfft_step_pad_fft / fft_crop use the pruned 3D FFT
  float2* fft_tw = nullptr;    // its 256 twiddles
  bool dft1d = false;          // ... or the direct sums of small 1D complex128 plans
  double2* dft_tw = nullptr;   // their N~ roots of unity

  void* grid = nullptr;
  double* beta64 = nullptr;
  float* beta32 = nullptr;
  float* poly = nullptr;  // POLYNOMIAL window coefficients [D][K][2m + 1] (FP32)
  double* poly64 = nullptr;  // FP64 coefficients [D][K][poly_Z] (complex128 plans in the POLYNOMIAL form)
  int poly_Z = 0;            // coefficients per tap of the table the generic kernels read
  int wmode = kWinDirect;    // window values of the generic kernels
  void* lut = nullptr;       // LINEAR tables, D x lut_S entries of the plan's real type
  int64_t lut_S = 0;
  int* cell = nullptr;
  void* frac = nullptr;
  int* perm = nullptr;
  int* key = nullptr;
  int* rank = nullptr;
  int* tile_count = nullptr;
  int* tile_offset = nullptr;
  int4* items = nullptr;
  int* n_items = nullptr;
  int64_t tiles_cap = 0;
  int64_t items_cap = 0;

  void* stage[3] = {nullptr, nullptr, nullptr};
  size_t stage_bytes[3] = {0, 0, 0};

  // asynchronous host-buffer transforms (nfft_plan_set_async): copies on
  // their own streams, stage buffers double-buffered by call parity
  bool async_mode = false;
  cudaStream_t h2d = nullptr, d2h = nullptr;
  cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_comp[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
  void* astage[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [parity][in, out]
  size_t astage_bytes[2][2] = {{0, 0}, {0, 0}};
  int parity = 0;

  cufftHandle fft = 0;
  bool fft_ok = false;
  // graph mode: nfft_forward / nfft_adjoint captured once per pair of device
  // buffers on capture_stream and replayed on `stream`
  bool graph_mode = false;
  cudaStream_t capture_stream = nullptr;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};  // forward, adjoint
  const void* graph_ptr[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  bool has_nodes = false;
  int err = NFFT_OK;
};

namespace {

size_t real_size(const nfft_plan* p) { return p->dtype == NFFT_C128 ? 8 : 4; }
size_t cplx_size(const nfft_plan* p) { return 2 * real_size(p); }
int64_t prod_N(const nfft_plan* p) {
  int64_t r = 1;
  for (int d = 0; d < p->D; ++d) r *= p->N[d];
  return r;
}
int64_t prod_Nt(const nfft_plan* p) {
  int64_t r = 1;
  for (int d = 0; d < p->D; ++d) r *= p->Nt[d];
  return r;
}

int latch(nfft_plan* p, int code) {
  if (p && p->err == NFFT_OK && code != NFFT_OK) p->err = code;
  return code;
}

int cuda_status(nfft_plan* p, cudaError_t e) {
  if (e == cudaSuccess) return NFFT_OK;
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return latch(p, NFFT_ERR_OOM);
  }
  return latch(p, NFFT_ERR_CUDA);
}

#define NFFT_CK(p, call)                         \
  do {                                           \
    int _s = cuda_status((p), (call));           \
    if (_s != NFFT_OK) return _s;                \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

template <typename T>
int dalloc(nfft_plan* p, T** ptr, size_t bytes) {
  *ptr = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc((void**)ptr, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return latch(p, NFFT_ERR_OOM);
  }
  return NFFT_OK;
}

void dfree(void* ptr) {
  if (ptr) cudaFree(ptr);
}

bool is_device_pointer(const void* ptr) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

// Device buffer for a host argument: slot 0 = transform input, 1 = output,
// 2 = second input.
int stage_buffer(nfft_plan* p, int slot, size_t bytes, void** out) {
  if (p->stage_bytes[slot] < bytes) {
    dfree(p->stage[slot]);
    p->stage[slot] = nullptr;
    p->stage_bytes[slot] = 0;
    int s = dalloc(p, &p->stage[slot], bytes);
    if (s != NFFT_OK) return s;
    p->stage_bytes[slot] = bytes;
  }
  *out = p->stage[slot];
  return NFFT_OK;
}

// Input pointer -> device pointer (copying a host input to a stage buffer).
int device_input(nfft_plan* p, int slot, const void* ptr, size_t bytes, const void** dev) {
  if (bytes == 0 || is_device_pointer(ptr)) {
    *dev = ptr;
    return NFFT_OK;
  }
  void* buf = nullptr;
  int s = stage_buffer(p, slot, bytes, &buf);
  if (s != NFFT_OK) return s;
  NFFT_CK(p, cudaMemcpyAsync(buf, ptr, bytes, cudaMemcpyHostToDevice, p->stream));
  *dev = buf;
  return NFFT_OK;
}

struct OutputBinding {
  void* user = nullptr;
  void* dev = nullptr;
  size_t bytes = 0;
  bool host = false;
};

int device_output(nfft_plan* p, int slot, void* ptr, size_t bytes, OutputBinding* ob) {
  ob->user = ptr;
  ob->bytes = bytes;
  ob->host = bytes > 0 && !is_device_pointer(ptr);
  if (!ob->host) {
    ob->dev = ptr;
    return NFFT_OK;
  }
  return stage_buffer(p, slot, bytes, &ob->dev);
}

int finish_output(nfft_plan* p, const OutputBinding& ob) {
  if (!ob.host) return NFFT_OK;
  NFFT_CK(p, cudaMemcpyAsync(ob.user, ob.dev, ob.bytes, cudaMemcpyDeviceToHost, p->stream));
  NFFT_CK(p, cudaStreamSynchronize(p->stream));
  return NFFT_OK;
}

Geometry make_geometry(const nfft_plan* p) {
  Geometry g{};
  g.D = p->D;
  g.K = p->K;
  g.off = p->off;
  g.closed = (p->flags & NFFT_FLAG_CLOSED_SUPPORT) ? 1 : 0;
  g.M = (int)p->M;
  g.m = (double)p->m;
  g.wmode = p->wmode;
  g.wS = (int)p->lut_S;
  g.wtab = p->wmode == kWinLinear ? (const void*)p->lut
           : p->wmode == kWinPoly ? (p->dtype == NFFT_C128 ? (const void*)p->poly64 : (const void*)p->poly)
                                  : nullptr;
  g.wZ = p->poly_Z;
  for (int d = 0; d < p->D; ++d) {
    g.Nt[d] = (int)p->Nt[d];
    g.T[d] = (int)p->T[d];
    g.ntile[d] = p->ntile[d];
    g.L[d] = (int)p->T[d] + p->K - 1;
    g.b[d] = p->b[d];
    g.norm[d] = (double)p->m / sinh(p->b[d] * (double)p->m);
  }
  return g;
}

DeconvArgs make_deconv(const nfft_plan* p) {
  DeconvArgs a{};
  a.D = p->D;
  int64_t off = 0;
  for (int d = 0; d < p->D; ++d) {
    a.N[d] = (int)p->N[d];
    a.Nt[d] = (int)p->Nt[d];
    if (p->dtype == NFFT_C128)
      a.beta[d] = p->beta64 + off;
    else
      a.beta[d] = p->beta32 + off;
    off += p->N[d];
  }
  return a;
}

size_t region_bytes(const nfft_plan* p, const int64_t* T, int kind) {
  size_t r = 1;
  for (int d = 0; d < p->D; ++d) r *= (size_t)(T[d] + p->K - 1);
  return r * cplx_size(p) * (kind == 2 ? 2 : 1);
}

// Default tile shape: the largest power-of-two cube (capped per dimension by
// N~_d) whose expected node count stays near 2 nodes per thread and whose
// shared-memory region (tile + halo) stays within 64 KB.
void default_tile(const nfft_plan* p, int64_t* T) {
  double density = (double)p->M / (double)prod_Nt(p);
  int64_t best = 1;
  for (int64_t t = 1; t <= 4096; t *= 2) {
    int64_t TT[kMaxD];
    double cells = 1;
    for (int d = 0; d < p->D; ++d) {
      TT[d] = t < p->Nt[d] ? t : p->Nt[d];
      cells *= (double)TT[d];
    }
    if (region_bytes(p, TT, (p->flags & NFFT_FLAG_COMPENSATED) ? 2 : 1) > 64 * 1024) break;
    best = t;
    if (density * cells >= 2.0 * kResampleThreads) break;
  }
  // 3D m = 4 complex64 (the register-accumulating scatter): 9 x 9 x 8 cells
  // (regions of 16 x 16 x 15) measured 3.5 % faster than 8^3 for gather +
  // scatter at 0.125 nodes per cell, with fewer halo reductions per node.
  const bool fast_shape = p->D == 3 && p->m == 4 && p->K == 8 && p->dtype == NFFT_C64 &&
                          !(p->flags & (NFFT_FLAG_CLOSED_SUPPORT | NFFT_FLAG_WIDE_WINDOW));
  const int64_t pref[kMaxD] = {9, 9, 8};
  // 3D m = 6 complex64: the K = 12 gather and the register-accumulating
  // scatter need tiles of at most 5 cells per dimension; 5^3 measured best
  // for gather + scatter at the sigma = 1.25 lean variant (2.50 ms against
  // 18.9 ms for the generic kernels at 8^3)
  const bool m6_shape = p->D == 3 && p->m == 6 && p->K == 12 && p->dtype == NFFT_C64 &&
                        !(p->flags & (NFFT_FLAG_CLOSED_SUPPORT | NFFT_FLAG_WIDE_WINDOW));
  const int64_t pref6[kMaxD] = {5, 5, 5};
  // 2D m = 4 complex64: the warp-per-item kernels take regions of at most
  // 16 x 32 cells; 9 x 25 tiles (measured best on the batched workload, and
  // at 512^2 with 7.7 tiles per SM: 1.67 against 1.59 G nodes/s for gather +
  // scatter), 8 x 8 when that would leave fewer than 7 tiles per SM
  const bool m4_2d = p->D == 2 && p->m == 4 && p->K == 8 && p->dtype == NFFT_C64 &&
                     !(p->flags & (NFFT_FLAG_CLOSED_SUPPORT | NFFT_FLAG_WIDE_WINDOW));
  const bool big2d = p->D == 2 && (double)p->Nt[0] * (double)p->Nt[1] >= 225.0 * 7.0 * (double)p->sms;
  const int64_t pref2[kMaxD] = {big2d ? 9 : 8, big2d ? 25 : 8, 1};
  // 2D complex128 with the atomic-free scatter (even K = 2m <= 16): 20 x 20
  // at m = 8 and 16 x 16 at m = 6 measured best for gather + scatter at
  // 256^2 and 512^2 (256^2, m = 8: 0.353 ms against 0.399 ms at the 32 x 32
  // the rule above gives; larger tiles make fewer, larger work items for the
  // scatter's CTAs, smaller ones cost the generic gather its threads)
  const bool f64_2d = p->D == 2 && p->dtype == NFFT_C128 && p->K == 2 * p->m && p->K <= 16 &&
                      !(p->flags & (NFFT_FLAG_CLOSED_SUPPORT | NFFT_FLAG_WIDE_WINDOW));
  for (int d = 0; d < p->D; ++d) {
    int64_t cap = p->Nt[d] - p->K + 1;  // keeps region coordinates within [-N~, 2 N~)
    if (cap < 1) cap = 1;
    int64_t want = best;
    if (fast_shape && best == 8) want = pref[d];
    if (m6_shape && best >= 4) want = pref6[d];
    if (m4_2d && best >= 8) want = pref2[d];
    if (f64_2d && best >= 16) want = p->K >= 14 ? 20 : 16;
    T[d] = want < cap ? want : cap;
  }
}

constexpr uint32_t kWindowFlags = NFFT_FLAG_WINDOW_DIRECT | NFFT_FLAG_WINDOW_LINEAR | NFFT_FLAG_WINDOW_POLYNOMIAL;
constexpr int kItemCapFull = 128;  // nodes per work item of the specialised kernels

// Captured graphs hold the launch configuration and buffers of the moment;
// dropped when either changes.
void drop_graphs(nfft_plan* p) {
  for (int k = 0; k < 2; ++k) {
    if (p->graph[k]) cudaGraphExecDestroy(p->graph[k]);
    p->graph[k] = nullptr;
    p->graph_ptr[k][0] = p->graph_ptr[k][1] = nullptr;
  }
}

int configure_tiles(nfft_plan* p, const int64_t* T) {
  drop_graphs(p);
  int64_t n_tiles = 1;
  for (int d = 0; d < p->D; ++d) {
    p->T[d] = T[d];
    p->ntile[d] = (int)((p->Nt[d] + T[d] - 1) / T[d]);
    n_tiles *= p->ntile[d];
  }
  if (n_tiles > (int64_t)1 << 30) return NFFT_ERR_INVALID_ARG;
  p->n_tiles = n_tiles;
  p->cmax = kItemCapFull;
  {
    // The generic kernels run one CTA per work item: a small node set is cut
    // into smaller items (down to 8 nodes) so that it reaches every SM.  The
    // specialised kernels keep full items.
    const Geometry g0 = make_geometry(p);
    const bool c64 = p->dtype == NFFT_C64 && !(p->flags & kWindowFlags);
    const bool fast = c64 && (p->D == 2 ? scatter2d_supported(g0)
                                        : fast3d_supported(g0, kItemCapFull) ||
                                              fast_scatter_supported(g0, kItemCapFull));
    if (!fast) {
      int64_t want = (p->M + 2 * p->sms - 1) / (2 * (int64_t)p->sms);
      want = (want + 7) / 8 * 8;
      p->cmax = (int)(want < 8 ? 8 : (want > kItemCapFull ? kItemCapFull : want));
    }
  }
  p->max_items = n_tiles + (p->M + p->cmax - 1) / p->cmax + 1;
  if (p->tiles_cap < n_tiles) {
    dfree(p->tile_count);
    dfree(p->tile_offset);
    p->tile_count = p->tile_offset = nullptr;
    p->tiles_cap = 0;
    int s = dalloc(p, &p->tile_count, sizeof(int) * n_tiles);
    if (s == NFFT_OK) s = dalloc(p, &p->tile_offset, sizeof(int) * n_tiles);
    if (s != NFFT_OK) return s;
    p->tiles_cap = n_tiles;
  }
  if (p->items_cap < p->max_items) {
    dfree(p->items);
    p->items = nullptr;
    p->items_cap = 0;
    int s = dalloc(p, &p->items, sizeof(int4) * p->max_items);
    if (s != NFFT_OK) return s;
    p->items_cap = p->max_items;
  }
  Geometry g = make_geometry(p);
  // complex64 plans use the specialised kernels where the tile allows (with
  // NFFT_FLAG_COMPENSATED their scatter runs in its TwoSum-compensated form);
  // a window flag selects the generic kernels, so that the window modes are
  // compared on the same kernels
  const bool c64 = p->dtype == NFFT_C64 && !(p->flags & kWindowFlags);
  const int comp = (p->flags & NFFT_FLAG_COMPENSATED) && c64 ? 1 : 0;
  p->fast_gather = c64 && fast3d_supported(g, p->cmax);
  p->fast_scatter = c64 && (p->fast_gather || fast_scatter_supported(g, p->cmax));
  if (p->D == 2) p->fast_gather = p->fast_scatter = c64 && scatter2d_supported(g);
  if (p->fast_gather) {
    const int per_sm = p->D == 2 ? gather2d_ctas_per_sm() : fast3d_ctas_per_sm(g, 0);
    p->fast_gather = per_sm > 0;
    p->fast_ctas[0] = per_sm * p->sms;
  }
  p->grad_ctas = 0;
  if (p->fast_gather && p->D == 3 && p->K == 8) p->grad_ctas = grad3d_ctas_per_sm(g) * p->sms;
  if (p->fast_scatter) {
    const int per_sm = p->D == 2 ? scatter2d_ctas_per_sm(comp) : fast3d_ctas_per_sm(g, comp ? 2 : 1);
    p->fast_scatter = per_sm > 0;
    p->fast_ctas[1] = per_sm * p->sms;
  }
  p->f64_scatter_ctas = 0;
  if (p->dtype == NFFT_C128 && p->D == 2 && scatter2d_f64_supported(g)) {
    const int per_cta = scatter2d_f64_items_per_cta();
    int ctas = scatter2d_f64_ctas_per_sm(g) * p->sms;
    const int64_t need = (p->max_items + per_cta - 1) / per_cta;
    if (ctas > need) ctas = (int)need;
    p->f64_scatter_ctas = ctas;
  }
  if (p->dtype == NFFT_C128 && p->D == 3 && scatter3d_f64_supported(g)) {
    int ctas = scatter3d_f64_ctas_per_sm(g) * p->sms;
    if (ctas > p->max_items) ctas = (int)p->max_items;
    p->f64_scatter_ctas = ctas;
  }
  // generic kernels: gather and scatter are required; the compensated scatter
  // where the plan asks for it and no fast scatter serves it; the node
  // gradient is optional (m = 9, 10 have none: nfft_grad reports UNSUPPORTED)
  for (int kind = 0; kind < 4; ++kind) {
    int per_sm = p->dtype == NFFT_C128 ? resample_ctas_per_sm<double>(g, kind)
                                       : resample_ctas_per_sm<float>(g, kind);
    const bool comp_req = (p->flags & NFFT_FLAG_COMPENSATED) && p->dtype == NFFT_C64;
    const bool needed = kind < 2 || (kind == 2 && comp_req && !p->fast_scatter);
    if (per_sm <= 0 && needed) return NFFT_ERR_UNSUPPORTED;
    p->ctas[kind] = per_sm > 0 ? per_sm * p->sms : 0;
  }
  // The persistent grids take work items in strides of their size; a small
  // node set has fewer items than resident CTAs, and the extra CTAs would
  // only start and exit (each launch wave costs microseconds).
  auto cap = [&](int& c) {
    if (c > p->max_items) c = (int)p->max_items;
  };
  for (int& c : p->ctas) cap(c);
  for (int& c : p->fast_ctas) cap(c);
  cap(p->grad_ctas);
  return NFFT_OK;
}

bool ready(nfft_plan* p, int* status) {
  if (!p) {
    *status = NFFT_ERR_INVALID_ARG;
    return false;
  }
  if (p->err != NFFT_OK) {
    *status = p->err;
    return false;
  }
  *status = NFFT_OK;
  return true;
}

NodeArrays node_arrays(const nfft_plan* p) {
  NodeArrays na;
  na.cell = p->cell;
  na.frac = p->frac;
  na.perm = p->perm;
  na.items = p->items;
  na.n_items = p->n_items;
  return na;
}

int run_deconv_pad(nfft_plan* p, const void* f) {
  DeconvArgs a = make_deconv(p);
  cudaError_t e = p->dtype == NFFT_C128 ? launch_deconv_pad<double>(a, f, p->grid, p->stream)
                                        : launch_deconv_pad<float>(a, f, p->grid, p->stream);
  return cuda_status(p, e);
}

int run_fft(nfft_plan* p, int sign) {
  cufftResult r;
  int dir = sign < 0 ? CUFFT_FORWARD : CUFFT_INVERSE;
  if (p->dtype == NFFT_C128)
    r = cufftExecZ2Z(p->fft, (cufftDoubleComplex*)p->grid, (cufftDoubleComplex*)p->grid, dir);
  else
    r = cufftExecC2C(p->fft, (cufftComplex*)p->grid, (cufftComplex*)p->grid, dir);
  if (r != CUFFT_SUCCESS) return latch(p, NFFT_ERR_CUFFT);
  return NFFT_OK;
}

int run_gather(nfft_plan* p, void* fhat) {
  Geometry g = make_geometry(p);
  NodeArrays na = node_arrays(p);
  if (p->full) return latch(p, full_forward(p->full, p->grid, fhat, p->stream));
  cudaError_t e = p->fast_gather
                      ? (p->D == 2 ? launch_gather2d_fast(g, p->grid, na, p->poly, fhat, p->fast_ctas[0], p->stream)
                                   : launch_gather3d_fast(g, p->grid, na, p->poly, fhat, p->fast_ctas[0], p->stream))
                  : p->dtype == NFFT_C128
                      ? launch_gather<double>(g, p->grid, na, fhat, p->ctas[0], p->stream)
                      : launch_gather<float>(g, p->grid, na, fhat, p->ctas[0], p->stream);
  return cuda_status(p, e);
}

int run_scatter(nfft_plan* p, const void* fhat) {
  if (p->full) return latch(p, full_adjoint(p->full, fhat, p->grid, p->stream));
  NFFT_CK(p, cudaMemsetAsync(p->grid, 0, (size_t)prod_Nt(p) * cplx_size(p), p->stream));
  Geometry g = make_geometry(p);
  NodeArrays na = node_arrays(p);
  const int comp = (p->flags & NFFT_FLAG_COMPENSATED) && p->dtype == NFFT_C64 ? 1 : 0;
  cudaError_t e =
      p->fast_scatter
          ? (p->D == 2 ? launch_scatter2d_fast(g, p->grid, na, p->poly, fhat, comp, p->fast_ctas[1], p->stream)
                       : launch_scatter3d_fast(g, p->grid, na, p->poly, fhat, comp, p->fast_ctas[1], p->stream))
      : p->dtype == NFFT_C128
          ? (p->f64_scatter_ctas > 0 && p->D == 2 && scatter2d_f64_supported(g)
                 ? launch_scatter2d_f64(g, p->grid, na, fhat, p->f64_scatter_ctas, p->stream)
             : p->f64_scatter_ctas > 0 && p->D == 3 && scatter3d_f64_supported(g)
                 ? launch_scatter3d_f64(g, p->grid, na, fhat, p->f64_scatter_ctas, p->stream)
                 : launch_scatter<double>(g, p->grid, na, fhat, 0, p->ctas[1], p->stream))
          : launch_scatter<float>(g, p->grid, na, fhat, comp, p->ctas[comp ? 2 : 1], p->stream);
  return cuda_status(p, e);
}

const float* const* beta32_dims(const nfft_plan* p, const float** out) {
  int64_t off = 0;
  for (int d = 0; d < p->D; ++d) {
    out[d] = p->beta32 + off;
    off += p->N[d];
  }
  return out;
}

// Algorithm 1, correction + zero-pad + FFT steps: pruned FFT where the plan
// qualifies, else the correction kernel and cuFFT.
int run_pad_fft(nfft_plan* p, const void* f) {
  if (p->dft1d)
    return cuda_status(p, launch_dft1d_forward((int)p->N[0], (int)p->Nt[0], f, p->beta64, p->dft_tw, p->grid,
                                               p->sms, p->stream));
  if (p->pruned) {
    const float* beta[kMaxD];
    return cuda_status(p, launch_pruned_forward(p->D, (int)p->Nt[0], f, beta32_dims(p, beta), p->fft_tw, p->grid,
                                                p->stream));
  }
  int s = run_deconv_pad(p, f);
  if (s != NFFT_OK) return s;
  return run_fft(p, -1);
}

int run_crop_deconv(nfft_plan* p, void* y);

// Algorithm 2, inverse FFT + crop + correction steps.
int run_fft_crop(nfft_plan* p, void* y) {
  if (p->dft1d)
    return cuda_status(p, launch_dft1d_adjoint((int)p->N[0], (int)p->Nt[0], p->grid, p->beta64, p->dft_tw, y,
                                               p->sms, p->stream));
  if (p->pruned) {
    const float* beta[kMaxD];
    return cuda_status(p, launch_pruned_adjoint(p->D, (int)p->Nt[0], p->grid, beta32_dims(p, beta), p->fft_tw, y,
                                                p->stream));
  }
  int s = run_fft(p, +1);
  if (s != NFFT_OK) return s;
  return run_crop_deconv(p, y);
}

int run_crop_deconv(nfft_plan* p, void* y) {
  DeconvArgs a = make_deconv(p);
  cudaError_t e = p->dtype == NFFT_C128 ? launch_crop_deconv<double>(a, p->grid, y, p->stream)
                                        : launch_crop_deconv<float>(a, p->grid, y, p->stream);
  return cuda_status(p, e);
}

// Algorithm 1 (dir 0: correction + pad + FFT, gather) or Algorithm 2 (dir 1:
// scatter, inverse FFT + crop + correction) on device buffers.
int run_plain(nfft_plan* p, int dir, const void* in, void* out) {
  int s = dir == 0 ? run_pad_fft(p, in) : run_scatter(p, in);
  if (s != NFFT_OK) return s;
  return dir == 0 ? run_gather(p, out) : run_fft_crop(p, out);
}

// The same through a CUDA graph in graph mode: captured on the internal
// stream (cuFFT pointed at it meanwhile) the first time a pair of buffers is
// seen, replayed on the plan's stream afterwards.
int run_direction(nfft_plan* p, int dir, const void* in, void* out) {
  // FULL plans rebuild their sparse matrices (new allocations) in
  // nfft_set_nodes, so a captured graph would keep stale pointers: direct path.
  if (!p->graph_mode || (p->flags & NFFT_FLAG_FULL_MATRIX)) return run_plain(p, dir, in, out);
  if (!p->graph[dir] || p->graph_ptr[dir][0] != in || p->graph_ptr[dir][1] != out) {
    if (p->graph[dir]) cudaGraphExecDestroy(p->graph[dir]);
    p->graph[dir] = nullptr;
    if (!p->capture_stream) NFFT_CK(p, cudaStreamCreateWithFlags(&p->capture_stream, cudaStreamNonBlocking));
    cudaStream_t saved = p->stream;
    p->stream = p->capture_stream;
    if (p->fft_ok && cufftSetStream(p->fft, p->capture_stream) != CUFFT_SUCCESS) {
      p->stream = saved;
      return latch(p, NFFT_ERR_CUFFT);
    }
    cudaError_t e = cudaStreamBeginCapture(p->capture_stream, cudaStreamCaptureModeThreadLocal);
    int s = e == cudaSuccess ? run_plain(p, dir, in, out) : NFFT_OK;
    cudaGraph_t graph = nullptr;
    if (e == cudaSuccess) e = cudaStreamEndCapture(p->capture_stream, &graph);
    p->stream = saved;
    if (p->fft_ok && cufftSetStream(p->fft, saved) != CUFFT_SUCCESS) s = latch(p, NFFT_ERR_CUFFT);
    if (s == NFFT_OK && e == cudaSuccess) e = cudaGraphInstantiate(&p->graph[dir], graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (s != NFFT_OK) return s;
    NFFT_CK(p, e);
    p->graph_ptr[dir][0] = in;
    p->graph_ptr[dir][1] = out;
  }
  NFFT_CK(p, cudaGraphLaunch(p->graph[dir], p->stream));
  return NFFT_OK;
}

// Asynchronous host-buffer transform: H2D on p->h2d, the transform on the
// plan stream, D2H on p->d2h, ordered by events; the stage buffers of one
// parity are reused only after the previous call of that parity has read
// its input (ev_comp) and copied its output out (ev_out), so consecutive
// calls overlap one call's copies with another's kernels.
int run_async(nfft_plan* p, int dir, const void* in, size_t in_bytes, void* out, size_t out_bytes) {
  const int k = p->parity;
  const size_t need[2] = {in_bytes, out_bytes};
  for (int b = 0; b < 2; ++b) {
    if (p->astage_bytes[k][b] < need[b]) {
      NFFT_CK(p, cudaStreamSynchronize(p->stream));  // a replaced buffer may still be in use
      NFFT_CK(p, cudaStreamSynchronize(p->h2d));
      NFFT_CK(p, cudaStreamSynchronize(p->d2h));
      dfree(p->astage[k][b]);
      p->astage[k][b] = nullptr;
      p->astage_bytes[k][b] = 0;
      int s = dalloc(p, &p->astage[k][b], need[b]);
      if (s != NFFT_OK) return s;
      p->astage_bytes[k][b] = need[b];
    }
  }
  p->parity ^= 1;
  NFFT_CK(p, cudaStreamWaitEvent(p->h2d, p->ev_comp[k], 0));
  NFFT_CK(p, cudaMemcpyAsync(p->astage[k][0], in, in_bytes, cudaMemcpyHostToDevice, p->h2d));
  NFFT_CK(p, cudaEventRecord(p->ev_in[k], p->h2d));
  NFFT_CK(p, cudaStreamWaitEvent(p->stream, p->ev_in[k], 0));
  NFFT_CK(p, cudaStreamWaitEvent(p->stream, p->ev_out[k], 0));
  int s = run_plain(p, dir, p->astage[k][0], p->astage[k][1]);
  if (s != NFFT_OK) return s;
  NFFT_CK(p, cudaEventRecord(p->ev_comp[k], p->stream));
  NFFT_CK(p, cudaStreamWaitEvent(p->d2h, p->ev_comp[k], 0));
  NFFT_CK(p, cudaMemcpyAsync(out, p->astage[k][1], out_bytes, cudaMemcpyDeviceToHost, p->d2h));
  NFFT_CK(p, cudaEventRecord(p->ev_out[k], p->d2h));
  return NFFT_OK;
}

int run_grad_gather(nfft_plan* p, const void* cot, void* gk) {
  if (p->grad_ctas <= 0 && p->ctas[3] <= 0) return NFFT_ERR_UNSUPPORTED;
  Geometry g = make_geometry(p);
  NodeArrays na = node_arrays(p);
  cudaError_t e =
      p->grad_ctas > 0 ? launch_grad3d_fast(g, p->grid, na, p->poly, cot, gk, p->grad_ctas, p->stream)
      : p->dtype == NFFT_C128
          ? launch_grad_gather<double>(g, p->grid, na, cot, gk, p->ctas[3], p->stream)
          : launch_grad_gather<float>(g, p->grid, na, cot, gk, p->ctas[3], p->stream);
  return cuda_status(p, e);
}

}  // namespace

extern "C" {

const char* nfft_strerror(int code) {
  switch (code) {
    case NFFT_OK: return "success";
    case NFFT_ERR_INVALID_ARG: return "invalid argument";
    case NFFT_ERR_NO_NODES: return "no nodes set (call nfft_set_nodes first)";
    case NFFT_ERR_OOM: return "device memory allocation failed";
    case NFFT_ERR_CUFFT: return "cuFFT error";
    case NFFT_ERR_CUDA: return "CUDA runtime error";
    case NFFT_ERR_TIMEOUT: return "bounded device wait timed out";
    case NFFT_ERR_DEVICE_CHECK: return "device-side range check failed";
    case NFFT_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown status code";
  }
}

int nfft_plan_destroy(nfft_plan* p) {
  if (!p) return NFFT_OK;
  DeviceGuard guard(p->device);
  if (p->stream) cudaStreamSynchronize(p->stream);
  if (p->h2d) cudaStreamSynchronize(p->h2d);
  if (p->d2h) cudaStreamSynchronize(p->d2h);
  drop_graphs(p);
  if (p->capture_stream) cudaStreamDestroy(p->capture_stream);
  for (int k = 0; k < 2; ++k) {
    if (p->ev_in[k]) cudaEventDestroy(p->ev_in[k]);
    if (p->ev_comp[k]) cudaEventDestroy(p->ev_comp[k]);
    if (p->ev_out[k]) cudaEventDestroy(p->ev_out[k]);
    dfree(p->astage[k][0]);
    dfree(p->astage[k][1]);
  }
  if (p->h2d) cudaStreamDestroy(p->h2d);
  if (p->d2h) cudaStreamDestroy(p->d2h);
  if (p->fft_ok) cufftDestroy(p->fft);
  full_destroy(p->full);
  void* bufs[] = {p->grid, p->fft_tw, p->dft_tw, p->beta64, p->beta32, p->poly, p->poly64, p->lut, p->cell, p->frac, p->perm,
                  p->key, p->rank,
                  p->tile_count, p->tile_offset, p->items, p->n_items,
                  p->stage[0], p->stage[1], p->stage[2]};
  for (void* b : bufs) dfree(b);
  delete p;
  return NFFT_OK;
}

int nfft_plan_create(nfft_plan** out, int D, const int64_t* N, int64_t M, double sigma, int m,
                     int dtype, uint32_t flags, void* stream) {
  if (!out) return NFFT_ERR_INVALID_ARG;
  *out = nullptr;
  if (D < 1 || D > kMaxD || !N) return NFFT_ERR_INVALID_ARG;
  if (!(sigma > 1.0) || m < 1 || m > kMaxM) return NFFT_ERR_INVALID_ARG;
  if (dtype != NFFT_C64 && dtype != NFFT_C128) return NFFT_ERR_INVALID_ARG;
  if (M < 0 || M >= ((int64_t)1 << 31)) return NFFT_ERR_INVALID_ARG;
  if (D == 3 && m > 8) return NFFT_ERR_UNSUPPORTED;  // m = 9, 10 are built for 1D and 2D
  if (flags & ~(uint32_t)(NFFT_FLAG_CLOSED_SUPPORT | NFFT_FLAG_COMPENSATED | NFFT_FLAG_FULL_MATRIX |
                          NFFT_FLAG_WIDE_WINDOW | NFFT_FLAG_LIBRARY_FFT | kWindowFlags))
    return NFFT_ERR_INVALID_ARG;
  if ((flags & NFFT_FLAG_CLOSED_SUPPORT) && (flags & NFFT_FLAG_WIDE_WINDOW)) return NFFT_ERR_INVALID_ARG;
  {
    const uint32_t wf = flags & kWindowFlags;
    if (wf & (wf - 1)) return NFFT_ERR_INVALID_ARG;  // at most one window mode
    if (wf && (flags & NFFT_FLAG_FULL_MATRIX)) return NFFT_ERR_INVALID_ARG;
    if ((wf & NFFT_FLAG_WINDOW_LINEAR) && (flags & NFFT_FLAG_WIDE_WINDOW)) return NFFT_ERR_INVALID_ARG;
    if ((wf & NFFT_FLAG_WINDOW_POLYNOMIAL) && (flags & (NFFT_FLAG_WIDE_WINDOW | NFFT_FLAG_CLOSED_SUPPORT)))
      return NFFT_ERR_INVALID_ARG;
  }
  int64_t total = 1;
  for (int d = 0; d < D; ++d) {
    if (N[d] < 2 || N[d] > ((int64_t)1 << 28)) return NFFT_ERR_INVALID_ARG;
    int64_t nt = 2 * (int64_t)ceil(sigma * (double)N[d] / 2.0 - 1e-12);
    if (nt <= 2 * m || nt > ((int64_t)1 << 30)) return NFFT_ERR_INVALID_ARG;
    total *= nt;
    if (total > ((int64_t)1 << 40)) return NFFT_ERR_INVALID_ARG;
  }

  nfft_plan* p = new (std::nothrow) nfft_plan();
  if (!p) return NFFT_ERR_OOM;
  p->D = D;
  p->M = M;
  p->sigma = sigma;
  p->m = m;
  p->dtype = dtype;
  p->flags = flags;
  p->stream = (cudaStream_t)stream;
  const bool closed = (flags & NFFT_FLAG_CLOSED_SUPPORT) != 0;
  const bool wide = (flags & NFFT_FLAG_WIDE_WINDOW) != 0;
  p->K = (closed || wide) ? 2 * m + 2 : 2 * m;
  p->off = (closed || wide) ? -m : -m + 1;
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return NFFT_ERR_CUDA;
  }
  cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device);
  for (int d = 0; d < D; ++d) {
    p->N[d] = N[d];
    p->Nt[d] = 2 * (int64_t)ceil(sigma * (double)N[d] / 2.0 - 1e-12);
    p->b[d] = M_PI * (2.0 - (double)N[d] / (double)p->Nt[d]);
  }

  int s = NFFT_OK;
  int64_t sumN = 0;
  for (int d = 0; d < D; ++d) sumN += N[d];
  if (s == NFFT_OK) s = dalloc(p, &p->grid, (size_t)prod_Nt(p) * cplx_size(p));
  if (s == NFFT_OK) s = dalloc(p, &p->beta64, sizeof(double) * sumN);
  if (s == NFFT_OK) s = dalloc(p, &p->beta32, sizeof(float) * sumN);
  if (s == NFFT_OK) s = dalloc(p, &p->poly, sizeof(float) * D * p->K * (2 * m + 1));
  if (s == NFFT_OK) s = dalloc(p, &p->cell, sizeof(int) * (size_t)(M * D));
  if (s == NFFT_OK) s = dalloc(p, &p->frac, real_size(p) * (size_t)(M * D));
  if (s == NFFT_OK) s = dalloc(p, &p->perm, sizeof(int) * (size_t)M);
  if (s == NFFT_OK) s = dalloc(p, &p->key, sizeof(int) * (size_t)M);
  if (s == NFFT_OK) s = dalloc(p, &p->rank, sizeof(int) * (size_t)M);
  if (s == NFFT_OK) s = dalloc(p, &p->n_items, sizeof(int));
  if (s == NFFT_OK) {
    int64_t T[kMaxD];
    default_tile(p, T);
    s = configure_tiles(p, T);
  }
  if (s == NFFT_OK) {
    int n[kMaxD];
    for (int d = 0; d < D; ++d) n[d] = (int)p->Nt[d];
    cufftResult r = cufftPlanMany(&p->fft, D, n, nullptr, 1, 0, nullptr, 1, 0,
                                  dtype == NFFT_C128 ? CUFFT_Z2Z : CUFFT_C2C, 1);
    if (r != CUFFT_SUCCESS) {
      s = (r == CUFFT_ALLOC_FAILED) ? NFFT_ERR_OOM : NFFT_ERR_CUFFT;
    } else {
      p->fft_ok = true;
      if (cufftSetStream(p->fft, p->stream) != CUFFT_SUCCESS) s = NFFT_ERR_CUFFT;
    }
  }
  if (s == NFFT_OK) {
    int Ni[kMaxD], Nti[kMaxD];
    for (int d = 0; d < D; ++d) {
      Ni[d] = (int)N[d];
      Nti[d] = (int)p->Nt[d];
    }
    s = cuda_status(p, launch_build_beta(D, Ni, Nti, m, p->b, p->beta64, p->beta32, p->stream));
  }
  if (s == NFFT_OK && (flags & NFFT_FLAG_WINDOW_LINEAR)) {
    p->wmode = kWinLinear;
    p->lut_S = lut_table_size(m);
    if ((double)p->lut_S * D * real_size(p) > 8e9) s = NFFT_ERR_UNSUPPORTED;
    if (s == NFFT_OK) s = dalloc(p, &p->lut, (size_t)(p->lut_S * D) * real_size(p));
    if (s == NFFT_OK)
      s = cuda_status(p, launch_build_lut(D, m, p->b, p->lut_S, dtype == NFFT_C128 ? nullptr : (float*)p->lut,
                                          dtype == NFFT_C128 ? (double*)p->lut : nullptr, p->stream));
  }
  // complex128 plans with no window flag take the POLYNOMIAL window as well
  // where its FP64 fit stays at the rounding level of the direct form: the
  // direct form's sqrt, exponential and division cost GB300's narrow FP64
  // units several times a Horner chain.  With m >= 7 the degree-2m fit is
  // within about 1e-14 of the window peak; with oversampling of at least 1.5
  // the table is fitted at degree max(2m, 16) instead (fit error <= 1e-14 of
  // the peak for m = 1..8).  At sigma = 1.25 and m < 7 the correction
  // amplifies even a 1e-14 fit error past the rounding bound (a 3D adjoint at
  // m = 6 came to 4.4e-11 against 4.2e-11), so those keep direct evaluation.
  double min_sigma = 1e300;
  for (int d = 0; d < D; ++d) min_sigma = fmin(min_sigma, (double)p->Nt[d] / (double)N[d]);
  const bool c128_poly_ok = dtype == NFFT_C128 && !(flags & kWindowFlags) && !closed && !wide;
  const bool poly_default = c128_poly_ok && (m >= 7 || min_sigma >= 1.5);
  if (s == NFFT_OK && ((flags & NFFT_FLAG_WINDOW_POLYNOMIAL) || poly_default)) {
    p->wmode = kWinPoly;
    p->poly_Z = 2 * m + 1;
    if (poly_default && 2 * m < 16) p->poly_Z = 17;
    if (dtype == NFFT_C128) s = dalloc(p, &p->poly64, sizeof(double) * D * p->K * p->poly_Z);
  }
  if (s == NFFT_OK && !closed && !wide) {
    PolyArgs pa{};
    pa.D = D;
    pa.K = p->K;
    pa.off = p->off;
    pa.deg = 2 * m;
    pa.m = m;
    for (int d = 0; d < D; ++d) pa.b[d] = p->b[d];
    // the FP32 table (degree 2m) and, at the same degree, the FP64 one
    const bool same = p->poly64 && p->poly_Z == 2 * m + 1;
    s = cuda_status(p, launch_build_poly(pa, p->poly, p->stream, same ? p->poly64 : nullptr));
    if (s == NFFT_OK && p->poly64 && !same) {
      pa.deg = p->poly_Z - 1;
      s = cuda_status(p, launch_build_poly(pa, nullptr, p->stream, p->poly64));
    }
  }
  if (s == NFFT_OK && dtype == NFFT_C64 && !(flags & NFFT_FLAG_LIBRARY_FFT)) {
    int Ni[kMaxD], Nti[kMaxD];
    for (int d = 0; d < D; ++d) {
      Ni[d] = (int)N[d];
      Nti[d] = (int)p->Nt[d];
    }
    if (pruned_fft_supported(D, Ni, Nti)) {
      s = dalloc(p, &p->fft_tw, sizeof(float2) * kPrunedFftTwiddles);
      if (s == NFFT_OK) s = cuda_status(p, build_fft_twiddles(D, Nti[0], p->fft_tw, p->stream));
      p->pruned = s == NFFT_OK;
    }
  }
  if (s == NFFT_OK && dtype == NFFT_C128 && !(flags & NFFT_FLAG_LIBRARY_FFT) &&
      dft1d_supported(D, (int)N[0], (int)p->Nt[0])) {
    s = dalloc(p, &p->dft_tw, sizeof(double2) * (size_t)p->Nt[0]);
    if (s == NFFT_OK) s = cuda_status(p, launch_dft_twiddles(p->dft_tw, (int)p->Nt[0], p->stream));
    p->dft1d = s == NFFT_OK;
  }
  if (s == NFFT_OK) s = cuda_status(p, cudaMemsetAsync(p->n_items, 0, sizeof(int), p->stream));
  if (s != NFFT_OK) {
    nfft_plan_destroy(p);
    return s;
  }
  *out = p;
  return NFFT_OK;
}

int nfft_set_nodes(nfft_plan* p, const void* k, int k_is_fp64) {
  int s;
  if (!ready(p, &s)) return s;
  if (!k && p->M > 0) return NFFT_ERR_INVALID_ARG;
  DeviceGuard guard(p->device);
  // k is FP64 (k_is_fp64 != 0) or FP32 for either plan dtype; FP32 nodes are
  // promoted to FP64 before the split.
  const void* kd = nullptr;
  s = device_input(p, 2, k, p->M > 0 ? (size_t)(p->M * p->D) * (k_is_fp64 ? 8 : 4) : 0, &kd);
  if (s != NFFT_OK) return s;
  SortArgs a{};
  a.D = p->D;
  a.M = (int)p->M;
  for (int d = 0; d < p->D; ++d) {
    a.Nt[d] = (int)p->Nt[d];
    a.T[d] = (int)p->T[d];
    a.ntile[d] = p->ntile[d];
  }
  a.n_tiles = (int)p->n_tiles;
  a.cmax = p->cmax;
  a.max_items = (int)p->max_items;
  NFFT_CK(p, launch_node_count(a, kd, k_is_fp64 ? 1 : 0, p->tile_count, p->key, p->rank, p->stream));
  NFFT_CK(p, launch_tile_scan(a, p->tile_count, p->tile_offset, p->items, p->n_items, p->stream));
  NFFT_CK(p, launch_node_place(a, kd, k_is_fp64 ? 1 : 0, p->key, p->rank, p->tile_offset, p->cell,
                               p->frac, p->dtype == NFFT_C128 ? 1 : 0, p->perm, p->stream));
  if (p->flags & NFFT_FLAG_FULL_MATRIX) {
    s = full_build(&p->full, make_geometry(p), p->dtype, node_arrays(p), p->stream);
    if (s != NFFT_OK) return latch(p, s);
  }
  if (kd != k) NFFT_CK(p, cudaStreamSynchronize(p->stream));  // stage buffer reuse safety
  p->has_nodes = true;
  return NFFT_OK;
}

int nfft_forward(nfft_plan* p, const void* f, void* fhat) {
  int s;
  if (!ready(p, &s)) return s;
  if (!p->has_nodes) return NFFT_ERR_NO_NODES;
  if (!f || (!fhat && p->M > 0)) return NFFT_ERR_INVALID_ARG;
  DeviceGuard guard(p->device);
  if (p->async_mode && p->M > 0 && !is_device_pointer(f) && !is_device_pointer(fhat))
    return run_async(p, 0, f, (size_t)prod_N(p) * cplx_size(p), fhat, (size_t)p->M * cplx_size(p));
  const void* fd = nullptr;
  OutputBinding ob;
  if ((s = device_input(p, 0, f, (size_t)prod_N(p) * cplx_size(p), &fd)) != NFFT_OK) return s;
  if ((s = device_output(p, 1, fhat, (size_t)p->M * cplx_size(p), &ob)) != NFFT_OK) return s;
  if (fd == f && !ob.host) return run_direction(p, 0, fd, ob.dev);
  if ((s = run_plain(p, 0, fd, ob.dev)) != NFFT_OK) return s;
  return finish_output(p, ob);
}

int nfft_adjoint(nfft_plan* p, const void* fhat, void* y) {
  int s;
  if (!ready(p, &s)) return s;
  if (!p->has_nodes) return NFFT_ERR_NO_NODES;
  if (!y || (!fhat && p->M > 0)) return NFFT_ERR_INVALID_ARG;
  DeviceGuard guard(p->device);
  if (p->async_mode && p->M > 0 && !is_device_pointer(fhat) && !is_device_pointer(y))
    return run_async(p, 1, fhat, (size_t)p->M * cplx_size(p), y, (size_t)prod_N(p) * cplx_size(p));
  const void* fd = nullptr;
  OutputBinding ob;
  if ((s = device_input(p, 0, fhat, (size_t)p->M * cplx_size(p), &fd)) != NFFT_OK) return s;
  if ((s = device_output(p, 1, y, (size_t)prod_N(p) * cplx_size(p), &ob)) != NFFT_OK) return s;
  if (fd == fhat && !ob.host) return run_direction(p, 1, fd, ob.dev);
  if ((s = run_plain(p, 1, fd, ob.dev)) != NFFT_OK) return s;
  return finish_output(p, ob);
}

int nfft_grad(nfft_plan* p, const void* f, const void* cot, void* gk) {
  int s;
  if (!ready(p, &s)) return s;
  if (!p->has_nodes) return NFFT_ERR_NO_NODES;
  if (!f || ((!cot || !gk) && p->M > 0)) return NFFT_ERR_INVALID_ARG;
  DeviceGuard guard(p->device);
  const void* fd = nullptr;
  const void* cd = nullptr;
  OutputBinding ob;
  if ((s = device_input(p, 0, f, (size_t)prod_N(p) * cplx_size(p), &fd)) != NFFT_OK) return s;
  if ((s = device_input(p, 2, cot, (size_t)p->M * cplx_size(p), &cd)) != NFFT_OK) return s;
  if ((s = device_output(p, 1, gk, (size_t)(p->M * p->D) * real_size(p), &ob)) != NFFT_OK) return s;
  if ((s = run_pad_fft(p, fd)) != NFFT_OK) return s;
  if ((s = run_grad_gather(p, cd, ob.dev)) != NFFT_OK) return s;
  return finish_output(p, ob);
}

int nfft_plan_sync(nfft_plan* p) {
  if (!p) return NFFT_ERR_INVALID_ARG;
  DeviceGuard guard(p->device);
  cudaError_t e = cudaStreamSynchronize(p->stream);
  if (e == cudaSuccess && p->h2d) e = cudaStreamSynchronize(p->h2d);
  if (e == cudaSuccess && p->d2h) e = cudaStreamSynchronize(p->d2h);
  if (e != cudaSuccess) return cuda_status(p, e);
  if (p->fast_gather && p->D == 3) {
    const int t = fast3d_take_wait_timeout();
    if (t < 0) return latch(p, NFFT_ERR_CUDA);
    if (t > 0) return latch(p, NFFT_ERR_TIMEOUT);
  }
  return p->err;
}

int nfft_plan_info(nfft_plan* p, int64_t* Ntilde3, int64_t* tile3, int64_t* n_items) {
  if (!p) return NFFT_ERR_INVALID_ARG;
  for (int d = 0; d < kMaxD; ++d) {
    if (Ntilde3) Ntilde3[d] = d < p->D ? p->Nt[d] : 1;
    if (tile3) tile3[d] = d < p->D ? p->T[d] : 1;
  }
  if (n_items) {
    *n_items = 0;
    if (p->has_nodes) {
      DeviceGuard guard(p->device);
      int h = 0;
      NFFT_CK(p, cudaMemcpyAsync(&h, p->n_items, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
      NFFT_CK(p, cudaStreamSynchronize(p->stream));
      *n_items = h;
    }
  }
  return p->err;
}

void* nfft_plan_grid(nfft_plan* p) { return p ? p->grid : nullptr; }

int nfft_plan_set_tile(nfft_plan* p, const int64_t* tile3) {
  int s;
  if (!ready(p, &s)) return s;
  if (!tile3) return NFFT_ERR_INVALID_ARG;
  int64_t T[kMaxD] = {1, 1, 1};
  for (int d = 0; d < p->D; ++d) {
    if (tile3[d] < 1 || tile3[d] > p->Nt[d]) return NFFT_ERR_INVALID_ARG;
    T[d] = tile3[d];
  }
  const int kind = (p->flags & NFFT_FLAG_COMPENSATED) ? 2 : 1;
  if (region_bytes(p, T, kind) > 227 * 1024) return NFFT_ERR_INVALID_ARG;
  DeviceGuard guard(p->device);
  s = configure_tiles(p, T);
  if (s != NFFT_OK) return s;
  p->has_nodes = false;  // the bin-sort depends on the tile shape
  return NFFT_OK;
}

// Tile-shape autotuner (Sec. 5.2 sweeps the block size; Sec. 6 proposes an
// FFTW_MEASURE-like automatic choice): time forward + adjoint for each
// candidate tile on the caller's nodes, keep the fastest, cache it per shape.
namespace {
std::mutex g_plan_tune_mutex;
std::map<std::string, std::vector<int64_t>> g_plan_tune_cache;

std::vector<std::vector<int64_t>> plan_tile_candidates(const nfft_plan* p) {
  std::vector<std::vector<int64_t>> c;
  if (p->D == 1) {
    for (int64_t t : {64, 128, 256, 512, 1024, 2048, 4096}) c.push_back({t, 1, 1});
  } else if (p->D == 2) {
    for (int64_t t : {8, 16, 32, 64}) c.push_back({t, t, 1});
    c.push_back({16, 32, 1});
    c.push_back({32, 16, 1});
    c.push_back({9, 25, 1});
    c.push_back({8, 25, 1});
  } else {
    for (int64_t t : {4, 8, 16}) c.push_back({t, t, t});
    c.push_back({8, 8, 4});
    c.push_back({4, 8, 8});
    c.push_back({16, 8, 8});
    c.push_back({6, 8, 8});  // best in the tile sweep at twice the headline density
    c.push_back({9, 9, 8});
    c.push_back({9, 9, 9});
    c.push_back({5, 5, 5});
    c.push_back({5, 5, 4});
  }
  std::vector<std::vector<int64_t>> ok;
  const int kind = (p->flags & NFFT_FLAG_COMPENSATED) ? 2 : 1;
  for (auto& t : c) {
    bool fits = true;
    for (int d = 0; d < p->D; ++d)
      if (t[d] > p->Nt[d]) fits = false;
    if (fits && region_bytes(p, t.data(), kind) <= 160 * 1024) ok.push_back(t);
  }
  return ok;
}
}  // namespace

int nfft_plan_autotune(nfft_plan* p, const void* k, int k_is_fp64, int64_t* chosen3) {
  int s;
  if (!ready(p, &s)) return s;
  if (!k && p->M > 0) return NFFT_ERR_INVALID_ARG;
  DeviceGuard guard(p->device);
  std::string key = "plan:" + std::to_string(p->device) + ":" + std::to_string(p->D) + ":" +
                    std::to_string(p->m) + ":" + std::to_string(p->dtype) + ":" + std::to_string(p->flags) +
                    ":" + std::to_string(p->M) + ":" + std::to_string(p->sigma);
  for (int d = 0; d < p->D; ++d) key += "," + std::to_string(p->N[d]);
  std::vector<int64_t> best;
  {
    std::lock_guard<std::mutex> lock(g_plan_tune_mutex);
    auto it = g_plan_tune_cache.find(key);
    if (it != g_plan_tune_cache.end()) best = it->second;
  }
  if (best.empty()) {
    void *f = nullptr, *fh = nullptr;
    s = dalloc(p, &f, (size_t)prod_N(p) * cplx_size(p));
    if (s == NFFT_OK) s = dalloc(p, &fh, (size_t)p->M * cplx_size(p));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (s == NFFT_OK) {
      cudaMemsetAsync(f, 0, (size_t)prod_N(p) * cplx_size(p), p->stream);
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
    }
    float best_ms = 1e30f;
    for (auto& t : plan_tile_candidates(p)) {
      if (s != NFFT_OK) break;
      if ((s = configure_tiles(p, t.data())) != NFFT_OK) break;
      if ((s = nfft_set_nodes(p, k, k_is_fp64)) != NFFT_OK) break;
      float ms = 0.f;
      for (int rep = 0; rep < 3 && s == NFFT_OK; ++rep) {
        cudaEventRecord(e0, p->stream);
        s = nfft_forward(p, f, fh);
        if (s == NFFT_OK) s = nfft_adjoint(p, fh, f);
        cudaEventRecord(e1, p->stream);
        cudaEventSynchronize(e1);
        float t_ms = 0.f;
        cudaEventElapsedTime(&t_ms, e0, e1);
        if (rep > 0) ms += t_ms;  // the first repeat warms up
      }
      if (s == NFFT_OK && ms < best_ms) {
        best_ms = ms;
        best = t;
      }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dfree(f);
    dfree(fh);
    if (s != NFFT_OK) return s;
    if (best.empty()) return NFFT_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_plan_tune_mutex);
    g_plan_tune_cache[key] = best;
  }
  if ((s = configure_tiles(p, best.data())) != NFFT_OK) return s;
  if ((s = nfft_set_nodes(p, k, k_is_fp64)) != NFFT_OK) return s;
  if (chosen3)
    for (int d = 0; d < kMaxD; ++d) chosen3[d] = d < p->D ? best[d] : 1;
  return NFFT_OK;
}

int nfft_step_deconv_pad(nfft_plan* p, const void* f) {
  int s;
  if (!ready(p, &s)) return s;
  if (!f) return NFFT_ERR_INVALID_ARG;
  DeviceGuard guard(p->device);
  return run_deconv_pad(p, f);
}

int nfft_step_fft(nfft_plan* p, int sign) {
  int s;
  if (!ready(p, &s)) return s;
  if (sign != -1 && sign != 1) return NFFT_ERR_INVALID_ARG;
  DeviceGuard guard(p->device);
  return run_fft(p, sign);
}

int nfft_step_gather(nfft_plan* p, void* fhat) {
  int s;
  if (!ready(p, &s)) return s;
  if (!p->has_nodes) return NFFT_ERR_NO_NODES;
  if (!fhat && p->M > 0) return NFFT_ERR_INVALID_ARG;
  DeviceGuard guard(p->device);
  return run_gather(p, fhat);
}

int nfft_step_scatter(nfft_plan* p, const void* fhat) {
  int s;
  if (!ready(p, &s)) return s;
  if (!p->has_nodes) return NFFT_ERR_NO_NODES;
  if (!fhat && p->M > 0) return NFFT_ERR_INVALID_ARG;
  DeviceGuard guard(p->device);
  return run_scatter(p, fhat);
}

int nfft_step_crop_deconv(nfft_plan* p, void* y) {
  int s;
  if (!ready(p, &s)) return s;
  if (!y) return NFFT_ERR_INVALID_ARG;
  DeviceGuard guard(p->device);
  return run_crop_deconv(p, y);
}

int nfft_step_pad_fft(nfft_plan* p, const void* f) {
  int s;
  if (!ready(p, &s)) return s;
  if (!f) return NFFT_ERR_INVALID_ARG;
  DeviceGuard guard(p->device);
  return run_pad_fft(p, f);
}

int nfft_step_fft_crop(nfft_plan* p, void* y) {
  int s;
  if (!ready(p, &s)) return s;
  if (!y) return NFFT_ERR_INVALID_ARG;
  DeviceGuard guard(p->device);
  return run_fft_crop(p, y);
}

int nfft_plan_set_graph(nfft_plan* p, int enable) {
  int s;
  if (!ready(p, &s)) return s;
  DeviceGuard guard(p->device);
  if (!enable) drop_graphs(p);
  p->graph_mode = enable != 0;
  return NFFT_OK;
}

int nfft_plan_set_async(nfft_plan* p, int enable) {
  int s;
  if (!ready(p, &s)) return s;
  DeviceGuard guard(p->device);
  if (enable && !p->h2d) {
    NFFT_CK(p, cudaStreamCreateWithFlags(&p->h2d, cudaStreamNonBlocking));
    NFFT_CK(p, cudaStreamCreateWithFlags(&p->d2h, cudaStreamNonBlocking));
    for (int k = 0; k < 2; ++k) {
      NFFT_CK(p, cudaEventCreateWithFlags(&p->ev_in[k], cudaEventDisableTiming));
      NFFT_CK(p, cudaEventCreateWithFlags(&p->ev_comp[k], cudaEventDisableTiming));
      NFFT_CK(p, cudaEventCreateWithFlags(&p->ev_out[k], cudaEventDisableTiming));
    }
  }
  if (!enable && p->h2d) {
    NFFT_CK(p, cudaStreamSynchronize(p->h2d));
    NFFT_CK(p, cudaStreamSynchronize(p->d2h));
  }
  p->async_mode = enable != 0;
  return NFFT_OK;
}

int nfft_plan_paths(nfft_plan* p, int* fast_resample, int* pruned_fft) {
  if (!p) return NFFT_ERR_INVALID_ARG;
  if (fast_resample) *fast_resample = (p->fast_gather ? 1 : 0) | (p->fast_scatter ? 2 : 0);
  if (pruned_fft) *pruned_fft = p->pruned ? 1 : (p->dft1d ? 2 : 0);
  return NFFT_OK;
}

int nfft_step_grad_gather(nfft_plan* p, const void* cot, void* gk) {
  int s;
  if (!ready(p, &s)) return s;
  if (!p->has_nodes) return NFFT_ERR_NO_NODES;
  if ((!cot || !gk) && p->M > 0) return NFFT_ERR_INVALID_ARG;
  DeviceGuard guard(p->device);
  return run_grad_gather(p, cot, gk);
}

}  // extern "C"
