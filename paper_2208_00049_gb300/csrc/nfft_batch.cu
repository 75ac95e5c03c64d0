// Batched NFFTs (many problems, uneven N and M, shared or distinct node sets)
// and the tile-shape autotuner.  See include/nfft_gb300.h.
//
// Layout: the oversampled grids of all problems sit in one buffer, grouped by
// size class so that each class is one batched cuFFT plan; the node sets'
// sorted records are concatenated; the work items of every problem form one
// list ({tile, first node, count, problem}) walked by one persistent gather /
// scatter launch.  Forward = deconv_pad (one launch, blockIdx.y = problem) ->
// one cuFFT per size class -> gather (one launch); adjoint = memset ->
// scatter (one launch) -> cuFFT per class -> crop_deconv (one launch).  The
// size classes' FFTs are independent and most are small (a 128 x 128 class
// cannot fill the GPU), so they run concurrently: forked from the batch's
// stream onto a few side streams (classes assigned largest first to the
// least loaded stream) and joined back with events.  With graph mode on,
// each sequence is captured once into a CUDA graph (the fork and join become
// parallel branches of the graph) and replayed while the caller's buffers
// stay the same.
//
// Tile shapes (the block size of Sec. 3.7.3, whose best value the paper finds
// by a sweep, Sec. 5.2, and proposes to choose automatically like
// FFTW_MEASURE, Sec. 6) are chosen by timing candidate shapes on the actual
// nodes.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "nfft_internal.cuh"

using namespace nfftgb;

struct nfft_batch {
  int D = 0, B = 0, S = 0;
  double sigma = 2.0;
  int m = 4, dtype = NFFT_C64;
  uint32_t flags = 0;
  cudaStream_t stream = nullptr;
  int device = 0, sms = 1;
  int K = 8, off = -3, cmax = 128;
  int64_t T[kMaxD] = {1, 1, 1};

  std::vector<int64_t> N, Nt;          // [B * D]
  std::vector<int> set_of;              // [B]
  std::vector<int64_t> M_set, node_off; // [S]
  std::vector<int64_t> grid_off, in_off, out_off, beta_off;  // [B]
  int64_t grid_total = 0, in_total = 0, out_total = 0, node_total = 0, beta_total = 0;
  int64_t poly_per = 0;                 // POLYNOMIAL coefficients per problem (0: not built)
  int64_t max_grid = 0, max_n = 0, max_set_nodes = 0, max_tiles = 0;
  std::vector<int> set_tiles;           // tiles of each node set
  std::vector<int64_t> set_item_base;   // offsets into set_items
  int64_t set_items_total = 0;

  struct SizeClass {
    std::vector<int64_t> nt;
    int64_t first_grid_off = 0;
    int count = 0;
    cufftHandle plan = 0;
    bool ok = false;
    int side = 0;  // side stream of this class's FFT
  };
  std::vector<SizeClass> classes;
  std::vector<cudaStream_t> fft_streams;  // empty: the FFTs run on the calling stream
  std::vector<cudaEvent_t> join_ev;       // one per side stream
  cudaEvent_t fork_ev = nullptr;

  void* grid = nullptr;
  double* beta64 = nullptr;
  float* beta32 = nullptr;
  float* poly = nullptr;  // [B][D][K][2m + 1], built for the standard (2m-tap) window only
  int* pad_blocks = nullptr;   // [B + 1] block ranges of the batched deconv_pad launch
  int* crop_blocks = nullptr;  // [B + 1] block ranges of the batched crop_deconv launch
  int n_pad_blocks = 0, n_crop_blocks = 0;
  BatchProblem* probs = nullptr;
  std::vector<BatchProblem> probs_host;
  int* cell = nullptr;
  void* frac = nullptr;
  int* perm = nullptr;
  int* key = nullptr;
  int* rank = nullptr;
  int* tile_count = nullptr;
  int* tile_offset = nullptr;
  int4* set_items = nullptr;
  int* set_nitems = nullptr;
  int4* items = nullptr;
  int* n_items = nullptr;
  int* item_off = nullptr;
  int64_t items_cap = 0;
  int ctas[2] = {0, 0};
  bool fast_scatter = false;  // 2D m = 4 complex64 register-accumulating scatter and warp gather
  int fast_ctas = 0, fast_gather_ctas = 0;

  bool has_nodes = false;
  bool graph_mode = false;
  cudaStream_t capture_stream = nullptr;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};  // forward, adjoint
  const void* graph_ptr[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  int err = NFFT_OK;
};

namespace {

constexpr int kFftSideStreams = 4;  // concurrent size-class FFTs

size_t rsize(int dtype) { return dtype == NFFT_C128 ? 8 : 4; }
size_t csize(int dtype) { return 2 * rsize(dtype); }

int bst(nfft_batch* b, cudaError_t e) {
  if (e == cudaSuccess) return NFFT_OK;
  cudaGetLastError();
  int code = e == cudaErrorMemoryAllocation ? NFFT_ERR_OOM : NFFT_ERR_CUDA;
  if (b && b->err == NFFT_OK) b->err = code;
  return code;
}

#define B_CK(b, call)                   \
  do {                                  \
    int _s = bst((b), (call));          \
    if (_s != NFFT_OK) return _s;       \
  } while (0)

template <typename T>
int balloc(nfft_batch* b, T** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (cudaMalloc((void**)p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    if (b->err == NFFT_OK) b->err = NFFT_ERR_OOM;
    return NFFT_ERR_OOM;
  }
  return NFFT_OK;
}

Geometry problem_geometry(const nfft_batch* b, int p) {
  Geometry g{};
  g.D = b->D;
  g.K = b->K;
  g.off = b->off;
  g.closed = (b->flags & NFFT_FLAG_CLOSED_SUPPORT) ? 1 : 0;
  g.M = (int)b->M_set[b->set_of[p]];
  g.m = (double)b->m;
  for (int d = 0; d < b->D; ++d) {
    const int64_t nt = b->Nt[p * b->D + d];
    int64_t t = b->T[d];
    int64_t cap = nt - b->K + 1;
    if (cap < 1) cap = 1;
    if (t > cap) t = cap;
    g.Nt[d] = (int)nt;
    g.T[d] = (int)t;
    g.ntile[d] = (int)((nt + t - 1) / t);
    g.L[d] = (int)t + b->K - 1;
    g.b[d] = M_PI * (2.0 - (double)b->N[p * b->D + d] / (double)nt);
    g.norm[d] = (double)b->m / sinh(g.b[d] * (double)b->m);
  }
  return g;
}

Geometry max_geometry(const nfft_batch* b) {
  Geometry gm = problem_geometry(b, 0);
  for (int p = 1; p < b->B; ++p) {
    Geometry g = problem_geometry(b, p);
    for (int d = 0; d < b->D; ++d)
      if (g.L[d] > gm.L[d]) gm.L[d] = g.L[d];
  }
  return gm;
}

size_t max_region_bytes(const nfft_batch* b, const int64_t* T) {
  size_t r = 1;
  for (int d = 0; d < b->D; ++d) r *= (size_t)(T[d] + b->K - 1);
  return r * csize(b->dtype);
}

// Tiles, work-item capacity, problem table and persistent grid sizes for the
// current tile shape.
int configure(nfft_batch* b) {
  b->probs_host.resize(b->B);
  b->set_tiles.assign(b->S, 0);
  b->max_tiles = 0;
  for (int p = 0; p < b->B; ++p) {
    BatchProblem P{};
    P.g = problem_geometry(b, p);
    for (int d = 0; d < b->D; ++d) P.N[d] = (int)b->N[p * b->D + d];
    P.grid_off = b->grid_off[p];
    P.node_off = b->node_off[b->set_of[p]];
    P.out_off = b->out_off[p];
    P.in_off = b->in_off[p];
    P.beta_off = b->beta_off[p];
    P.poly_off = p * b->poly_per;
    b->probs_host[p] = P;
    int64_t nt = 1;
    for (int d = 0; d < b->D; ++d) nt *= P.g.ntile[d];
    if (nt > ((int64_t)1 << 30)) return NFFT_ERR_INVALID_ARG;
    b->set_tiles[b->set_of[p]] = (int)nt;
    if (nt > b->max_tiles) b->max_tiles = nt;
  }
  b->set_item_base.assign(b->S, 0);
  int64_t tot = 0, items_total = 0;
  for (int s = 0; s < b->S; ++s) {
    b->set_item_base[s] = tot;
    tot += b->set_tiles[s] + (b->M_set[s] + b->cmax - 1) / b->cmax + 1;
  }
  for (int p = 0; p < b->B; ++p) {
    const int s = b->set_of[p];
    items_total += b->set_tiles[s] + (b->M_set[s] + b->cmax - 1) / b->cmax + 1;
  }
  // (re)allocate tile and item buffers
  cudaFree(b->tile_count);
  cudaFree(b->tile_offset);
  cudaFree(b->set_items);
  cudaFree(b->items);
  b->tile_count = b->tile_offset = nullptr;
  b->set_items = b->items = nullptr;
  int s = balloc(b, &b->tile_count, sizeof(int) * b->max_tiles);
  if (s == NFFT_OK) s = balloc(b, &b->tile_offset, sizeof(int) * b->max_tiles);
  if (s == NFFT_OK) s = balloc(b, &b->set_items, sizeof(int4) * tot);
  if (s == NFFT_OK) s = balloc(b, &b->items, sizeof(int4) * items_total);
  if (s != NFFT_OK) return s;
  b->set_items_total = tot;
  b->items_cap = items_total;
  B_CK(b, cudaMemcpyAsync(b->probs, b->probs_host.data(), sizeof(BatchProblem) * b->B, cudaMemcpyHostToDevice,
                          b->stream));
  const Geometry gm = max_geometry(b);
  for (int kind = 0; kind < 2; ++kind) {
    int per = b->dtype == NFFT_C128 ? resample_batch_ctas_per_sm<double>(gm, kind)
                                    : resample_batch_ctas_per_sm<float>(gm, kind);
    if (per <= 0) return NFFT_ERR_UNSUPPORTED;
    b->ctas[kind] = per * b->sms;
  }
  b->fast_scatter = b->D == 2 && b->dtype == NFFT_C64 && !(b->flags & NFFT_FLAG_COMPENSATED) && b->poly_per > 0;
  for (int p = 0; p < b->B && b->fast_scatter; ++p) b->fast_scatter = scatter2d_supported(b->probs_host[p].g);
  if (b->fast_scatter) {
    const int per = scatter2d_ctas_per_sm(), per_g = gather2d_ctas_per_sm();
    b->fast_scatter = per > 0 && per_g > 0;
    b->fast_ctas = per * b->sms;
    b->fast_gather_ctas = per_g * b->sms;
  }
  for (int k = 0; k < 2; ++k) {
    if (b->graph[k]) cudaGraphExecDestroy(b->graph[k]);
    b->graph[k] = nullptr;
  }
  b->has_nodes = false;
  return NFFT_OK;
}

void default_batch_tile(const nfft_batch* b, int64_t* T) {
  const int64_t t = b->D == 1 ? 256 : (b->D == 2 ? 32 : 8);
  for (int d = 0; d < kMaxD; ++d) T[d] = d < b->D ? t : 1;
}

int batch_set_nodes_stream(nfft_batch* b, const void* k, int k_is_fp64, cudaStream_t st) {
  const size_t kel = k_is_fp64 ? 8 : 4;
  B_CK(b, cudaMemsetAsync(b->set_nitems, 0, sizeof(int) * b->S, st));
  for (int s = 0; s < b->S; ++s) {
    int p = 0;
    while (b->set_of[p] != s) ++p;  // every set has a problem (checked at create)
    const Geometry g = b->probs_host[p].g;
    SortArgs a{};
    a.D = b->D;
    a.M = (int)b->M_set[s];
    for (int d = 0; d < b->D; ++d) {
      a.Nt[d] = g.Nt[d];
      a.T[d] = g.T[d];
      a.ntile[d] = g.ntile[d];
    }
    a.n_tiles = b->set_tiles[s];
    a.cmax = b->cmax;
    a.max_items = (int)(b->set_tiles[s] + (b->M_set[s] + b->cmax - 1) / b->cmax + 1);
    const int64_t no = b->node_off[s];
    const void* ks = (const char*)k + kel * (size_t)(no * b->D);
    int* cell = b->cell + b->D * no;
    void* frac = (char*)b->frac + rsize(b->dtype) * (size_t)(b->D * no);
    B_CK(b, launch_node_count(a, ks, k_is_fp64, b->tile_count, b->key, b->rank, st));
    B_CK(b, launch_tile_scan(a, b->tile_count, b->tile_offset, b->set_items + b->set_item_base[s],
                             b->set_nitems + s, st));
    B_CK(b, launch_node_place(a, ks, k_is_fp64, b->key, b->rank, b->tile_offset, cell, frac,
                              b->dtype == NFFT_C128 ? 1 : 0, b->perm + no, st));
  }
  // problem item lists: offsets need the per-set counts on the host
  std::vector<int> cnt(b->S);
  B_CK(b, cudaMemcpyAsync(cnt.data(), b->set_nitems, sizeof(int) * b->S, cudaMemcpyDeviceToHost, st));
  B_CK(b, cudaStreamSynchronize(st));
  std::vector<int> offs(b->B + 1, 0);
  for (int p = 0; p < b->B; ++p) offs[p + 1] = offs[p] + cnt[b->set_of[p]];
  B_CK(b, cudaMemcpyAsync(b->item_off, offs.data(), sizeof(int) * (b->B + 1), cudaMemcpyHostToDevice, st));
  for (int p = 0; p < b->B; ++p) {
    const int s = b->set_of[p];
    B_CK(b, launch_items_expand(b->set_items + b->set_item_base[s], b->set_nitems + s, cnt[s] > 0 ? cnt[s] : 1,
                                b->items, b->item_off + p, p, st));
  }
  B_CK(b, cudaMemcpyAsync(b->n_items, b->item_off + b->B, sizeof(int), cudaMemcpyDeviceToDevice, st));
  B_CK(b, cudaStreamSynchronize(st));  // host vectors above go out of scope
  b->has_nodes = true;
  return NFFT_OK;
}

BatchNodes batch_nodes(const nfft_batch* b) {
  BatchNodes nb;
  nb.cell = b->cell;
  nb.frac = b->frac;
  nb.perm = b->perm;
  nb.items = b->items;
  nb.n_items = b->n_items;
  return nb;
}

int run_fft_classes(nfft_batch* b, int sign, cudaStream_t st) {
  const int ns = (int)b->fft_streams.size();
  if (ns > 0) {  // fork
    B_CK(b, cudaEventRecord(b->fork_ev, st));
    for (cudaStream_t side : b->fft_streams) B_CK(b, cudaStreamWaitEvent(side, b->fork_ev, 0));
  }
  for (auto& c : b->classes) {
    if (cufftSetStream(c.plan, ns > 0 ? b->fft_streams[c.side] : st) != CUFFT_SUCCESS) return NFFT_ERR_CUFFT;
    const int dir = sign < 0 ? CUFFT_FORWARD : CUFFT_INVERSE;
    cufftResult r;
    if (b->dtype == NFFT_C128) {
      auto* g = (cufftDoubleComplex*)b->grid + c.first_grid_off;
      r = cufftExecZ2Z(c.plan, g, g, dir);
    } else {
      auto* g = (cufftComplex*)b->grid + c.first_grid_off;
      r = cufftExecC2C(c.plan, g, g, dir);
    }
    if (r != CUFFT_SUCCESS) return NFFT_ERR_CUFFT;
  }
  for (int k = 0; k < ns; ++k) {  // join
    B_CK(b, cudaEventRecord(b->join_ev[k], b->fft_streams[k]));
    B_CK(b, cudaStreamWaitEvent(st, b->join_ev[k], 0));
  }
  return NFFT_OK;
}

const void* beta_ptr(const nfft_batch* b) {
  return b->dtype == NFFT_C128 ? (const void*)b->beta64 : (const void*)b->beta32;
}

int enqueue_forward(nfft_batch* b, const void* f, void* fhat, cudaStream_t st) {
  const Geometry gm = max_geometry(b);
  cudaError_t e = b->dtype == NFFT_C128
                      ? launch_deconv_pad_batch<double>(b->D, b->B, b->pad_blocks, b->n_pad_blocks, b->probs,
                                                        beta_ptr(b), f, b->grid, st)
                      : launch_deconv_pad_batch<float>(b->D, b->B, b->pad_blocks, b->n_pad_blocks, b->probs,
                                                       beta_ptr(b), f, b->grid, st);
  B_CK(b, e);
  int s = run_fft_classes(b, -1, st);
  if (s != NFFT_OK) return s;
  e = b->fast_scatter
          ? launch_gather2d_fast_batch(b->probs, b->grid, batch_nodes(b), b->poly, fhat, b->fast_gather_ctas, st)
      : b->dtype == NFFT_C128
          ? launch_gather_batch<double>(b->probs, gm, b->grid, batch_nodes(b), fhat, b->ctas[0], st)
          : launch_gather_batch<float>(b->probs, gm, b->grid, batch_nodes(b), fhat, b->ctas[0], st);
  B_CK(b, e);
  return NFFT_OK;
}

int enqueue_adjoint(nfft_batch* b, const void* fhat, void* y, cudaStream_t st) {
  const Geometry gm = max_geometry(b);
  B_CK(b, cudaMemsetAsync(b->grid, 0, (size_t)b->grid_total * csize(b->dtype), st));
  cudaError_t e = b->fast_scatter
                      ? launch_scatter2d_fast_batch(b->probs, b->grid, batch_nodes(b), b->poly, fhat, b->fast_ctas, st)
                  : b->dtype == NFFT_C128
                      ? launch_scatter_batch<double>(b->probs, gm, b->grid, batch_nodes(b), fhat, b->ctas[1], st)
                      : launch_scatter_batch<float>(b->probs, gm, b->grid, batch_nodes(b), fhat, b->ctas[1], st);
  B_CK(b, e);
  int s = run_fft_classes(b, +1, st);
  if (s != NFFT_OK) return s;
  e = b->dtype == NFFT_C128
          ? launch_crop_deconv_batch<double>(b->D, b->B, b->crop_blocks, b->n_crop_blocks, b->probs, beta_ptr(b),
                                             b->grid, y, st)
          : launch_crop_deconv_batch<float>(b->D, b->B, b->crop_blocks, b->n_crop_blocks, b->probs, beta_ptr(b),
                                            b->grid, y, st);
  B_CK(b, e);
  return NFFT_OK;
}

// Run one direction directly or through its captured graph.
int run_direction(nfft_batch* b, int dir, const void* in, void* out) {
  if (!b->graph_mode)
    return dir == 0 ? enqueue_forward(b, in, out, b->stream) : enqueue_adjoint(b, in, out, b->stream);
  if (!b->graph[dir] || b->graph_ptr[dir][0] != in || b->graph_ptr[dir][1] != out) {
    if (b->graph[dir]) cudaGraphExecDestroy(b->graph[dir]);
    b->graph[dir] = nullptr;
    B_CK(b, cudaStreamSynchronize(b->stream));
    B_CK(b, cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal));
    int s = dir == 0 ? enqueue_forward(b, in, out, b->capture_stream)
                     : enqueue_adjoint(b, in, out, b->capture_stream);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->capture_stream, &graph);
    if (s != NFFT_OK) {
      if (graph) cudaGraphDestroy(graph);
      return s;
    }
    B_CK(b, e);
    e = cudaGraphInstantiate(&b->graph[dir], graph, 0);
    cudaGraphDestroy(graph);
    B_CK(b, e);
    b->graph_ptr[dir][0] = in;
    b->graph_ptr[dir][1] = out;
  }
  B_CK(b, cudaGraphLaunch(b->graph[dir], b->stream));
  return NFFT_OK;
}

bool batch_ready(nfft_batch* b, int* st) {
  if (!b) {
    *st = NFFT_ERR_INVALID_ARG;
    return false;
  }
  *st = b->err;
  return b->err == NFFT_OK;
}

struct Guard {
  int prev = -1;
  explicit Guard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~Guard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// ---------------------------------------------------------------- autotune
std::mutex g_tune_mutex;
std::map<std::string, std::vector<int64_t>> g_tune_cache;

std::vector<std::vector<int64_t>> tile_candidates(int D, int K, int dtype) {
  std::vector<std::vector<int64_t>> c;
  const size_t cs = 2 * rsize(dtype);
  auto fits = [&](const std::vector<int64_t>& t) {
    size_t r = 1;
    for (int d = 0; d < D; ++d) r *= (size_t)(t[d] + K - 1);
    return r * cs <= 96 * 1024;
  };
  if (D == 1) {
    for (int64_t t : {64, 128, 256, 512, 1024, 2048}) c.push_back({t, 1, 1});
  } else if (D == 2) {
    for (int64_t t : {8, 16, 32, 64}) c.push_back({t, t, 1});
    c.push_back({16, 32, 1});
    c.push_back({32, 16, 1});
    c.push_back({9, 25, 1});
    c.push_back({8, 25, 1});
  } else {
    for (int64_t t : {4, 8, 16}) c.push_back({t, t, t});
    c.push_back({8, 8, 4});
    c.push_back({4, 8, 8});
  }
  std::vector<std::vector<int64_t>> ok;
  for (auto& t : c)
    if (fits(t)) ok.push_back(t);
  return ok;
}

}  // namespace

extern "C" {

int nfft_batch_destroy(nfft_batch* b) {
  if (!b) return NFFT_OK;
  Guard guard(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (int k = 0; k < 2; ++k)
    if (b->graph[k]) cudaGraphExecDestroy(b->graph[k]);
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  for (cudaStream_t side : b->fft_streams) cudaStreamDestroy(side);
  for (cudaEvent_t ev : b->join_ev) cudaEventDestroy(ev);
  if (b->fork_ev) cudaEventDestroy(b->fork_ev);
  for (auto& c : b->classes)
    if (c.ok) cufftDestroy(c.plan);
  void* bufs[] = {b->grid, b->beta64, b->beta32, b->poly, b->pad_blocks, b->crop_blocks, b->probs, b->cell, b->frac, b->perm, b->key, b->rank,
                  b->tile_count, b->tile_offset, b->set_items, b->set_nitems, b->items, b->n_items,
                  b->item_off};
  for (void* p : bufs)
    if (p) cudaFree(p);
  delete b;
  return NFFT_OK;
}

int nfft_batch_create(nfft_batch** out, int D, int B, const int64_t* N, const int32_t* set_of, int S,
                      const int64_t* M_set, double sigma, int m, int dtype, uint32_t flags, void* stream) {
  if (!out) return NFFT_ERR_INVALID_ARG;
  *out = nullptr;
  if (D < 1 || D > kMaxD || B < 1 || S < 1 || S > B || !N || !set_of || !M_set) return NFFT_ERR_INVALID_ARG;
  if (!(sigma > 1.0) || m < 1 || m > kMaxM) return NFFT_ERR_INVALID_ARG;
  if (m > 8) return NFFT_ERR_UNSUPPORTED;  // the batched kernels are built for m <= 8
  if (dtype != NFFT_C64 && dtype != NFFT_C128) return NFFT_ERR_INVALID_ARG;
  if (flags & ~(uint32_t)(NFFT_FLAG_CLOSED_SUPPORT | NFFT_FLAG_WIDE_WINDOW)) return NFFT_ERR_INVALID_ARG;
  if ((flags & NFFT_FLAG_CLOSED_SUPPORT) && (flags & NFFT_FLAG_WIDE_WINDOW)) return NFFT_ERR_INVALID_ARG;
  nfft_batch* b = new (std::nothrow) nfft_batch();
  if (!b) return NFFT_ERR_OOM;
  b->D = D;
  b->B = B;
  b->S = S;
  b->sigma = sigma;
  b->m = m;
  b->dtype = dtype;
  b->flags = flags;
  b->stream = (cudaStream_t)stream;
  const bool closed = (flags & NFFT_FLAG_CLOSED_SUPPORT) != 0;
  const bool wide = (flags & NFFT_FLAG_WIDE_WINDOW) != 0;
  b->K = (closed || wide) ? 2 * m + 2 : 2 * m;
  b->off = (closed || wide) ? -m : -m + 1;
  b->N.assign(N, N + (size_t)B * D);
  b->Nt.resize((size_t)B * D);
  b->set_of.assign(set_of, set_of + B);
  b->M_set.assign(M_set, M_set + S);
  int st = NFFT_OK;
  std::vector<int> set_first(S, -1);
  for (int s = 0; s < S && st == NFFT_OK; ++s)
    if (M_set[s] < 0 || M_set[s] >= ((int64_t)1 << 31)) st = NFFT_ERR_INVALID_ARG;
  for (int p = 0; p < B && st == NFFT_OK; ++p) {
    const int s = set_of[p];
    if (s < 0 || s >= S) {
      st = NFFT_ERR_INVALID_ARG;
      break;
    }
    int64_t tot = 1;
    for (int d = 0; d < D; ++d) {
      const int64_t n = N[(size_t)p * D + d];
      const int64_t nt = 2 * (int64_t)ceil(sigma * (double)n / 2.0 - 1e-12);
      if (n < 2 || n > ((int64_t)1 << 28) || nt <= 2 * m || nt > ((int64_t)1 << 30)) st = NFFT_ERR_INVALID_ARG;
      b->Nt[(size_t)p * D + d] = nt;
      tot *= nt;
    }
    if (set_first[s] < 0) {
      set_first[s] = p;
    } else {
      for (int d = 0; d < D; ++d)  // problems sharing a node set share its grid size
        if (N[(size_t)p * D + d] != N[(size_t)set_first[s] * D + d]) st = NFFT_ERR_INVALID_ARG;
    }
  }
  for (int s = 0; s < S && st == NFFT_OK; ++s)
    if (set_first[s] < 0) st = NFFT_ERR_INVALID_ARG;  // every node set is used
  if (st != NFFT_OK) {
    delete b;
    return st;
  }
  if (cudaGetDevice(&b->device) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return NFFT_ERR_CUDA;
  }
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);

  // size classes: grids of one class are contiguous
  std::vector<int> cls_of(B, -1);
  for (int p = 0; p < B; ++p) {
    std::vector<int64_t> nt(b->Nt.begin() + (size_t)p * D, b->Nt.begin() + (size_t)(p + 1) * D);
    int c = 0;
    for (; c < (int)b->classes.size(); ++c)
      if (b->classes[c].nt == nt) break;
    if (c == (int)b->classes.size()) {
      nfft_batch::SizeClass sc;
      sc.nt = nt;
      b->classes.push_back(sc);
    }
    cls_of[p] = c;
    b->classes[c].count++;
  }
  b->grid_off.assign(B, 0);
  int64_t goff = 0;
  for (int c = 0; c < (int)b->classes.size(); ++c) {
    b->classes[c].first_grid_off = goff;
    int64_t sz = 1;
    for (int64_t v : b->classes[c].nt) sz *= v;
    for (int p = 0; p < B; ++p)
      if (cls_of[p] == c) {
        b->grid_off[p] = goff;
        goff += sz;
      }
    if (sz > b->max_grid) b->max_grid = sz;
  }
  b->grid_total = goff;
  b->in_off.assign(B, 0);
  b->out_off.assign(B, 0);
  b->beta_off.assign(B, 0);
  for (int p = 0; p < B; ++p) {
    int64_t n = 1, sn = 0;
    for (int d = 0; d < D; ++d) {
      n *= N[(size_t)p * D + d];
      sn += N[(size_t)p * D + d];
    }
    b->in_off[p] = b->in_total;
    b->in_total += n;
    b->out_off[p] = b->out_total;
    b->out_total += M_set[set_of[p]];
    b->beta_off[p] = b->beta_total;
    b->beta_total += sn;
    if (n > b->max_n) b->max_n = n;
  }
  b->node_off.assign(S, 0);
  for (int s = 0; s < S; ++s) {
    b->node_off[s] = b->node_total;
    b->node_total += M_set[s];
    if (M_set[s] > b->max_set_nodes) b->max_set_nodes = M_set[s];
  }

  Guard guard(b->device);
  if (st == NFFT_OK) st = balloc(b, &b->grid, (size_t)b->grid_total * csize(dtype));
  if (st == NFFT_OK) st = balloc(b, &b->beta64, sizeof(double) * b->beta_total);
  if (st == NFFT_OK) st = balloc(b, &b->beta32, sizeof(float) * b->beta_total);
  const bool std_window = !(flags & (NFFT_FLAG_CLOSED_SUPPORT | NFFT_FLAG_WIDE_WINDOW));
  if (std_window) b->poly_per = (int64_t)D * b->K * (2 * m + 1);
  if (st == NFFT_OK && std_window) st = balloc(b, &b->poly, sizeof(float) * B * b->poly_per);
  if (st == NFFT_OK) st = balloc(b, &b->probs, sizeof(BatchProblem) * B);
  if (st == NFFT_OK) st = balloc(b, &b->cell, sizeof(int) * (size_t)(b->node_total * D));
  if (st == NFFT_OK) st = balloc(b, &b->frac, rsize(dtype) * (size_t)(b->node_total * D));
  if (st == NFFT_OK) st = balloc(b, &b->perm, sizeof(int) * (size_t)b->node_total);
  if (st == NFFT_OK) st = balloc(b, &b->key, sizeof(int) * (size_t)b->max_set_nodes);
  if (st == NFFT_OK) st = balloc(b, &b->rank, sizeof(int) * (size_t)b->max_set_nodes);
  if (st == NFFT_OK) st = balloc(b, &b->set_nitems, sizeof(int) * S);
  if (st == NFFT_OK) st = balloc(b, &b->n_items, sizeof(int));
  if (st == NFFT_OK) st = balloc(b, &b->item_off, sizeof(int) * (B + 1));
  if (st == NFFT_OK && cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
    st = NFFT_ERR_CUDA;
  for (auto& c : b->classes) {
    if (st != NFFT_OK) break;
    int n[kMaxD];
    int64_t sz = 1;
    for (int d = 0; d < D; ++d) {
      n[d] = (int)c.nt[d];
      sz *= c.nt[d];
    }
    cufftResult r = cufftPlanMany(&c.plan, D, n, nullptr, 1, (int)sz, nullptr, 1, (int)sz,
                                  dtype == NFFT_C128 ? CUFFT_Z2Z : CUFFT_C2C, c.count);
    if (r != CUFFT_SUCCESS) st = r == CUFFT_ALLOC_FAILED ? NFFT_ERR_OOM : NFFT_ERR_CUFFT;
    else c.ok = true;
  }
  // side streams for the class FFTs: each class, largest first, goes to the
  // stream with the fewest grid points so far
  const int n_side = std::min<int>(kFftSideStreams, (int)b->classes.size());
  if (st == NFFT_OK && n_side > 1) {
    std::vector<int> order(b->classes.size());
    std::vector<int64_t> load(n_side, 0);
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    auto points = [&](int i) {
      int64_t sz = b->classes[i].count;
      for (int64_t v : b->classes[i].nt) sz *= v;
      return sz;
    };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return points(x) > points(y); });
    for (int i : order) {
      int k = 0;
      for (int j = 1; j < n_side; ++j)
        if (load[j] < load[k]) k = j;
      b->classes[i].side = k;
      load[k] += points(i);
    }
    for (int k = 0; k < n_side && st == NFFT_OK; ++k) {
      cudaStream_t side = nullptr;
      cudaEvent_t ev = nullptr;
      if (cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking) != cudaSuccess) st = NFFT_ERR_CUDA;
      else b->fft_streams.push_back(side);
      if (st == NFFT_OK && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) st = NFFT_ERR_CUDA;
      else if (st == NFFT_OK) b->join_ev.push_back(ev);
    }
    if (st == NFFT_OK && cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming) != cudaSuccess)
      st = NFFT_ERR_CUDA;
  }
  // block ranges of the batched correction kernels: about four grid-stride
  // iterations per thread for every problem (complex pairs for deconv_pad)
  if (st == NFFT_OK) {
    constexpr int64_t per_block = 4 * kBatchDeconvThreads;
    std::vector<int> pad(B + 1, 0), crop(B + 1, 0);
    for (int p = 0; p < B; ++p) {
      int64_t pairs = 1, n = 1;
      for (int d = 0; d < D; ++d) {
        pairs *= b->Nt[(size_t)p * D + d];
        n *= N[(size_t)p * D + d];
      }
      pairs /= 2;
      const int64_t np = (pairs + per_block - 1) / per_block, nc = (n + per_block - 1) / per_block;
      if ((int64_t)pad[p] + np > INT32_MAX || (int64_t)crop[p] + nc > INT32_MAX) {
        st = NFFT_ERR_INVALID_ARG;
        break;
      }
      pad[p + 1] = pad[p] + (int)np;
      crop[p + 1] = crop[p] + (int)nc;
    }
    if (st == NFFT_OK) st = balloc(b, &b->pad_blocks, sizeof(int) * (B + 1));
    if (st == NFFT_OK) st = balloc(b, &b->crop_blocks, sizeof(int) * (B + 1));
    if (st == NFFT_OK) {
      b->n_pad_blocks = pad[B];
      b->n_crop_blocks = crop[B];
      st = bst(b, cudaMemcpy(b->pad_blocks, pad.data(), sizeof(int) * (B + 1), cudaMemcpyHostToDevice));
      if (st == NFFT_OK)
        st = bst(b, cudaMemcpy(b->crop_blocks, crop.data(), sizeof(int) * (B + 1), cudaMemcpyHostToDevice));
    }
  }
  // deconvolution vectors, one set per problem
  for (int p = 0; p < B && st == NFFT_OK; ++p) {
    int Ni[kMaxD], Nti[kMaxD];
    double bb[kMaxD];
    for (int d = 0; d < D; ++d) {
      Ni[d] = (int)N[(size_t)p * D + d];
      Nti[d] = (int)b->Nt[(size_t)p * D + d];
      bb[d] = M_PI * (2.0 - (double)Ni[d] / (double)Nti[d]);
    }
    st = bst(b, launch_build_beta(D, Ni, Nti, m, bb, b->beta64 + b->beta_off[p], b->beta32 + b->beta_off[p],
                                  b->stream));
    if (st == NFFT_OK && b->poly) {
      PolyArgs pa{};
      pa.D = D;
      pa.K = b->K;
      pa.off = b->off;
      pa.deg = 2 * m;
      pa.m = m;
      for (int d = 0; d < D; ++d) pa.b[d] = bb[d];
      st = bst(b, launch_build_poly(pa, b->poly + p * b->poly_per, b->stream));
    }
  }
  if (st == NFFT_OK) {
    default_batch_tile(b, b->T);
    st = configure(b);
  }
  if (st != NFFT_OK) {
    nfft_batch_destroy(b);
    return st;
  }
  *out = b;
  return NFFT_OK;
}

int nfft_batch_set_nodes(nfft_batch* b, const void* k, int k_is_fp64) {
  int st;
  if (!batch_ready(b, &st)) return st;
  if (!k) return NFFT_ERR_INVALID_ARG;
  Guard guard(b->device);
  return batch_set_nodes_stream(b, k, k_is_fp64 ? 1 : 0, b->stream);
}

int nfft_batch_forward(nfft_batch* b, const void* f, void* fhat) {
  int st;
  if (!batch_ready(b, &st)) return st;
  if (!b->has_nodes) return NFFT_ERR_NO_NODES;
  if (!f || !fhat) return NFFT_ERR_INVALID_ARG;
  Guard guard(b->device);
  return run_direction(b, 0, f, fhat);
}

int nfft_batch_adjoint(nfft_batch* b, const void* fhat, void* y) {
  int st;
  if (!batch_ready(b, &st)) return st;
  if (!b->has_nodes) return NFFT_ERR_NO_NODES;
  if (!fhat || !y) return NFFT_ERR_INVALID_ARG;
  Guard guard(b->device);
  return run_direction(b, 1, fhat, y);
}

int nfft_batch_set_graph(nfft_batch* b, int enable) {
  int st;
  if (!batch_ready(b, &st)) return st;
  b->graph_mode = enable != 0;
  return NFFT_OK;
}

int nfft_batch_set_tile(nfft_batch* b, const int64_t* tile3) {
  int st;
  if (!batch_ready(b, &st)) return st;
  if (!tile3) return NFFT_ERR_INVALID_ARG;
  int64_t T[kMaxD] = {1, 1, 1};
  for (int d = 0; d < b->D; ++d) {
    if (tile3[d] < 1) return NFFT_ERR_INVALID_ARG;
    T[d] = tile3[d];
  }
  if (max_region_bytes(b, T) > 200 * 1024) return NFFT_ERR_INVALID_ARG;
  Guard guard(b->device);
  B_CK(b, cudaStreamSynchronize(b->stream));
  for (int d = 0; d < kMaxD; ++d) b->T[d] = T[d];
  return configure(b);
}

int nfft_batch_info(nfft_batch* b, int64_t* tile3, int64_t* n_items, int64_t* n_fft_classes) {
  if (!b) return NFFT_ERR_INVALID_ARG;
  for (int d = 0; d < kMaxD; ++d)
    if (tile3) tile3[d] = d < b->D ? b->T[d] : 1;
  if (n_fft_classes) *n_fft_classes = (int64_t)b->classes.size();
  if (n_items) {
    *n_items = 0;
    if (b->has_nodes) {
      Guard guard(b->device);
      int h = 0;
      B_CK(b, cudaMemcpyAsync(&h, b->n_items, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
      B_CK(b, cudaStreamSynchronize(b->stream));
      *n_items = h;
    }
  }
  return b->err;
}

int nfft_batch_autotune(nfft_batch* b, const void* k, int k_is_fp64, int64_t* chosen3) {
  int st;
  if (!batch_ready(b, &st)) return st;
  if (!k) return NFFT_ERR_INVALID_ARG;
  Guard guard(b->device);
  std::string key = "batch:" + std::to_string(b->device) + ":" + std::to_string(b->D) + ":" +
                    std::to_string(b->m) + ":" + std::to_string(b->dtype) + ":" + std::to_string(b->B);
  for (int64_t v : b->N) key += "," + std::to_string(v);
  for (int64_t v : b->M_set) key += ";" + std::to_string(v);
  std::vector<int64_t> best;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) best = it->second;
  }
  if (best.empty()) {
    void *f = nullptr, *fh = nullptr;
    st = balloc(b, &f, (size_t)b->in_total * csize(b->dtype));
    if (st == NFFT_OK) st = balloc(b, &fh, (size_t)b->out_total * csize(b->dtype));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (st == NFFT_OK) {
      cudaMemsetAsync(f, 0, (size_t)b->in_total * csize(b->dtype), b->stream);
      cudaMemsetAsync(fh, 0, (size_t)b->out_total * csize(b->dtype), b->stream);
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
    }
    float best_ms = 1e30f;
    const bool gm = b->graph_mode;
    b->graph_mode = false;
    for (auto& t : tile_candidates(b->D, b->K, b->dtype)) {
      if (st != NFFT_OK) break;
      for (int d = 0; d < kMaxD; ++d) b->T[d] = t[d];
      if ((st = configure(b)) != NFFT_OK) break;
      if ((st = batch_set_nodes_stream(b, k, k_is_fp64, b->stream)) != NFFT_OK) break;
      float ms = 0.f;
      for (int rep = 0; rep < 3 && st == NFFT_OK; ++rep) {
        cudaEventRecord(e0, b->stream);
        st = enqueue_forward(b, f, fh, b->stream);
        if (st == NFFT_OK) st = enqueue_adjoint(b, fh, f, b->stream);
        cudaEventRecord(e1, b->stream);
        cudaEventSynchronize(e1);
        float t_ms = 0.f;
        cudaEventElapsedTime(&t_ms, e0, e1);
        if (rep > 0) ms += t_ms;  // first repeat warms up
      }
      if (st == NFFT_OK && ms < best_ms) {
        best_ms = ms;
        best = t;
      }
    }
    b->graph_mode = gm;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (f) cudaFree(f);
    if (fh) cudaFree(fh);
    if (st != NFFT_OK) return st;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = best;
  }
  for (int d = 0; d < kMaxD; ++d) b->T[d] = best[d];
  if ((st = configure(b)) != NFFT_OK) return st;
  if ((st = batch_set_nodes_stream(b, k, k_is_fp64, b->stream)) != NFFT_OK) return st;
  if (chosen3)
    for (int d = 0; d < kMaxD; ++d) chosen3[d] = best[d];
  return NFFT_OK;
}

}  // extern "C"
