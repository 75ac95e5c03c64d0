// nfft_spread_noalloc: adjoint resampling (spreading) of up to
// NFFT_NOALLOC_MAX_NODES nodes onto a caller-provided oversampled grid with
// no device allocation at all.
//
// Some callers cannot call cudaMalloc: code running under another
// framework's allocator (a raw cudaMalloc beside a caching allocator
// fragments memory and can implicitly synchronise the device), latency-
// critical loops that cannot take that implicit synchronisation, and services
// with a fixed memory budget that must be reserved when the library is
// loaded.  For them the bin-sort scratch (node keys, ranks, sorted cells and
// fractions, the permutation, per-tile counts and offsets, work items) lives
// in one file-scope __device__ array of fixed size, which every GPU that
// loads this library holds until the process exits.
//
// The array is shared by every call on a device and keeps the last call's
// contents; everything that must start at zero (the per-tile counters) is
// cleared by each call on its stream.  Calls whose work overlaps on the GPU
// (different streams, or host threads racing on one device) race on the
// array and must be serialised by the caller.
//
// Host code cannot use the array's name as a device address: the first call
// on a device looks the address up with cudaGetSymbolAddress (with that
// device current) and caches it, so that first call should be made before
// any stream capture begins.  The cached address belongs to the device's
// current context: after cudaDeviceReset (or anything else that destroys and
// recreates the primary context) the array may live elsewhere, so this entry
// point must not be used across a device reset.
#include <math.h>

#include <mutex>

#include "nfft_internal.cuh"

using namespace nfftgb;

namespace {

constexpr int64_t kMaxNodes = NFFT_NOALLOC_MAX_NODES;
constexpr int64_t kMaxTiles = NFFT_NOALLOC_MAX_TILES;
constexpr int kCmax = 128;
constexpr int64_t kMaxItems = kMaxTiles + kMaxNodes / kCmax + 1;
constexpr int kMaxDevices = 64;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffKey = 0;
constexpr size_t kOffRank = align256(kOffKey + 4 * kMaxNodes);
constexpr size_t kOffCell = align256(kOffRank + 4 * kMaxNodes);
constexpr size_t kOffFrac = align256(kOffCell + 4 * kMaxD * kMaxNodes);
constexpr size_t kOffPerm = align256(kOffFrac + 4 * kMaxD * kMaxNodes);
constexpr size_t kOffTileCount = align256(kOffPerm + 4 * kMaxNodes);
constexpr size_t kOffTileOffset = align256(kOffTileCount + 4 * kMaxTiles);
constexpr size_t kOffItems = align256(kOffTileOffset + 4 * kMaxTiles);
constexpr size_t kOffNItems = align256(kOffItems + 16 * kMaxItems);
constexpr size_t kScratchBytes = align256(kOffNItems + 4);

__device__ __align__(256) unsigned char g_spread_scratch[kScratchBytes];

std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array for the current device (looked up once
// per device; the host-side symbol is not a device address).
int scratch_address(int device, unsigned char** out) {
  if (device < 0 || device >= kMaxDevices) return NFFT_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[device]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_spread_scratch);
    if (e != cudaSuccess || !ptr) {
      cudaGetLastError();
      return NFFT_ERR_CUDA;
    }
    g_scratch_addr[device] = ptr;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[device]);
  return NFFT_OK;
}

// Device memory (*dev = its device) or managed memory (*dev = -1); false for
// host memory and for pointers CUDA does not know.
bool on_device(const void* ptr, int* dev) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  *dev = attr.type == cudaMemoryTypeDevice ? attr.device : -1;
  return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int nfft_spread_noalloc(int D, const int64_t* N, double sigma, int m, int64_t M,
                                   const double* k, const void* fhat, void* grid, void* stream) {
  if (D < 1 || D > kMaxD || !N || !grid) return NFFT_ERR_INVALID_ARG;
  if (!(sigma > 1.0) || m < 1 || m > kMaxM || M < 0) return NFFT_ERR_INVALID_ARG;
  if (M > 0 && (!k || !fhat)) return NFFT_ERR_INVALID_ARG;
  if (M > kMaxNodes) return NFFT_ERR_UNSUPPORTED;  // beyond the static scratch

  Geometry g{};
  g.D = D;
  g.K = 2 * m;
  g.off = -m + 1;
  g.closed = 0;
  g.M = (int)M;
  g.m = (double)m;
  int64_t grid_elems = 1, n_tiles = 1;
  const int tile_default = D == 3 ? 8 : (D == 2 ? 32 : 256);
  for (int d = 0; d < D; ++d) {
    if (N[d] < 2 || N[d] > ((int64_t)1 << 28)) return NFFT_ERR_INVALID_ARG;
    const int64_t nt = 2 * (int64_t)ceil(sigma * (double)N[d] / 2.0 - 1e-12);
    if (nt <= 2 * m || nt > ((int64_t)1 << 30)) return NFFT_ERR_INVALID_ARG;
    int64_t t = tile_default;
    if (t > nt - g.K + 1) t = nt - g.K + 1;
    if (t < 1) t = 1;
    g.Nt[d] = (int)nt;
    g.T[d] = (int)t;
    g.ntile[d] = (int)((nt + t - 1) / t);
    g.L[d] = (int)t + g.K - 1;
    g.b[d] = M_PI * (2.0 - (double)N[d] / (double)nt);
    g.norm[d] = (double)m / sinh(g.b[d] * (double)m);
    grid_elems *= nt;
    n_tiles *= g.ntile[d];
    if (n_tiles > kMaxTiles) return NFFT_ERR_UNSUPPORTED;  // beyond the static scratch
  }
  int dev_k = -1, dev_f = -1, dev_g = -1;
  if (M > 0 && (!on_device(k, &dev_k) || !on_device(fhat, &dev_f))) return NFFT_ERR_INVALID_ARG;
  if (!on_device(grid, &dev_g)) return NFFT_ERR_INVALID_ARG;

  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) {
    cudaGetLastError();
    return NFFT_ERR_CUDA;
  }
  // the kernels run on the current device: memory of another GPU is rejected
  for (int dv : {dev_k, dev_f, dev_g})
    if (dv >= 0 && dv != device) return NFFT_ERR_INVALID_ARG;
  unsigned char* base = nullptr;
  int st = scratch_address(device, &base);
  if (st != NFFT_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;

  int* key = reinterpret_cast<int*>(base + kOffKey);
  int* rank = reinterpret_cast<int*>(base + kOffRank);
  int* cell = reinterpret_cast<int*>(base + kOffCell);
  float* frac = reinterpret_cast<float*>(base + kOffFrac);
  int* perm = reinterpret_cast<int*>(base + kOffPerm);
  int* tile_count = reinterpret_cast<int*>(base + kOffTileCount);
  int* tile_offset = reinterpret_cast<int*>(base + kOffTileOffset);
  int4* items = reinterpret_cast<int4*>(base + kOffItems);
  int* n_items = reinterpret_cast<int*>(base + kOffNItems);

  SortArgs a{};
  a.D = D;
  a.M = (int)M;
  for (int d = 0; d < D; ++d) {
    a.Nt[d] = g.Nt[d];
    a.T[d] = g.T[d];
    a.ntile[d] = g.ntile[d];
  }
  a.n_tiles = (int)n_tiles;
  a.cmax = kCmax;
  a.max_items = (int)kMaxItems;

  // the tile counters are cleared inside launch_node_count; the grid here
  if (launch_node_count(a, k, 1, tile_count, key, rank, s) != cudaSuccess) return NFFT_ERR_CUDA;
  if (launch_tile_scan(a, tile_count, tile_offset, items, n_items, s) != cudaSuccess)
    return NFFT_ERR_CUDA;
  if (launch_node_place(a, k, 1, key, rank, tile_offset, cell, frac, 0, perm, s) != cudaSuccess)
    return NFFT_ERR_CUDA;
  if (cudaMemsetAsync(grid, 0, (size_t)grid_elems * sizeof(float2), s) != cudaSuccess) {
    cudaGetLastError();
    return NFFT_ERR_CUDA;
  }
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const int per_sm = resample_ctas_per_sm<float>(g, 1);
  if (per_sm <= 0) return NFFT_ERR_UNSUPPORTED;
  NodeArrays na;
  na.cell = cell;
  na.frac = frac;
  na.perm = perm;
  na.items = items;
  na.n_items = n_items;
  if (launch_scatter<float>(g, grid, na, fhat, 0, per_sm * sms, s) != cudaSuccess) {
    cudaGetLastError();
    return NFFT_ERR_CUDA;
  }
  return NFFT_OK;
}
