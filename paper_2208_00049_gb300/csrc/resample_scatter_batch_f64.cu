// batched scatter kernels, f64 plans.
#include "resample.cuh"
namespace nfftgb {
template void* pick_scatter_batch<double>(int, int);
}  // namespace nfftgb
