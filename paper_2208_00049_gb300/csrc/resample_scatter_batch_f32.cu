// batched scatter kernels, f32 plans.
#include "resample.cuh"
namespace nfftgb {
template void* pick_scatter_batch<float>(int, int);
}  // namespace nfftgb
