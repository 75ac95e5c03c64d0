// batched gather kernels, f32 plans.
#include "resample.cuh"
namespace nfftgb {
template void* pick_gather_batch<float>(int, int);
}  // namespace nfftgb
