// batched gather kernels, f64 plans.
#include "resample.cuh"
namespace nfftgb {
template void* pick_gather_batch<double>(int, int);
}  // namespace nfftgb
