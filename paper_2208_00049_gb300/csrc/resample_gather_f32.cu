// gather kernels, FP32 (complex64) plans.
#include "resample.cuh"
namespace nfftgb {
template void* pick_gather<float>(int, int);
}  // namespace nfftgb
