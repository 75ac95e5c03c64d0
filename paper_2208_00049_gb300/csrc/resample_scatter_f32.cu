// scatter kernels, FP32 (complex64) plans.
#include "resample.cuh"
namespace nfftgb {
template void* pick_scatter<float>(int, int, int);
}  // namespace nfftgb
