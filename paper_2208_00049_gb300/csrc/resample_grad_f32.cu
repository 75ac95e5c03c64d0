// grad kernels, FP32 (complex64) plans.
#include "resample.cuh"
namespace nfftgb {
template void* pick_grad<float>(int, int);
}  // namespace nfftgb
