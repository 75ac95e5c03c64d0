// gather kernels, FP64 (complex128) plans.
#include "resample.cuh"
namespace nfftgb {
template void* pick_gather<double>(int, int);
}  // namespace nfftgb
