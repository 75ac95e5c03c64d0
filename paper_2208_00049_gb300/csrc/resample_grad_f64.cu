// grad kernels, FP64 (complex128) plans.
#include "resample.cuh"
namespace nfftgb {
template void* pick_grad<double>(int, int);
}  // namespace nfftgb
