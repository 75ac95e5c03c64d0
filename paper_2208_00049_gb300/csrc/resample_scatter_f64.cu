// scatter kernels, FP64 (complex128) plans.
#include "resample.cuh"
namespace nfftgb {
template void* pick_scatter<double>(int, int, int);
}  // namespace nfftgb
