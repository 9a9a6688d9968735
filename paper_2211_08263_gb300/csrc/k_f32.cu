// FP32 instantiation of the pass kernels (inner PCG of the mixed-precision solve).
#include "passes_impl.cuh"

namespace wfft {
WFFT_INSTANTIATE(float)
}  // namespace wfft
