// FP64 grouped-launch instantiation of the pass kernels (several instances of
// uneven sizes per launch).
#include "passes_impl.cuh"

namespace wfft {
WFFT_INSTANTIATE_BATCH(double)
}  // namespace wfft
