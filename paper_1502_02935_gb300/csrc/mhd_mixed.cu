// mhd_mixed.cu -- the mixed instantiation: FP32 bulk arithmetic, FP64 pressure recovery
// and FP64 accumulation of the conserved state.
#include "mhd_kernels.cuh"

namespace mhd {
Backend backend_mixed() { return make_backend<float>(); }
}  // namespace mhd
