// mhd_fp64.cu -- the plain FP64 instantiation of the step kernels.
#include "mhd_kernels.cuh"

namespace mhd {
Backend backend_fp64() { return make_backend<double>(); }
}  // namespace mhd
