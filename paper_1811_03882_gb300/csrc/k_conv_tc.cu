// k_conv_tc.cu — tensor-core implicit-GEMM convolution (tcgen05 + TMA).
#include "common.cuh"
#include "kernels.h"

namespace dn {

cudaError_t conv_tc(const ConvLaunch&, int, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace dn
