// Instantiations of the integer block kernels for N = 16.
#include "block_kernels.cuh"

namespace cdct {

KernelSet kernels_n16(int variant, int conv, int dtype) {
  if (variant == 1) {
    return conv == 0 ? kernel_set_int<16, ParamsTilde, 0>(dtype) : kernel_set_int<16, ParamsTilde, 1>(dtype);
  }
  return conv == 0 ? kernel_set_int<16, ParamsHat, 0>(dtype) : kernel_set_int<16, ParamsHat, 1>(dtype);
}

}  // namespace cdct
