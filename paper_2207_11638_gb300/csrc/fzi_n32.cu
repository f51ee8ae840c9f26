// Instantiations of the integer block kernels for N = 32.
#include "block_kernels.cuh"

namespace cdct {

KernelSet kernels_n32(int variant, int conv, int dtype) {
  if (variant == 1) {
    return conv == 0 ? kernel_set_int<32, ParamsTilde, 0>(dtype) : kernel_set_int<32, ParamsTilde, 1>(dtype);
  }
  return conv == 0 ? kernel_set_int<32, ParamsHat, 0>(dtype) : kernel_set_int<32, ParamsHat, 1>(dtype);
}

}  // namespace cdct
