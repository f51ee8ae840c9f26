// Instantiations of the integer block kernels for N = 32.
#include "block_kernels.cuh"
#include "pipe_kernels.cuh"

namespace cdct {

KernelSet kernels_n32(int variant, int conv, int dtype) {
  if (variant == 1) {
    return conv == 0 ? kernel_set_int<32, ParamsTilde, 0>(dtype) : kernel_set_int<32, ParamsTilde, 1>(dtype);
  }
  return conv == 0 ? kernel_set_int<32, ParamsHat, 0>(dtype) : kernel_set_int<32, ParamsHat, 1>(dtype);
}

// Pipelined fused kernel: compile-time r for the paper convention at
// r in {256}; any other r (and the transpose convention) uses the
// runtime mask.
template <class P, typename InT>
static int pipe_n32(int conv, const PipeArgs& pa, int r, int num_sms, void* stream) {
  if (conv == 0) return pipe_launch_r<32, P, 0, InT, 2, 256>(pa, r, num_sms, stream);
  return pipe_launch_r<32, P, 1, InT, 2>(pa, r, num_sms, stream);
}

int pipe_launch_n32(int variant, int conv, int dtype, const PipeArgs& pa, int r, int num_sms, void* stream) {
  if (variant == 1) {
    return dtype == 0 ? pipe_n32<ParamsTilde, uint8_t>(conv, pa, r, num_sms, stream)
                      : pipe_n32<ParamsTilde, int16_t>(conv, pa, r, num_sms, stream);
  }
  return dtype == 0 ? pipe_n32<ParamsHat, uint8_t>(conv, pa, r, num_sms, stream)
                    : pipe_n32<ParamsHat, int16_t>(conv, pa, r, num_sms, stream);
}

}  // namespace cdct
