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

// Pipelined fused kernel.  Compile-time r for the paper convention at r in
// {256} with the default staging depth (2); the alternative depths (1: four
// resident CTAs per SM, 3) have r = 256; any other r, and the transpose convention, use the runtime
// mask.  Descriptor-table batches use the default depth.
template <class P, typename InT, bool TABLE>
static int pipe_n32(int conv, const PipeArgs& pa, int r, int num_sms, PipeTuning t, void* stream) {
  const int stages = t.stages == 0 ? 2 : t.stages;
  if (conv == 0) {
    if constexpr (TABLE) {
      return pipe_launch_r<32, P, 0, InT, 2, true, 256>(pa, r, num_sms, t.ctas_per_sm, stream);
    } else {
      if (stages == 1) return pipe_launch_r<32, P, 0, InT, 1, false, 256>(pa, r, num_sms, t.ctas_per_sm, stream);
      if (stages == 2) return pipe_launch_r<32, P, 0, InT, 2, false, 256>(pa, r, num_sms, t.ctas_per_sm, stream);
      return pipe_launch_r<32, P, 0, InT, 3, false, 256>(pa, r, num_sms, t.ctas_per_sm, stream);
    }
  }
  return pipe_launch_r<32, P, 1, InT, 2, TABLE>(pa, r, num_sms, t.ctas_per_sm, stream);
}

int pipe_launch_n32(int variant, int conv, int dtype, const PipeArgs& pa, int r, int num_sms, PipeTuning t,
                    void* stream) {
  const bool table = pa.unit_map != nullptr;
  if (variant == 1) {
    if (dtype == 0)
      return table ? pipe_n32<ParamsTilde, uint8_t, true>(conv, pa, r, num_sms, t, stream)
                   : pipe_n32<ParamsTilde, uint8_t, false>(conv, pa, r, num_sms, t, stream);
    return table ? pipe_n32<ParamsTilde, int16_t, true>(conv, pa, r, num_sms, t, stream)
                 : pipe_n32<ParamsTilde, int16_t, false>(conv, pa, r, num_sms, t, stream);
  }
  if (dtype == 0)
    return table ? pipe_n32<ParamsHat, uint8_t, true>(conv, pa, r, num_sms, t, stream)
                 : pipe_n32<ParamsHat, uint8_t, false>(conv, pa, r, num_sms, t, stream);
  return table ? pipe_n32<ParamsHat, int16_t, true>(conv, pa, r, num_sms, t, stream)
               : pipe_n32<ParamsHat, int16_t, false>(conv, pa, r, num_sms, t, stream);
}

}  // namespace cdct
