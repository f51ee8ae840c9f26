// Instantiations of the integer block kernels for N = 8.
#include "block_kernels.cuh"
#include "pipe_kernels.cuh"

namespace cdct {

KernelSet kernels_n8(int variant, int conv, int dtype) {
  if (variant == 1) {
    return conv == 0 ? kernel_set_int<8, ParamsTilde, 0>(dtype) : kernel_set_int<8, ParamsTilde, 1>(dtype);
  }
  return conv == 0 ? kernel_set_int<8, ParamsHat, 0>(dtype) : kernel_set_int<8, ParamsHat, 1>(dtype);
}

// Pipelined fused kernel.  Compile-time r for the paper convention at r in
// {1, 6, 10, 16, 28, 64} with the default staging depth (3); the alternative depth (2)
// has r = 16; any other r, and the transpose convention, use the runtime
// mask.  Descriptor-table batches use the default depth.
template <class P, typename InT, bool TABLE>
static int pipe_n8(int conv, const PipeArgs& pa, int r, int num_sms, PipeTuning t, void* stream) {
  const int stages = t.stages == 0 ? 3 : t.stages;
  if (conv == 0) {
    if constexpr (TABLE) {
      return pipe_launch_r<8, P, 0, InT, 3, true, 16>(pa, r, num_sms, t.ctas_per_sm, stream);
    } else {
      if (stages == 3) return pipe_launch_r<8, P, 0, InT, 3, false, 1, 6, 10, 16, 28, 64>(pa, r, num_sms, t.ctas_per_sm, stream);
      return pipe_launch_r<8, P, 0, InT, 2, false, 16>(pa, r, num_sms, t.ctas_per_sm, stream);
    }
  }
  return pipe_launch_r<8, P, 1, InT, 3, TABLE>(pa, r, num_sms, t.ctas_per_sm, stream);
}

int pipe_launch_n8(int variant, int conv, int dtype, const PipeArgs& pa, int r, int num_sms, PipeTuning t,
                    void* stream) {
  const bool table = pa.unit_map != nullptr;
  if (variant == 1) {
    if (dtype == 0)
      return table ? pipe_n8<ParamsTilde, uint8_t, true>(conv, pa, r, num_sms, t, stream)
                   : pipe_n8<ParamsTilde, uint8_t, false>(conv, pa, r, num_sms, t, stream);
    return table ? pipe_n8<ParamsTilde, int16_t, true>(conv, pa, r, num_sms, t, stream)
                 : pipe_n8<ParamsTilde, int16_t, false>(conv, pa, r, num_sms, t, stream);
  }
  if (dtype == 0)
    return table ? pipe_n8<ParamsHat, uint8_t, true>(conv, pa, r, num_sms, t, stream)
                 : pipe_n8<ParamsHat, uint8_t, false>(conv, pa, r, num_sms, t, stream);
  return table ? pipe_n8<ParamsHat, int16_t, true>(conv, pa, r, num_sms, t, stream)
               : pipe_n8<ParamsHat, int16_t, false>(conv, pa, r, num_sms, t, stream);
}

}  // namespace cdct
