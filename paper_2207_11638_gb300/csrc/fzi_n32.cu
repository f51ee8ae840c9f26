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

// Pipelined fused kernel.  The paper convention at r = 256 (= N^2 / 4) without
// kept-coefficient output runs the separable packed body (stage depth 1 by
// default, or 2); other r, the transpose convention and kept output run the
// fold + core body: compile-time r = 256 at depths 1-3 (default 2), the
// runtime mask otherwise.  Descriptor-table batches use the default depths.
template <class P, typename InT, bool TABLE>
static int pipe_n32(int conv, const PipeArgs& pa, int r, int num_sms, PipeTuning t, void* stream) {
  int rc = 0;
  if (TABLE || t.stages != 2) {
    if (pipe_try_sep<32, P, InT, 256, 1, TABLE>(pa, conv, r, num_sms, t.ctas_per_sm, stream, rc)) return rc;
  } else {
    if (pipe_try_sep<32, P, InT, 256, 2, false>(pa, conv, r, num_sms, t.ctas_per_sm, stream, rc)) return rc;
  }
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
