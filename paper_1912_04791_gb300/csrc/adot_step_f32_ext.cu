// float32 (float-float state) instantiation of the time-step kernels with the
// friction source and the sediment feed compiled in (a translation unit of its
// own, so that it compiles beside the plain kernels).
#include "adot_step_impl.cuh"

namespace adot {

cudaError_t launch_step_f32_ext(const StepParams& p, int law, StepVariant v, StateF32 in,
                                StateF32 out, int slot, cudaStream_t s) {
  return launch_step_impl<float, true>(p, law, v, in, out, slot, s);
}

cudaError_t launch_step_sur_f32_ext(const StepParams& p, StateF32 in, StateF32 out, int slot,
                                    cudaStream_t s) {
  if (p.ctl == nullptr || p.absA == nullptr || p.n < 1) return cudaErrorInvalidValue;
  const int64_t g = (p.n + 1 + 254) / 255;
  if (g > 0x7fffffffLL) return cudaErrorInvalidValue;
  k_step<float, LAW_GRASS, 256, 64, true, true><<<(unsigned)g, 256, 0, s>>>(p, in, out, slot);
  return cudaGetLastError();
}

}  // namespace adot
