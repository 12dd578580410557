// float32 (float-float state) instantiation of the second-order time step.
#include "adot_step2_impl.cuh"

namespace adot {

cudaError_t launch_step2_f32(const StepParams& p, int law, StepVariant v, StateF32 in,
                             StateF32 out, int slot, cudaStream_t s) {
  return launch_step2_impl<float>(p, law, v, in, out, slot, s);
}

}  // namespace adot
