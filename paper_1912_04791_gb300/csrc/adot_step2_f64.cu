// float64 instantiation of the second-order time step.
#include "adot_step2_impl.cuh"

namespace adot {

cudaError_t launch_step2_f64(const StepParams& p, int law, StepVariant v, StateF64 in,
                             StateF64 out, int slot, cudaStream_t s) {
  return launch_step2_impl<double>(p, law, v, in, out, slot, s);
}

}  // namespace adot
