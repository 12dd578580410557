// float64 instantiation of the time-step kernels with the friction source and
// the sediment feed compiled in.
#include "adot_step_impl.cuh"

namespace adot {

cudaError_t launch_step_f64_ext(const StepParams& p, int law, StepVariant v, StateF64 in,
                                StateF64 out, int slot, cudaStream_t s) {
  return launch_step_impl<double, true>(p, law, v, in, out, slot, s);
}

}  // namespace adot
