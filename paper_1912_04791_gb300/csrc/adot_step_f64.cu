// float64 instantiation of the fused time-step kernel.
#include "adot_step_impl.cuh"

namespace adot {

cudaError_t launch_step_f64(const StepParams& p, int law, StepVariant v, StateF64 in, StateF64 out,
                            int slot, cudaStream_t s) {
  if (p.scheme == 1) return launch_step_price_f64(p, law, v, in, out, slot, s);
  if (p.order == 2) return launch_step2_f64(p, law, v, in, out, slot, s);
  if (step_needs_ext(p)) return launch_step_f64_ext(p, law, v, in, out, slot, s);
  return launch_step_impl<double, false>(p, law, v, in, out, slot, s);
}

cudaError_t launch_rho_f64(const StepParams& p, int law, StateF64 st, int slot, cudaStream_t s) {
  return launch_rho_impl<double>(p, law, st, slot, s);
}

}  // namespace adot
