// float32 (float-float state) instantiation of the fused time-step kernel.
#include "adot_step_impl.cuh"

namespace adot {

bool step_block_supported(int block) { return block == 128 || block == 256 || block == 512; }

bool step_variant_supported(StepVariant v) {
  for (int i = 0; i < kNumStepVariants; ++i)
    if (kStepVariants[i].block == v.block && kStepVariants[i].reg_cap == v.reg_cap &&
        kStepVariants[i].warp_tiles == v.warp_tiles)
      return true;
  return false;
}

cudaError_t launch_step_f32(const StepParams& p, int law, StepVariant v, StateF32 in, StateF32 out,
                            int slot, cudaStream_t s) {
  if (p.scheme == 1) return launch_step_price_f32(p, law, v, in, out, slot, s);
  if (p.order == 2) return launch_step2_f32(p, law, v, in, out, slot, s);
  if (step_needs_ext(p)) return launch_step_f32_ext(p, law, v, in, out, slot, s);
  return launch_step_impl<float, false>(p, law, v, in, out, slot, s);
}

cudaError_t launch_step_sur_f32(const StepParams& p, StateF32 in, StateF32 out, int slot,
                                cudaStream_t s) {
  if (p.ctl == nullptr || p.absA == nullptr || p.n < 1) return cudaErrorInvalidValue;
  if (step_needs_ext(p)) return launch_step_sur_f32_ext(p, in, out, slot, s);
  const int64_t g = (p.n + 1 + 254) / 255;
  if (g > 0x7fffffffLL) return cudaErrorInvalidValue;
  k_step<float, LAW_GRASS, 256, 64, true><<<(unsigned)g, 256, 0, s>>>(p, in, out, slot);
  return cudaGetLastError();
}

cudaError_t launch_rho_f32(const StepParams& p, int law, StateF32 st, int slot, cudaStream_t s) {
  return launch_rho_impl<float>(p, law, st, slot, s);
}

}  // namespace adot
