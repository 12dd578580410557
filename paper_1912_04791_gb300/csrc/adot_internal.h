// Internal declarations shared by the kernel translation units and the C-ABI
// runtime. Not part of the public interface (include/adot.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "adot_math.cuh"

namespace adot {

// One slot of the device control block. Step n reads slot n % 3, writes slot
// (n+1) % 3 and clears the CFL maximum of slot (n+2) % 3, so no slot is read
// and written by the same launch.
struct CtlSlot {
  double t;                     // time at the start of the step that reads the slot
  double dt;                    // dt of the step that wrote the slot
  long long steps;              // steps taken since the state was set
  unsigned long long rho_bits;  // max spectral radius of the state (float bits or double bits)
};

struct Ctl {
  CtlSlot s[3];
  double t_end;     // steps are clipped to land on t_end; no work once t >= t_end
  unsigned status;  // sticky ST_* bits
  unsigned pad;
  // work-pool head of the warp-tile step kernel: 0 between launches (the warp
  // that takes the launch's last ticket puts it back)
  unsigned grab;
  // cells the float32 warp-tile step left to k_fixup (an edge needing the
  // float64 redo), and k_fixup's finished blocks: both 0 between steps (the
  // last block of k_fixup puts them back)
  unsigned fix_count;
  unsigned fix_done;
  unsigned pad2;
};

struct StateF32 {
  float2* h;
  float2* q;
  float2* z;
};

struct StateF64 {
  double* h;
  double* q;
  double* z;
};

// Parameters common to every time-step launch (fixed for a context).
struct StepParams {
  int64_t n;
  double dx;
  double cfl;
  int periodic;
  int bc_left, bc_right;
  double bcl[3], bcr[3];
  LawT<float> lf;
  LawT<double> ld;
  double fric;              // g / K_s^2 of the Strickler friction source; 0 = none
  double feed_l, feed_r;    // xi q_s,in imposed through a BC_INFLOW_QS end
  int order;                // 1: Eq. scheme; 2: MUSCL-Hancock (k_step2_warp)
  int scheme;               // 0: DOT jump function (Eq. DOTjumpN); 1: PRICE-C (Eq. PRICEjump)
  double price_eps;         // PRICE-C: epsilon of I_eps (Eq. Im)
  Ctl* ctl;
  const float* absA;  // surrogate |A|_Psi per edge, [9][n+1] (NaN in row 0: analytic edge)
  unsigned* fix_list; // [n] cells left to k_fixup by the float32 warp-tile step (nullptr: redo in place)
};

enum : int {
  BC_TRANSMISSIVE = 0,
  BC_PERIODIC = 1,
  BC_INFLOW_Q = 2,
  BC_OUTFLOW_H = 3,
  BC_INFLOW_QZ = 4,
  BC_INFLOW_QS = 5,
  BC_OUTFLOW_HS = 6
};

// Whether a configuration runs the step kernels with the friction source, the
// sediment feed and the slope-continuing ghosts compiled in.
inline bool step_needs_ext(const StepParams& p) {
  if (p.fric != 0.0) return true;
  if (p.periodic) return false;
  for (int k : {p.bc_left, p.bc_right})
    if (k == BC_INFLOW_QS || k == BC_OUTFLOW_HS) return true;
  return false;
}

// A compiled variant of the step kernel: threads per block and the register
// cap per thread (0 = none) given to the register allocator.
struct StepVariant {
  int block;
  int reg_cap;
  int warp_tiles;  // 1: persistent warp-tile kernel (k_step_warp), 0: block kernel (k_step)
};

// The compiled variants, in the order the autotuner tries them. The warp-tile
// shapes with register caps 32 and 40 exist for PRICE-C only (its edge needs no
// eigen-solve); PRICE-C runs the warp-tile shapes of 256 threads with caps 64,
// 40 and 32.
constexpr int kNumStepVariants = 12;
constexpr StepVariant kStepVariants[kNumStepVariants] = {
    {256, 0, 0},  {256, 64, 0}, {128, 0, 0}, {128, 64, 0}, {512, 0, 0},  {512, 64, 0},
    {256, 64, 1}, {128, 64, 1}, {128, 72, 1}, {256, 80, 1}, {256, 40, 1}, {256, 32, 1}};

bool step_block_supported(int block);
bool step_variant_supported(StepVariant v);

// One time step (Eq. scheme): fluctuations on every edge, update of every cell,
// CFL maximum of the updated state. slot = step index mod 3.
cudaError_t launch_step_f32(const StepParams& p, int law, StepVariant v, StateF32 in, StateF32 out,
                            int slot, cudaStream_t s);
cudaError_t launch_step_f64(const StepParams& p, int law, StepVariant v, StateF64 in, StateF64 out,
                            int slot, cudaStream_t s);

// The same with the friction source and the sediment feed compiled in; the
// plain entry points forward to these when the configuration uses either.
cudaError_t launch_step_f32_ext(const StepParams& p, int law, StepVariant v, StateF32 in,
                                StateF32 out, int slot, cudaStream_t s);
cudaError_t launch_step_f64_ext(const StepParams& p, int law, StepVariant v, StateF64 in,
                                StateF64 out, int slot, cudaStream_t s);

// Second-order (MUSCL-Hancock) time step, warp-tile variants only; the plain
// entry points forward to these when p.order == 2.
cudaError_t launch_step2_f32(const StepParams& p, int law, StepVariant v, StateF32 in,
                             StateF32 out, int slot, cudaStream_t s);
cudaError_t launch_step2_f64(const StepParams& p, int law, StepVariant v, StateF64 in,
                             StateF64 out, int slot, cudaStream_t s);

// PRICE-C time step (p.scheme == 1), warp tiles only: the plain entry points
// forward to these. A variant that is not one of PRICE-C's runs as 256 x 64.
cudaError_t launch_step_price_f32(const StepParams& p, int law, StepVariant v, StateF32 in,
                                  StateF32 out, int slot, cudaStream_t s);
cudaError_t launch_step_price_f64(const StepParams& p, int law, StepVariant v, StateF64 in,
                                  StateF64 out, int slot, cudaStream_t s);

// Stateless PRICE-C fluctuations of n edges ([3][n] float64 device arrays) with
// nu = dt/dx and p.price_eps, in float64 (precision 0) or float32 from
// float-float inputs (precision 1).
cudaError_t launch_price_fluct(int precision, int law, const StepParams& p, double nu,
                               const double* WL, const double* WR, int64_t n, double* Dm,
                               double* Dp, cudaStream_t s);

// Time step whose edges take |A|_Psi from p.absA (float32, Grass law, 256 x 64).
cudaError_t launch_step_sur_f32(const StepParams& p, StateF32 in, StateF32 out, int slot,
                                cudaStream_t s);
cudaError_t launch_step_sur_f32_ext(const StepParams& p, StateF32 in, StateF32 out, int slot,
                                    cudaStream_t s);

// n edge samples of a state (edge index drawn with splitmix64 from seed and the
// sample number): raw inputs X [n][7] (h, q, z left and right, A_g) and float64
// labels T [n][9] = sum_k w_k |A(Psi_k)|, stored as float32.
cudaError_t launch_harvest_f32(const StepParams& p, StateF32 st, int slot, int64_t n, uint64_t seed,
                               float Ag, float* X, float* T, cudaStream_t s);
cudaError_t launch_harvest_f64(const StepParams& p, StateF64 st, int slot, int64_t n, uint64_t seed,
                               float Ag, float* X, float* T, cudaStream_t s);

// CFL maximum of a state into ctl->s[slot].rho_bits (which must be zero), and
// admissibility (h > 0, finite) into ctl->status.
cudaError_t launch_rho_f32(const StepParams& p, int law, StateF32 st, int slot, cudaStream_t s);
cudaError_t launch_rho_f64(const StepParams& p, int law, StateF64 st, int slot, cudaStream_t s);

// Adds to *count the quadrature nodes of a float-float state whose float32
// cubic-root solve the step kernels redo in float64 (3 per edge; edges 0..n,
// or 0..n-1 when periodic).
cudaError_t launch_redo_count_f32(const StepParams& p, int law, StateF32 st, int slot,
                                  unsigned long long* count, cudaStream_t s);

// float64 <-> float-float conversion of n values.
cudaError_t launch_to_ff(const double* src, float2* dst, int64_t n, cudaStream_t s);
cudaError_t launch_from_ff(const float2* src, double* dst, int64_t n, cudaStream_t s);

// Stateless fluctuations of n edges; WL, WR, Dm, Dp are device [3][n] float64.
// rho_bits (double bits) and status are device scalars updated with atomics.
cudaError_t launch_fluct(int precision, int law, const LawT<float>& lf, const LawT<double>& ld,
                         const double* WL, const double* WR, int64_t n, double* Dm, double* Dp,
                         unsigned long long* rho_bits, unsigned* status, cudaStream_t s);

// Fixed-order float64 sums of the three state arrays: partial has room for
// sums_partial_blocks(n) * 3 doubles; out receives 3 doubles.
int sums_partial_blocks(int64_t n);
cudaError_t launch_sums_f32(StateF32 st, int64_t n, double* partial, double* out, cudaStream_t s);
cudaError_t launch_sums_f64(StateF64 st, int64_t n, double* partial, double* out, cudaStream_t s);

}  // namespace adot
