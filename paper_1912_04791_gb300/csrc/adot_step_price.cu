// PRICE-C time step (Sec. 3.2, Eq. PRICEjump, AiPRICE, Apsi, Im), the paper's
// centred comparison scheme, as an instantiation of the persistent warp-tile
// step kernel with the PRICE-C edge (edge_fluct_price), in float64 and in
// float32 with the float-float state; with and without the friction source,
// the sediment feed and the slope-continuing ghosts. Without an eigen-solve
// per node the edge costs about a tenth of the DOT edge, and the step is bound
// by the 48 bytes per cell-update it moves through HBM; the register cap is
// lower than the DOT kernel's so that more warps keep loads in flight.
//
// Also the stateless PRICE-C fluctuations of independent edges, for the C ABI.
#include "adot_step_impl.cuh"

namespace adot {

namespace {

// The PRICE-C launch shapes: 256 threads with a register cap of 64 (4 resident
// blocks per SM, the DOT warp-tile shape), 40 (6 blocks) or 32 (8 blocks).
template <typename R, int LAW, bool EXT, int B, int CAP>
cudaError_t launch_shape(const StepParams& p, typename Prec<R>::State in,
                         typename Prec<R>::State out, int slot, cudaStream_t s) {
  int sms = 152, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t per_sm = MinBlocks<B, CAP>::value;
  const int64_t tiles = (p.n + 30) / 31;
  const int64_t wpb = B / 32;
  int64_t g = (tiles + wpb - 1) / wpb;
  if (g > sms * per_sm) g = sms * per_sm;
  k_step_warp<R, LAW, B, CAP, EXT, 1><<<(unsigned)g, B, 0, s>>>(p, in, out, slot,
                                                               warp_split<1>(p.n, g * (B / 32)));
  return cudaGetLastError();
}

template <typename R, int LAW, bool EXT>
cudaError_t launch_law(const StepParams& p, StepVariant v, typename Prec<R>::State in,
                       typename Prec<R>::State out, int slot, cudaStream_t s) {
  if (p.ctl == nullptr || p.n < 1) return cudaErrorInvalidValue;
  if (v.warp_tiles && v.block == 256) {
    if (v.reg_cap == 32) return launch_shape<R, LAW, EXT, 256, 32>(p, in, out, slot, s);
    if (v.reg_cap == 40) return launch_shape<R, LAW, EXT, 256, 40>(p, in, out, slot, s);
  }
  return launch_shape<R, LAW, EXT, 256, 64>(p, in, out, slot, s);
}

template <typename R, bool EXT>
cudaError_t launch_scheme(const StepParams& p, int law, StepVariant v, typename Prec<R>::State in,
                          typename Prec<R>::State out, int slot, cudaStream_t s) {
  if (law == LAW_GRASS) return launch_law<R, LAW_GRASS, EXT>(p, v, in, out, slot, s);
  if (law == LAW_MPM) return launch_law<R, LAW_MPM, EXT>(p, v, in, out, slot, s);
  if (law == LAW_GRASS_THR || law == LAW_POWER)
    return launch_law<R, LAW_GRASS_THR, EXT>(p, v, in, out, slot, s);
  return cudaErrorInvalidValue;
}

// D-/+ of n independent PRICE-C edges from [3][n] float64 arrays; in float32
// the inputs are first rounded to float-float, as the time-step state is.
template <typename R, int LAW>
__global__ void __launch_bounds__(256) k_price_fluct(const StepParams p, R nu, R inv_nu,
                                                     const double* __restrict__ WL,
                                                     const double* __restrict__ WR, int64_t n,
                                                     double* __restrict__ Dm,
                                                     double* __restrict__ Dp) {
  using S = typename Prec<R>::S;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    S wl[3], wr[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      wl[r] = Prec<R>::from_double(WL[r * n + e]);
      wr[r] = Prec<R>::from_double(WR[r * n + e]);
    }
    R dm[3], dp[3];
    edge_fluct_price<R, LAW>(p, nu, inv_nu, wl, wr, dm, dp);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      Dm[r * n + e] = (double)dm[r];
      Dp[r * n + e] = (double)dp[r];
    }
  }
}

template <typename R>
cudaError_t launch_fluct_prec(int law, const StepParams& p, double nu, const double* WL,
                              const double* WR, int64_t n, double* Dm, double* Dp,
                              cudaStream_t s) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  const unsigned G = (unsigned)(g < 1 ? 1 : g);
  const R rnu = R(nu), rinv = R(1.0 / nu);
  if (law == LAW_GRASS)
    k_price_fluct<R, LAW_GRASS><<<G, 256, 0, s>>>(p, rnu, rinv, WL, WR, n, Dm, Dp);
  else if (law == LAW_MPM)
    k_price_fluct<R, LAW_MPM><<<G, 256, 0, s>>>(p, rnu, rinv, WL, WR, n, Dm, Dp);
  else if (law == LAW_GRASS_THR || law == LAW_POWER)
    k_price_fluct<R, LAW_GRASS_THR><<<G, 256, 0, s>>>(p, rnu, rinv, WL, WR, n, Dm, Dp);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_step_price_f32(const StepParams& p, int law, StepVariant v, StateF32 in,
                                  StateF32 out, int slot, cudaStream_t s) {
  if (step_needs_ext(p)) return launch_scheme<float, true>(p, law, v, in, out, slot, s);
  return launch_scheme<float, false>(p, law, v, in, out, slot, s);
}

cudaError_t launch_step_price_f64(const StepParams& p, int law, StepVariant v, StateF64 in,
                                  StateF64 out, int slot, cudaStream_t s) {
  if (step_needs_ext(p)) return launch_scheme<double, true>(p, law, v, in, out, slot, s);
  return launch_scheme<double, false>(p, law, v, in, out, slot, s);
}

cudaError_t launch_price_fluct(int precision, int law, const StepParams& p, double nu,
                               const double* WL, const double* WR, int64_t n, double* Dm,
                               double* Dp, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (!(nu > 0.0)) return cudaErrorInvalidValue;
  if (precision == 0) return launch_fluct_prec<double>(law, p, nu, WL, WR, n, Dm, Dp, s);
  return launch_fluct_prec<float>(law, p, nu, WL, WR, n, Dm, Dp, s);
}

}  // namespace adot
