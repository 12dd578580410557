// Auxiliary kernels: stateless edge fluctuations, float64 <-> float-float
// conversion and fixed-order conserved sums.
#include <type_traits>

#include "../../include/adot.h"
#include "adot_step_impl.cuh"

namespace adot {

static unsigned grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  return (unsigned)(g < 1 ? 1 : g);
}

// D-/+ of n independent edges (Eq. DOTjumpN) from [3][n] float64 arrays. In
// float32 the inputs are rounded to float-float, as the time-step state is.
// rho_bits collects the largest spectral radius met at a quadrature node.
template <typename R, int LAW>
__global__ void __launch_bounds__(256) k_fluct(const StepParams p, const double* __restrict__ WL,
                                               const double* __restrict__ WR, int64_t n,
                                               double* __restrict__ Dm, double* __restrict__ Dp,
                                               unsigned long long* rho_bits, unsigned* status) {
  using S = typename Prec<R>::S;
  __shared__ double sRed[8];
  unsigned flags = 0;
  double rho = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    S wl[3], wr[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      wl[r] = Prec<R>::from_double(WL[r * n + e]);
      wr[r] = Prec<R>::from_double(WR[r * n + e]);
    }
    R dm[3], dp[3];
    edge_fluct<R, LAW>(p, wl, wr, dm, dp, flags);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      Dm[r * n + e] = (double)dm[r];
      Dp[r * n + e] = (double)dp[r];
    }
    const R dh = Prec<R>::diff(wr[0], wl[0]), dq = Prec<R>::diff(wr[1], wl[1]);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const R s = (k == 0) ? R(GL3_S0) : ((k == 1) ? R(0.5) : R(GL3_S2));
      const R hk = Prec<R>::hi(wl[0]) + s * dh, qk = Prec<R>::hi(wl[1]) + s * dq;
      if (hk > R(0)) rho = fmax(rho, (double)spectral_radius<R, LAW>(Prec<R>::law(p), hk, qk));
      else flags |= ST_DEPTH;
    }
  }
  if (!(rho <= 3.0e300)) {
    flags |= ST_NONFINITE;
    rho = 0.0;
  }
  rho = warp_max(rho);
  if ((threadIdx.x & 31) == 0) sRed[threadIdx.x >> 5] = rho;
  __syncthreads();
  if (threadIdx.x < 32) {
    rho = (threadIdx.x < 8) ? sRed[threadIdx.x] : 0.0;
    rho = warp_max(rho);
    if (threadIdx.x == 0 && rho > 0.0)
      atomicMax(rho_bits, (unsigned long long)__double_as_longlong(rho));
  }
  if (flags) atomicOr(status, flags);
}

cudaError_t launch_fluct(int precision, int law, const LawT<float>& lf, const LawT<double>& ld,
                         const double* WL, const double* WR, int64_t n, double* Dm, double* Dp,
                         unsigned long long* rho_bits, unsigned* status, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  StepParams p{};
  p.lf = lf;
  p.ld = ld;
  int64_t g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  const unsigned G = (unsigned)g;
  if (precision == 0) {
    if (law == LAW_GRASS) k_fluct<double, LAW_GRASS><<<G, 256, 0, s>>>(p, WL, WR, n, Dm, Dp, rho_bits, status);
    else if (law == LAW_MPM) k_fluct<double, LAW_MPM><<<G, 256, 0, s>>>(p, WL, WR, n, Dm, Dp, rho_bits, status);
    else if (law == LAW_GRASS_THR || law == LAW_POWER)
      k_fluct<double, LAW_GRASS_THR><<<G, 256, 0, s>>>(p, WL, WR, n, Dm, Dp, rho_bits, status);
    else return cudaErrorInvalidValue;
  } else {
    if (law == LAW_GRASS) k_fluct<float, LAW_GRASS><<<G, 256, 0, s>>>(p, WL, WR, n, Dm, Dp, rho_bits, status);
    else if (law == LAW_MPM) k_fluct<float, LAW_MPM><<<G, 256, 0, s>>>(p, WL, WR, n, Dm, Dp, rho_bits, status);
    else if (law == LAW_GRASS_THR || law == LAW_POWER)
      k_fluct<float, LAW_GRASS_THR><<<G, 256, 0, s>>>(p, WL, WR, n, Dm, Dp, rho_bits, status);
    else return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Edge samples with float64 labels (see launch_harvest_f32).
template <typename R>
__global__ void __launch_bounds__(256) k_harvest(const StepParams p, const typename Prec<R>::State st,
                                                 int slot, int64_t n, uint64_t seed, float Ag,
                                                 float* __restrict__ X, float* __restrict__ T,
                                                 unsigned* status) {
  using S = typename Prec<R>::S;
  unsigned flags = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = (int64_t)(splitmix64(seed ^ (0xD1B54A32D192ED03ull * (uint64_t)(i + 1))) %
                                (uint64_t)(p.n + 1));
    S wl[3], wr[3];
    load_edge<R>(p, st, e, slot, wl, wr);
    double dl[3], dr[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      if constexpr (std::is_same<R, float>::value) {
        dl[r] = ff_to_double(*reinterpret_cast<const float2*>(&wl[r]));
        dr[r] = ff_to_double(*reinterpret_cast<const float2*>(&wr[r]));
      } else {
        dl[r] = *reinterpret_cast<const double*>(&wl[r]);
        dr[r] = *reinterpret_cast<const double*>(&wr[r]);
      }
      X[i * 7 + r] = (float)dl[r];
      X[i * 7 + 3 + r] = (float)dr[r];
    }
    X[i * 7 + 6] = Ag;
    double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double sk = (k == 0) ? GL3_S0 : ((k == 1) ? 0.5 : GL3_S2);
      const double w = (k == 1) ? GL3_W1 : GL3_W0;
      double M[9];
      abs_A_matrix_f64<LAW_GRASS>(p.ld, dl[0] + sk * (dr[0] - dl[0]), dl[1] + sk * (dr[1] - dl[1]), M,
                                  flags);
#pragma unroll
      for (int r = 0; r < 9; ++r) acc[r] += w * M[r];
    }
#pragma unroll
    for (int r = 0; r < 9; ++r) T[i * 9 + r] = (float)acc[r];
  }
  if (flags && status) atomicOr(status, flags);
}

cudaError_t launch_harvest_f32(const StepParams& p, StateF32 st, int slot, int64_t n, uint64_t seed,
                               float Ag, float* X, float* T, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_harvest<float><<<grid_for(n), 256, 0, s>>>(p, st, slot, n, seed, Ag, X, T, &p.ctl->status);
  return cudaGetLastError();
}

cudaError_t launch_harvest_f64(const StepParams& p, StateF64 st, int slot, int64_t n, uint64_t seed,
                               float Ag, float* X, float* T, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_harvest<double><<<grid_for(n), 256, 0, s>>>(p, st, slot, n, seed, Ag, X, T, &p.ctl->status);
  return cudaGetLastError();
}

// Quadrature nodes of a float-float state whose float32 cubic-root solve the
// step kernels redo in float64: the same test (1 - arg^2 below
// TAU_FP64_FALLBACK, or not finite) on the same node values, the two outer
// Gauss-Legendre nodes in the paired form and the midpoint in the scalar form,
// as edge_fluct_f32x2 evaluates them. A diagnostic over the current state; it
// is not part of a time step.
template <int LAW>
__global__ void __launch_bounds__(256) k_redo_count(const StepParams p, const StateF32 st, int slot,
                                                    int64_t n_edges,
                                                    unsigned long long* __restrict__ count) {
  unsigned long long mine = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_edges;
       e += (int64_t)gridDim.x * blockDim.x) {
    float2 wl[3], wr[3];
    load_edge<float, true>(p, st, e, slot, wl, wr);
    const float dh = ff_diff(wr[0], wl[0]), dq = ff_diff(wr[1], wl[1]);
    const float h0 = wl[0].x, q0 = wl[1].x;
    const float2 s2 = make_float2((float)GL3_S0, (float)GL3_S2);
    Eig2 e2;
    node_eig_x2<LAW>(p.lf, fma2(s2, p2(dh), p2(h0)), fma2(s2, p2(dq), p2(q0)), e2);
    const float dx0 = fmaf(-e2.arg.x, e2.arg.x, 1.0f), dx1 = fmaf(-e2.arg.y, e2.arg.y, 1.0f);
    Eig<float> em;
    node_eig<float, LAW>(p.lf, h0 + 0.5f * dh, q0 + 0.5f * dq, em);
    const float dm = 1.0f - em.arg * em.arg;
    mine += (!(dx0 >= TAU_FP64_FALLBACK) ? 1 : 0) + (!(dx1 >= TAU_FP64_FALLBACK) ? 1 : 0) +
            (!(dm >= TAU_FP64_FALLBACK) ? 1 : 0);
  }
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(count, mine);
}

cudaError_t launch_redo_count_f32(const StepParams& p, int law, StateF32 st, int slot,
                                  unsigned long long* count, cudaStream_t s) {
  const int64_t ne = p.periodic ? p.n : p.n + 1;
  if (law == LAW_GRASS)
    k_redo_count<LAW_GRASS><<<grid_for(ne), 256, 0, s>>>(p, st, slot, ne, count);
  else if (law == LAW_MPM)
    k_redo_count<LAW_MPM><<<grid_for(ne), 256, 0, s>>>(p, st, slot, ne, count);
  else if (law == LAW_GRASS_THR || law == LAW_POWER)
    k_redo_count<LAW_GRASS_THR><<<grid_for(ne), 256, 0, s>>>(p, st, slot, ne, count);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_to_ff(const double* __restrict__ src, float2* __restrict__ dst,
                                               int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = ff_from_double(src[i]);
}

__global__ void __launch_bounds__(256) k_from_ff(const float2* __restrict__ src, double* __restrict__ dst,
                                                 int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = ff_to_double(src[i]);
}

cudaError_t launch_to_ff(const double* src, float2* dst, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_to_ff<<<grid_for(n), 256, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}

cudaError_t launch_from_ff(const float2* src, double* dst, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_from_ff<<<grid_for(n), 256, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Fixed-order sums: block b sums a fixed contiguous chunk (thread-strided,
// then a fixed shared-memory tree); one block then sums the block partials
// the same way. The order depends only on n, so results are reproducible.
// ---------------------------------------------------------------------------

int sums_partial_blocks(int64_t n) {
  int64_t b = (n + 4095) / 4096;
  if (b > 1024) b = 1024;
  return (int)(b < 1 ? 1 : b);
}

__device__ __forceinline__ double load_d(const float2* a, int64_t i) { return ff_to_double(a[i]); }
__device__ __forceinline__ double load_d(const double* a, int64_t i) { return a[i]; }

template <typename P>
__device__ __forceinline__ void block_tree_sum3(double v[3], double* out) {
  __shared__ double sh[3][256];
  for (int r = 0; r < 3; ++r) sh[r][threadIdx.x] = v[r];
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int r = 0; r < 3; ++r) sh[r][threadIdx.x] += sh[r][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int r = 0; r < 3; ++r) out[r] = sh[r][0];
}

template <typename P>
__global__ void __launch_bounds__(256) k_sums_partial(const P* h, const P* q, const P* z, int64_t n,
                                                      int64_t chunk, double* partial) {
  const int64_t b0 = (int64_t)blockIdx.x * chunk;
  const int64_t b1 = (b0 + chunk < n) ? b0 + chunk : n;
  double v[3] = {0.0, 0.0, 0.0};
  for (int64_t i = b0 + threadIdx.x; i < b1; i += 256) {
    v[0] += load_d(h, i);
    v[1] += load_d(q, i);
    v[2] += load_d(z, i);
  }
  block_tree_sum3<P>(v, partial + 3 * blockIdx.x);
}

__global__ void __launch_bounds__(256) k_sums_final(const double* partial, int nb, double* out) {
  double v[3] = {0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < nb; i += 256)
    for (int r = 0; r < 3; ++r) v[r] += partial[3 * i + r];
  block_tree_sum3<double>(v, out);
}

template <typename P>
static cudaError_t launch_sums(const P* h, const P* q, const P* z, int64_t n, double* partial,
                               double* out, cudaStream_t s) {
  const int nb = sums_partial_blocks(n);
  const int64_t chunk = (n + nb - 1) / nb;
  k_sums_partial<P><<<nb, 256, 0, s>>>(h, q, z, n, chunk, partial);
  k_sums_final<<<1, 256, 0, s>>>(partial, nb, out);
  return cudaGetLastError();
}

cudaError_t launch_sums_f32(StateF32 st, int64_t n, double* partial, double* out, cudaStream_t s) {
  return launch_sums<float2>(st.h, st.q, st.z, n, partial, out, s);
}

cudaError_t launch_sums_f64(StateF64 st, int64_t n, double* partial, double* out, cudaStream_t s) {
  return launch_sums<double>(st.h, st.q, st.z, n, partial, out, s);
}

}  // namespace adot

// Probe of the library's float32 device math for the tests (no counterpart in
// the paper): kind 0 = acos_third (the polynomial arccos(x) / 3 of the step
// kernels), kind 1 = CUDA's acosf(x) / 3, on n values x of device memory.
namespace {
__global__ void k_math_probe(int kind, const float* __restrict__ x, float* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = kind == 0 ? adot::acos_third(x[i]) : acosf(x[i]) * (float)(1.0 / 3.0);
}
}  // namespace

extern "C" adot_status adot_math_probe(int32_t kind, const float* x, float* y, int64_t n, void* cuda_stream) {
  if (kind < 0 || kind > 1 || n < 0 || (n > 0 && (!x || !y))) return ADOT_E_INVALID_ARG;
  if (n == 0) return ADOT_OK;
  const int64_t g64 = (n + 255) / 256;
  const unsigned g = (unsigned)(g64 < 152 * 32 ? g64 : 152 * 32);
  k_math_probe<<<g, 256, 0, (cudaStream_t)cuda_stream>>>(kind, x, y, n);
  if (cudaGetLastError() != cudaSuccess) return ADOT_E_CUDA;
  return cudaStreamSynchronize((cudaStream_t)cuda_stream) == cudaSuccess ? ADOT_OK : ADOT_E_CUDA;
}
