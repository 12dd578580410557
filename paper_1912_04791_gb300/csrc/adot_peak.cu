// Throughput probes of the arithmetic pipes that bound the step kernels (no
// counterpart in the paper): the measured denominators of their ALU rooflines.
//
// Every probe runs a resident grid (8 blocks of 256 threads per SM) in which
// each thread advances 8 independent chains for `iters` iterations, so that
// each SM sub-partition always has independent instructions to issue and the
// pipe, not latency, is the limit. The result of every chain is folded into
// one store per thread under a condition that never holds for the inputs
// given, so the compiler keeps the work. Kinds:
//   0 FFMA    float32 fused multiply-add, counted as 2 flops
//   1 FFMA2   paired float32 fused multiply-add (__ffma2_rn), 4 flops
//   2 RSQ     float32 reciprocal square root on the multi-function unit
//   3 SIN     float32 sine approximation on the multi-function unit
//   4 DFMA    float64 fused multiply-add, 2 flops
//   5 TANH    float32 hyperbolic tangent approximation on the multi-function unit
//   6 TANH2   paired bfloat16 hyperbolic tangent approximation (2 ops)
#include <cuda_runtime.h>

#include "../../include/adot.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

__device__ __forceinline__ float mufu_rsq(float x) {
  float y;
  asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float mufu_tanh(float x) {
  float y;
  asm volatile("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ unsigned mufu_tanh_bf16x2(unsigned x) {
  unsigned y;
  asm volatile("tanh.approx.bf16x2 %0, %1;" : "=r"(y) : "r"(x));
  return y;
}

__device__ __forceinline__ float mufu_sin(float x) {
  float y;
  asm volatile("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <int KIND>
__global__ void __launch_bounds__(kThreads) k_pipe_probe(float* out, double* out64, int iters,
                                                         float a, float b) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if constexpr (KIND == 4) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1e-3 * (t + c);
    const double da = a, db = b;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], da, db);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1.0) out64[t] = s;
  } else if constexpr (KIND == 6) {
    // bf16 pairs near 0.5 (0x3f00): tanh maps them into (0.46, 0.47), a fixed point region
    unsigned x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 0x3f003f00u + (unsigned)((t + c) & 7) * 0x00010001u;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = mufu_tanh_bf16x2(x[c] + 0x00010001u);
    }
    unsigned s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s ^= x[c];
    if (s == 0xffffffffu) out[t] = (float)s;
  } else if constexpr (KIND == 1) {
    float2 x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = make_float2(1.0f + 1e-3f * (t + c), 2.0f + 1e-3f * c);
    const float2 pa = make_float2(a, a), pb = make_float2(b, b);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], pa, pb);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
    if (s == -1.0f) out[t] = s;
  } else {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.0f + 1e-3f * (t + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) {
        if constexpr (KIND == 0) x[c] = fmaf(x[c], a, b);
        if constexpr (KIND == 2) x[c] = mufu_rsq(x[c] + b);
        if constexpr (KIND == 3) x[c] = mufu_sin(x[c] + b);
        if constexpr (KIND == 5) x[c] = mufu_tanh(x[c] + b);
      }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1.0f) out[t] = s;
  }
}

template <int KIND>
cudaError_t launch_probe(unsigned grid, float* out, double* out64, int iters, cudaStream_t s) {
  k_pipe_probe<KIND><<<grid, kThreads, 0, s>>>(out, out64, iters, 0.999999f, 1e-7f);
  return cudaGetLastError();
}

cudaError_t launch_kind(int kind, unsigned grid, float* out, double* out64, int iters,
                        cudaStream_t s) {
  switch (kind) {
    case 0: return launch_probe<0>(grid, out, out64, iters, s);
    case 1: return launch_probe<1>(grid, out, out64, iters, s);
    case 2: return launch_probe<2>(grid, out, out64, iters, s);
    case 3: return launch_probe<3>(grid, out, out64, iters, s);
    case 5: return launch_probe<5>(grid, out, out64, iters, s);
    case 6: return launch_probe<6>(grid, out, out64, iters, s);
    default: return launch_probe<4>(grid, out, out64, iters, s);
  }
}

}  // namespace

extern "C" adot_status adot_measure_pipe(int kind, int device, double* rate_out,
                                         double* seconds_out) {
  if (kind < 0 || kind > 6 || !rate_out) return ADOT_E_INVALID_ARG;
  if (device >= 0 && cudaSetDevice(device) != cudaSuccess) return ADOT_E_CUDA;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return ADOT_E_CUDA;
  const unsigned grid = (unsigned)(sms * kBlocksPerSm);
  const int64_t threads = (int64_t)grid * kThreads;
  // about 30-60 ms per timed launch at the expected rates
  const int iters = (kind == 0 || kind == 1) ? (1 << 18) : (kind == 4 ? (1 << 12) : (1 << 15));
  float* out = nullptr;
  double* out64 = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  adot_status st = ADOT_E_CUDA;
  float ms = 0.0f;
  if (cudaMalloc((void**)&out, sizeof(float) * threads) != cudaSuccess) goto done;
  if (cudaMalloc((void**)&out64, sizeof(double) * threads) != cudaSuccess) goto done;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) goto done;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) goto done;
  if (launch_kind(kind, grid, out, out64, iters / 8, s) != cudaSuccess) goto done;  // warm-up
  if (cudaEventRecord(e0, s) != cudaSuccess) goto done;
  if (launch_kind(kind, grid, out, out64, iters, s) != cudaSuccess) goto done;
  if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) goto done;
  if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.0f)) goto done;
  {
    const double per_op = (kind == 0 || kind == 4 || kind == 6) ? 2.0 : (kind == 1 ? 4.0 : 1.0);
    const double ops = per_op * (double)kChains * (double)iters * (double)threads;
    *rate_out = ops / (ms * 1e-3);
    if (seconds_out) *seconds_out = ms * 1e-3;
    st = ADOT_OK;
  }
done:
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (out) cudaFree(out);
  if (out64) cudaFree(out64);
  return st;
}
