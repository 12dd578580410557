// Allocation-free time stepping (adot_step_noalloc).
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory manager (a custom op whose device memory must come from
// the host framework's allocator), real-time or embedded loops that reserve
// all memory up front, and code running while another component holds the
// device allocator. For them this entry point advances a caller-owned float64
// state without allocating anything. The step kernel's scratch (the second
// ping-pong state buffer and the control block holding time, dt and the CFL
// maximum) lives in the file-scope device array below instead of in
// context-owned allocations. The array is part of the module image: every GPU
// that loads the library holds it (ADOT_NOALLOC_MAX_CELLS cells, about 1.5 MB)
// until the process exits. Every call shares it, so calls that overlap on the
// GPU race; it keeps the last call's contents, and the control block, which
// must start from zero, is cleared at the start of every call.
//
// Under CUDA's lazy module loading the driver places this translation unit's
// module (and so the array) on a device when something in it is first used,
// which here is the set-up's cudaGetSymbolAddress; each step kernel is loaded
// at its first launch. The first call on a device with a given configuration
// is therefore the one that may allocate, and later calls allocate nothing.
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>

#include "../../include/adot.h"
#include "adot_internal.h"

namespace adot {
adot_status validate_config(const adot_config* c);
void make_step_params(const adot_config* cfg, StepParams* p);
}  // namespace adot

using namespace adot;

namespace {

// 256 bytes of control block, then three arrays of ADOT_NOALLOC_MAX_CELLS doubles.
constexpr int kCtlWords = 32;
static_assert(sizeof(Ctl) <= kCtlWords * sizeof(double), "control block exceeds its scratch slot");
constexpr size_t kScratchWords = kCtlWords + 3 * (size_t)ADOT_NOALLOC_MAX_CELLS;

static __device__ __align__(256) double g_noalloc_scratch[kScratchWords];

// Device address of g_noalloc_scratch per device, found once per device. In
// host code the array's name is a host-side stand-in, not a device address.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

adot_status scratch_for_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ADOT_E_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return ADOT_E_CUDA;
    g_scratch_ptr[dev] = (double*)p;
  }
  *out = g_scratch_ptr[dev];
  return ADOT_OK;
}

// Clears the control block and starts the clock at t0 with no end time.
__global__ void k_noalloc_ctl_init(Ctl* ctl, double t0) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int s = 0; s < 3; ++s) {
    ctl->s[s].t = 0.0;
    ctl->s[s].dt = 0.0;
    ctl->s[s].steps = 0;
    ctl->s[s].rho_bits = 0ull;
  }
  ctl->s[0].t = t0;
  ctl->t_end = INFINITY;
  ctl->status = 0u;
  ctl->pad = 0u;
  ctl->grab = 0u;
  ctl->fix_count = 0u;
  ctl->fix_done = 0u;
  ctl->pad2 = 0u;
}

adot_status from_bits(unsigned bits) {
  if (bits & ST_NONFINITE) return ADOT_E_NONFINITE;
  if (bits & ST_DEPTH) return ADOT_E_NONPOSITIVE_DEPTH;
  if (bits & ST_NONHYPERBOLIC) return ADOT_E_NONHYPERBOLIC;
  if (bits & ST_TIMEOUT) return ADOT_E_TIMEOUT;
  return ADOT_OK;
}

}  // namespace

extern "C" adot_status adot_step_noalloc(const adot_config* cfg, double* h, double* q, double* z,
                                         int64_t n_steps, double* t_io, void* cuda_stream) {
  adot_status st = validate_config(cfg);
  if (st) return st;
  if (!h || !q || !z || !t_io || n_steps < 0 || !isfinite(*t_io)) return ADOT_E_INVALID_ARG;
  if (cfg->precision != ADOT_FP64) return ADOT_E_UNSUPPORTED;
  if (cfg->n_cells > ADOT_NOALLOC_MAX_CELLS) return ADOT_E_INVALID_ARG;
  if (cfg->device >= 0 && cudaSetDevice(cfg->device) != cudaSuccess) return ADOT_E_CUDA;
  double* scratch = nullptr;
  st = scratch_for_current_device(&scratch);
  if (st) return st;

  const int64_t n = cfg->n_cells;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  StepParams p;
  make_step_params(cfg, &p);
  p.ctl = (Ctl*)scratch;
  double* buf = scratch + kCtlWords;
  const StateF64 user{h, q, z};
  const StateF64 tmp{buf, buf + ADOT_NOALLOC_MAX_CELLS, buf + 2 * ADOT_NOALLOC_MAX_CELLS};
  const StepVariant v{256, 64, p.order == 2 ? 1 : 0};  // order 2 runs warp tiles
  const int law = cfg->law.kind;

  k_noalloc_ctl_init<<<1, 32, 0, s>>>(p.ctl, *t_io);
  if (cudaGetLastError() != cudaSuccess) return ADOT_E_CUDA;
  if (launch_rho_f64(p, law, user, 0, s) != cudaSuccess) return ADOT_E_CUDA;
  for (int64_t k = 0; k < n_steps; ++k) {
    const bool even = (k % 2) == 0;
    if (launch_step_f64(p, law, v, even ? user : tmp, even ? tmp : user, (int)(k % 3), s) !=
        cudaSuccess)
      return ADOT_E_CUDA;
  }
  if (n_steps % 2 == 1) {  // the last step wrote the scratch copy: bring it back
    const size_t bytes = sizeof(double) * (size_t)n;
    if (cudaMemcpyAsync(h, tmp.h, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(q, tmp.q, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(z, tmp.z, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return ADOT_E_CUDA;
  }
  Ctl host;
  if (cudaMemcpyAsync(&host, p.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return ADOT_E_CUDA;
  *t_io = host.s[n_steps % 3].t;
  return from_bits(host.status);
}
