// C-ABI runtime of the A-DOT library (declared in include/adot.h).
//
// A context owns two ping-pong state buffers, a device control block (time,
// dt, step count and CFL maximum in three rotating slots plus a sticky status
// word), host-pinned mirrors for status reads, and a CUDA graph of
// `steps_per_graph` consecutive time-step launches. A run of steps replays the
// graph whenever the step counter is at a multiple of 6 (the rotation period
// of the three control slots and the two buffers) and launches single steps
// otherwise, so the graph's fixed kernel arguments always match.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <tuple>

#include "../../include/adot.h"
#include "adot_internal.h"

using namespace adot;

struct adot_ctx {
  adot_config cfg;
  int device;
  int prec;  // 0 = float64, 1 = float-float
  int law;
  StepVariant var;  // step kernel variant in use
  bool tuned;       // variant fixed by the config, the cache or adot_autotune
  int steps_per_graph;
  cudaStream_t stream;
  bool own_stream;
  cudaStream_t cap_stream;
  StepParams p;
  void* buf[2][3];  // [ping-pong][h, q, z]
  int cur;          // buffer holding the current state
  int phase;        // steps launched since set_state, mod 6
  Ctl* d_ctl;
  Ctl* h_ctl;       // pinned mirror
  double* d_io;     // 3 * n float64 staging for conversions
  unsigned* d_fix;  // float32: n cells left to k_fixup by a step
  double* d_partial;
  double* d_sums;
  double* h_sums;   // pinned, 3
  double* d_fl;     // 12 * fl_cap float64 for host-pointer fluctuation calls
  int64_t fl_cap;
  unsigned long long* d_flrho;  // fluctuation scratch: rho bits + status
  unsigned long long* h_flrho;  // pinned mirror (2 words)
  cudaGraphExec_t graph;
  bool graph_ready;
  bool state_set;
  double t_end_dev;  // t_end currently stored in the control block
  // learned surrogate of |A|_Psi (float32 Grass contexts)
  adot_mlp* mlp;
  float fr_lo, fr_hi;
  float* d_absA;                 // [9][n+1]
  unsigned long long* d_fb;      // edges that fell back (cumulative)
  long long sur_steps0;          // step counter when the surrogate was attached
  unsigned long long fb0;        // fallback count when it was attached
};

namespace adot {
cudaError_t launch_mlp_edges(const adot_mlp* m, const StepParams& sp, StateF32 st, int slot,
                             float Ag, float fr_lo, float fr_hi, float* absA,
                             unsigned long long* fb, cudaStream_t s);
bool mlp_ready(const adot_mlp* m);
}  // namespace adot

namespace {


#define CK(expr)                               \
  do {                                         \
    cudaError_t _e = (expr);                   \
    if (_e != cudaSuccess) return ADOT_E_CUDA; \
  } while (0)

adot_status status_from_bits(unsigned bits) {
  if (bits & ST_NONFINITE) return ADOT_E_NONFINITE;
  if (bits & ST_DEPTH) return ADOT_E_NONPOSITIVE_DEPTH;
  if (bits & ST_NONHYPERBOLIC) return ADOT_E_NONHYPERBOLIC;
  if (bits & ST_TIMEOUT) return ADOT_E_TIMEOUT;
  return ADOT_OK;
}

bool valid_bc(int k) { return k >= ADOT_BC_TRANSMISSIVE && k <= ADOT_BC_OUTFLOW_HS; }

}  // namespace

namespace adot {
adot_status validate_config(const adot_config* c);
void make_step_params(const adot_config* cfg, StepParams* p);
}  // namespace adot

adot_status adot::validate_config(const adot_config* c) {
  if (!c) return ADOT_E_INVALID_ARG;
  if (c->n_cells < 1) return ADOT_E_INVALID_ARG;
  if (!(c->x_max > c->x_min) || !isfinite(c->x_min) || !isfinite(c->x_max)) return ADOT_E_INVALID_ARG;
  if (!(c->cfl > 0.0 && c->cfl <= 1.0)) return ADOT_E_INVALID_ARG;
  if (!(c->law.g > 0.0) || !(c->law.xi > 0.0) || !isfinite(c->law.Ag)) return ADOT_E_INVALID_ARG;
  if (c->law.kind == ADOT_LAW_MPM) {
    if (!(c->law.s_rel > 1.0) || !(c->law.d50 > 0.0) || !(c->law.manning_n >= 0.0))
      return ADOT_E_INVALID_ARG;
  } else if (c->law.kind == ADOT_LAW_GRASS_THR) {
    if (!(c->law.u_cr >= 0.0) || !isfinite(c->law.u_cr)) return ADOT_E_INVALID_ARG;
  } else if (c->law.kind == ADOT_LAW_POWER) {
    if (!(c->law.u_cr >= 0.0) || !isfinite(c->law.u_cr)) return ADOT_E_INVALID_ARG;
    if (!(c->law.beta >= 1.0) || !isfinite(c->law.beta)) return ADOT_E_INVALID_ARG;
  } else if (c->law.kind != ADOT_LAW_GRASS) {
    return ADOT_E_INVALID_ARG;
  }
  if (c->precision != ADOT_FP64 && c->precision != ADOT_FP32) return ADOT_E_INVALID_ARG;
  if (!valid_bc(c->bc_left) || !valid_bc(c->bc_right)) return ADOT_E_INVALID_ARG;
  if ((c->bc_left == ADOT_BC_PERIODIC) != (c->bc_right == ADOT_BC_PERIODIC)) return ADOT_E_INVALID_ARG;
  for (int i = 0; i < 3; ++i)
    if (!isfinite(c->bc_left_value[i]) || !isfinite(c->bc_right_value[i])) return ADOT_E_INVALID_ARG;
  if (!(c->ks >= 0.0) || !isfinite(c->ks)) return ADOT_E_INVALID_ARG;
  if (c->order < 0 || c->order > 2) return ADOT_E_INVALID_ARG;
  if (c->block_threads != 0 && !step_block_supported(c->block_threads)) return ADOT_E_INVALID_ARG;
  if (c->scheme != ADOT_SCHEME_DOT && c->scheme != ADOT_SCHEME_PRICE_C) return ADOT_E_INVALID_ARG;
  const bool price = c->scheme == ADOT_SCHEME_PRICE_C;
  if (price && (!(c->price_eps >= 0.0) || !isfinite(c->price_eps))) return ADOT_E_INVALID_ARG;
  const bool price_cap = c->reg_cap == 32 || c->reg_cap == 40;
  if (c->reg_cap != 0 && c->reg_cap != 64 && c->reg_cap != 72 && c->reg_cap != 80 &&
      c->reg_cap != -1 && !price_cap)
    return ADOT_E_INVALID_ARG;
  if (price_cap && !price) return ADOT_E_UNSUPPORTED;  // caps 32 and 40 serve PRICE-C only
  // PRICE-C runs the first-order warp-tile kernel of 256 threads
  if (price && (c->order == 2 || c->step_kernel == 1 || c->reg_cap == -1 || c->reg_cap == 72 ||
                c->reg_cap == 80 || (c->block_threads != 0 && c->block_threads != 256)))
    return ADOT_E_UNSUPPORTED;
  if (c->step_kernel < 0 || c->step_kernel > 2) return ADOT_E_INVALID_ARG;
  if (c->steps_per_graph < 0 || c->device < -1) return ADOT_E_INVALID_ARG;
  if (c->order == 2 && (c->step_kernel == 1 || c->reg_cap == -1 || c->ks != 0.0 ||
                        c->bc_left == ADOT_BC_INFLOW_QS || c->bc_right == ADOT_BC_INFLOW_QS))
    return ADOT_E_UNSUPPORTED;
  return ADOT_OK;
}

// Launch parameters of a configuration (everything but the control block).
void adot::make_step_params(const adot_config* cfg, StepParams* out) {
  StepParams& p = *out;
  p = StepParams{};
  const int64_t n = cfg->n_cells;
  p.n = n;
  p.dx = (cfg->x_max - cfg->x_min) / (double)n;
  p.cfl = cfg->cfl;
  p.periodic = (cfg->bc_left == ADOT_BC_PERIODIC) ? 1 : 0;
  p.bc_left = cfg->bc_left;
  p.bc_right = cfg->bc_right;
  for (int i = 0; i < 3; ++i) {
    p.bcl[i] = cfg->bc_left_value[i];
    p.bcr[i] = cfg->bc_right_value[i];
  }
  const adot_law& L = cfg->law;
  double K3 = 3.0 * L.xi * L.Ag;
  double mpm_c = 0.0, mpm_scale = 0.0;
  if (L.kind == ADOT_LAW_MPM) {
    mpm_c = L.manning_n * L.manning_n / ((L.s_rel - 1.0) * L.d50);
    mpm_scale = L.xi * sqrt(L.g * (L.s_rel - 1.0) * L.d50 * L.d50 * L.d50);
  }
  const bool thr = L.kind == ADOT_LAW_GRASS_THR || L.kind == ADOT_LAW_POWER;
  const double ucr = thr ? L.u_cr : 0.0;
  const double beta = (L.kind == ADOT_LAW_POWER) ? L.beta : 3.0;
  if (L.kind == ADOT_LAW_POWER) K3 = beta * L.xi * L.Ag;
  const double xa = L.xi * L.Ag;
  p.ld = LawT<double>{L.g, K3, mpm_c, mpm_scale, ucr, beta, xa};
  p.lf = LawT<float>{(float)L.g,   (float)K3,  (float)mpm_c, (float)mpm_scale,
                     (float)ucr,   (float)beta, (float)xa};
  p.fric = (cfg->ks > 0.0) ? L.g / (cfg->ks * cfg->ks) : 0.0;
  p.feed_l = L.xi * cfg->bc_left_value[1];
  p.feed_r = L.xi * cfg->bc_right_value[1];
  p.order = (cfg->order == 2) ? 2 : 1;
  p.scheme = (cfg->scheme == ADOT_SCHEME_PRICE_C) ? 1 : 0;
  p.price_eps = p.scheme ? cfg->price_eps : 0.0;
}

namespace {

StateF32 st32(adot_ctx* c, int which) {
  return StateF32{(float2*)c->buf[which][0], (float2*)c->buf[which][1], (float2*)c->buf[which][2]};
}
StateF64 st64(adot_ctx* c, int which) {
  return StateF64{(double*)c->buf[which][0], (double*)c->buf[which][1], (double*)c->buf[which][2]};
}

cudaError_t launch_one_v(adot_ctx* c, StepVariant v, cudaStream_t s, int cur, int phase) {
  const int slot = phase % 3;
  if (c->mlp) {  // surrogate |A|_Psi for every edge, then the update
    cudaError_t e = launch_mlp_edges(c->mlp, c->p, st32(c, cur), slot, (float)c->cfg.law.Ag,
                                     c->fr_lo, c->fr_hi, c->d_absA, c->d_fb, s);
    if (e != cudaSuccess) return e;
    StepParams p = c->p;
    p.absA = c->d_absA;
    return launch_step_sur_f32(p, st32(c, cur), st32(c, 1 - cur), slot, s);
  }
  if (c->prec == ADOT_FP32)
    return launch_step_f32(c->p, c->law, v, st32(c, cur), st32(c, 1 - cur), slot, s);
  return launch_step_f64(c->p, c->law, v, st64(c, cur), st64(c, 1 - cur), slot, s);
}

cudaError_t launch_one(adot_ctx* c, cudaStream_t s, int cur, int phase) {
  return launch_one_v(c, c->var, s, cur, phase);
}

adot_status build_graph(adot_ctx* c) {
  if (c->graph_ready) {
    cudaGraphExecDestroy(c->graph);
    c->graph_ready = false;
  }
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t err = cudaSuccess;
  for (int k = 0; k < c->steps_per_graph && err == cudaSuccess; ++k)
    err = launch_one(c, c->cap_stream, k & 1, k % 6);
  cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &g);
  if (err != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return ADOT_E_CUDA;
  }
  err = cudaGraphInstantiate(&c->graph, g, 0);
  cudaGraphDestroy(g);
  if (err != cudaSuccess) return ADOT_E_CUDA;
  c->graph_ready = true;
  return ADOT_OK;
}

adot_status enqueue(adot_ctx* c, int64_t n) {
  while (n > 0) {
    if (c->phase == 0 && n >= c->steps_per_graph) {
      adot_status st = build_graph(c);
      if (st) return st;
      CK(cudaGraphLaunch(c->graph, c->stream));
      n -= c->steps_per_graph;  // a multiple of 6: phase and buffer unchanged
    } else {
      CK(launch_one(c, c->stream, c->cur, c->phase));
      c->cur ^= 1;
      c->phase = (c->phase + 1) % 6;
      --n;
    }
  }
  return ADOT_OK;
}

// Process-wide cache of tuned variants: (device, law, precision, log2 n, filters,
// friction / feed kernels or not, order of the scheme, jump function).
using TuneKey = std::tuple<int, int, int, int, int, int, int, int, int, int>;
std::mutex g_tune_mu;
std::map<TuneKey, StepVariant> g_tune_cache;

TuneKey tune_key(const adot_ctx* c) {
  int lg = 0;
  for (int64_t n = c->p.n; n > 1; n >>= 1) ++lg;
  return std::make_tuple(c->device, c->law, c->prec, lg, c->cfg.block_threads, c->cfg.reg_cap,
                         c->cfg.step_kernel, step_needs_ext(c->p) ? 1 : 0, c->p.order,
                         c->p.scheme);
}

bool candidate(const adot_config& cfg, StepVariant v) {
  if (cfg.block_threads && v.block != cfg.block_threads) return false;
  if (cfg.reg_cap > 0 && v.reg_cap != cfg.reg_cap) return false;
  if (cfg.reg_cap == -1 && v.reg_cap != 0) return false;
  if (cfg.step_kernel == 1 && v.warp_tiles) return false;
  if (cfg.step_kernel == 2 && !v.warp_tiles) return false;
  if (cfg.order == 2 && !v.warp_tiles) return false;  // the second-order kernel is warp tiles
  const bool price_shape = v.warp_tiles && v.block == 256 &&
                           (v.reg_cap == 64 || v.reg_cap == 40 || v.reg_cap == 32);
  if (cfg.scheme == ADOT_SCHEME_PRICE_C) return price_shape;
  if (v.reg_cap == 40 || v.reg_cap == 32) return false;  // PRICE-C shapes
  return true;
}

// Times each candidate variant on the current state: trial steps read the
// current buffer and write the other one, with the current control slot, so
// neither the state nor the step counter advances. The slot they write is
// reset afterwards.
adot_status tune(adot_ctx* c, int64_t trial) {
  if (trial < 1) trial = 1;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return ADOT_E_CUDA;
  }
  float best_ms = 0.0f;
  StepVariant best = c->var;
  bool have = false;
  cudaError_t err = cudaSuccess;
  for (int i = 0; i < kNumStepVariants && err == cudaSuccess; ++i) {
    const StepVariant v = kStepVariants[i];
    if (!candidate(c->cfg, v)) continue;
    for (int k = 0; k < 2 && err == cudaSuccess; ++k) err = launch_one_v(c, v, c->stream, c->cur, c->phase);
    if (err == cudaSuccess) err = cudaEventRecord(e0, c->stream);
    for (int64_t k = 0; k < trial && err == cudaSuccess; ++k)
      err = launch_one_v(c, v, c->stream, c->cur, c->phase);
    if (err == cudaSuccess) err = cudaEventRecord(e1, c->stream);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess && (!have || ms < best_ms)) {
      best_ms = ms;
      best = v;
      have = true;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return ADOT_E_CUDA;
  CK(cudaMemsetAsync(&c->d_ctl->s[(c->phase + 1) % 3].rho_bits, 0, sizeof(unsigned long long),
                     c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->var = best;
  c->tuned = true;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[tune_key(c)] = best;
  }
  return build_graph(c);
}

adot_status set_t_end(adot_ctx* c, double t_end) {
  if (c->t_end_dev == t_end) return ADOT_OK;
  // the pinned mirror is only written while the stream is idle (callers sync)
  CK(cudaStreamSynchronize(c->stream));
  c->h_ctl->t_end = t_end;
  CK(cudaMemcpyAsync(&c->d_ctl->t_end, &c->h_ctl->t_end, sizeof(double), cudaMemcpyHostToDevice,
                     c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->t_end_dev = t_end;
  return ADOT_OK;
}

adot_status read_ctl(adot_ctx* c) {
  CK(cudaMemcpyAsync(c->h_ctl, c->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return ADOT_OK;
}

// Fixes the step variant once a state is present: from the config, the
// process-wide cache, or by timing the candidates on this state.
adot_status choose_variant(adot_ctx* c) {
  if (!c->tuned) {
    bool cached = false;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune_cache.find(tune_key(c));
      if (it != g_tune_cache.end()) {
        c->var = it->second;
        cached = true;
      }
    }
    if (cached) {
      c->tuned = true;
      return build_graph(c);
    }
    return tune(c, 8);
  }
  return ADOT_OK;
}


// Checkpoint header: fixed 128 bytes ahead of the raw state words.
struct CkptHeader {
  uint32_t magic;    // 'ADOT' little-endian
  uint32_t version;  // 1
  int64_t n_cells;
  int32_t precision;
  int32_t law;
  double t, dt;
  int64_t steps;
  uint64_t rho_bits;
  uint32_t status;
  uint32_t state_words;  // bytes per stored value: 8 (float-float pair or float64)
  uint64_t fingerprint;
  uint8_t reserved[128 - 72];
};
static_assert(sizeof(CkptHeader) == 128, "checkpoint header is 128 bytes");
constexpr uint32_t kCkptMagic = 0x544F4441u;

// FNV-1a over the config fields that enter the arithmetic (not the launch shape).
uint64_t fnv1a(uint64_t h, const void* p, size_t n) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

uint64_t config_fingerprint(const adot_config& c) {
  uint64_t h = 1469598103934665603ull;
  h = fnv1a(h, &c.n_cells, sizeof c.n_cells);
  h = fnv1a(h, &c.x_min, sizeof c.x_min);
  h = fnv1a(h, &c.x_max, sizeof c.x_max);
  h = fnv1a(h, &c.cfl, sizeof c.cfl);
  h = fnv1a(h, &c.law.kind, sizeof c.law.kind);
  h = fnv1a(h, &c.law.g, sizeof c.law.g);
  h = fnv1a(h, &c.law.xi, sizeof c.law.xi);
  h = fnv1a(h, &c.law.Ag, sizeof c.law.Ag);
  h = fnv1a(h, &c.law.s_rel, sizeof c.law.s_rel);
  h = fnv1a(h, &c.law.d50, sizeof c.law.d50);
  h = fnv1a(h, &c.law.manning_n, sizeof c.law.manning_n);
  h = fnv1a(h, &c.law.u_cr, sizeof c.law.u_cr);
  h = fnv1a(h, &c.law.beta, sizeof c.law.beta);
  h = fnv1a(h, &c.ks, sizeof c.ks);
  const int32_t order = (c.order == 2) ? 2 : 1;
  h = fnv1a(h, &order, sizeof order);
  if (c.scheme == ADOT_SCHEME_PRICE_C) {  // DOT configurations keep their earlier fingerprint
    h = fnv1a(h, &c.scheme, sizeof c.scheme);
    h = fnv1a(h, &c.price_eps, sizeof c.price_eps);
  }
  h = fnv1a(h, &c.precision, sizeof c.precision);
  h = fnv1a(h, &c.bc_left, sizeof c.bc_left);
  h = fnv1a(h, &c.bc_right, sizeof c.bc_right);
  h = fnv1a(h, c.bc_left_value, sizeof c.bc_left_value);
  h = fnv1a(h, c.bc_right_value, sizeof c.bc_right_value);
  return h;
}

int64_t checkpoint_bytes(const adot_ctx* c) {
  return (int64_t)sizeof(CkptHeader) + 3 * c->p.n * 8;
}

void free_ctx(adot_ctx* c) {
  if (!c) return;
  if (c->graph_ready) cudaGraphExecDestroy(c->graph);
  for (int b = 0; b < 2; ++b)
    for (int k = 0; k < 3; ++k)
      if (c->buf[b][k]) cudaFree(c->buf[b][k]);
  if (c->d_ctl) cudaFree(c->d_ctl);
  if (c->h_ctl) cudaFreeHost(c->h_ctl);
  if (c->d_io) cudaFree(c->d_io);
  if (c->d_fix) cudaFree(c->d_fix);
  if (c->d_partial) cudaFree(c->d_partial);
  if (c->d_sums) cudaFree(c->d_sums);
  if (c->h_sums) cudaFreeHost(c->h_sums);
  if (c->d_fl) cudaFree(c->d_fl);
  if (c->d_flrho) cudaFree(c->d_flrho);
  if (c->h_flrho) cudaFreeHost(c->h_flrho);
  if (c->d_absA) cudaFree(c->d_absA);
  if (c->d_fb) cudaFree(c->d_fb);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  free(c);
}

}  // namespace

extern "C" {

const char* adot_version(void) { return "adot-gb300 0.1 (sm_103a)"; }

const char* adot_status_string(adot_status s) {
  switch (s) {
    case ADOT_OK: return "ok";
    case ADOT_E_INVALID_ARG: return "invalid argument";
    case ADOT_E_NONPOSITIVE_DEPTH: return "non-positive water depth";
    case ADOT_E_NONFINITE: return "non-finite value";
    case ADOT_E_NONHYPERBOLIC: return "non-hyperbolic state";
    case ADOT_E_CUDA: return "CUDA error";
    case ADOT_E_TIMEOUT: return "device wait timed out";
    case ADOT_E_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

adot_status adot_create(const adot_config* cfg, void* cuda_stream, adot_ctx** out) {
  if (!out) return ADOT_E_INVALID_ARG;
  *out = nullptr;
  adot_status st = validate_config(cfg);
  if (st) return st;
  int dev = 0;
  if (cfg->device >= 0 && cudaSetDevice(cfg->device) != cudaSuccess) return ADOT_E_CUDA;
  if (cudaGetDevice(&dev) != cudaSuccess) return ADOT_E_CUDA;
  adot_ctx* c = (adot_ctx*)calloc(1, sizeof(adot_ctx));
  if (!c) return ADOT_E_CUDA;
  c->cfg = *cfg;
  c->device = dev;
  c->prec = cfg->precision;
  c->law = cfg->law.kind;
  c->var = StepVariant{cfg->block_threads ? cfg->block_threads : 256,
                       cfg->reg_cap == -1 ? 0 : 64, cfg->step_kernel == 2 ? 1 : 0};
  if (!step_variant_supported(c->var) || !candidate(*cfg, c->var)) {  // e.g. warp tiles without a cap
    for (int i = 0; i < kNumStepVariants; ++i)
      if (candidate(*cfg, kStepVariants[i])) {
        c->var = kStepVariants[i];
        break;
      }
  }
  {
    int n_cand = 0;
    for (int i = 0; i < kNumStepVariants; ++i) n_cand += candidate(*cfg, kStepVariants[i]) ? 1 : 0;
    c->tuned = (n_cand <= 1);
  }
  int spg = cfg->steps_per_graph ? cfg->steps_per_graph : 48;
  c->steps_per_graph = ((spg + 5) / 6) * 6;
  c->t_end_dev = INFINITY;
  const int64_t n = cfg->n_cells;

  make_step_params(cfg, &c->p);
  StepParams& p = c->p;

  cudaError_t e = cudaSuccess;
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
  } else {
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    c->own_stream = true;
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
  const size_t elem = (c->prec == ADOT_FP32) ? sizeof(float2) : sizeof(double);
  for (int b = 0; b < 2 && e == cudaSuccess; ++b)
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaMalloc(&c->buf[b][k], elem * (size_t)n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_ctl, sizeof(Ctl));
  p.ctl = c->d_ctl;
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&c->h_ctl, sizeof(Ctl), cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_partial, sizeof(double) * 3 * sums_partial_blocks(n));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_sums, sizeof(double) * 3);
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&c->h_sums, sizeof(double) * 3, cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_flrho, sizeof(unsigned long long) * 2);
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&c->h_flrho, sizeof(unsigned long long) * 2, cudaHostAllocDefault);
  if (e == cudaSuccess && c->prec == ADOT_FP32) e = cudaMalloc((void**)&c->d_io, sizeof(double) * 3 * (size_t)n);
  if (e == cudaSuccess && c->prec == ADOT_FP32) e = cudaMalloc((void**)&c->d_fix, sizeof(unsigned) * (size_t)n);
  p.fix_list = c->d_fix;
  if (e == cudaSuccess) {
    memset(c->h_ctl, 0, sizeof(Ctl));
    c->h_ctl->t_end = INFINITY;
    e = cudaMemcpyAsync(c->d_ctl, c->h_ctl, sizeof(Ctl), cudaMemcpyHostToDevice, c->stream);
  }
  for (int b = 0; b < 2 && e == cudaSuccess; ++b)
    for (int k = 0; k < 3 && e == cudaSuccess; ++k)
      e = cudaMemsetAsync(c->buf[b][k], 0, elem * (size_t)n, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess || build_graph(c) != ADOT_OK) {
    free_ctx(c);
    return ADOT_E_CUDA;
  }
  *out = c;
  return ADOT_OK;
}

void adot_destroy(adot_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  free_ctx(c);
}

adot_status adot_set_state(adot_ctx* c, const double* h, const double* q, const double* z,
                           int on_device, double t0) {
  if (!c || !h || !q || !z || !isfinite(t0)) return ADOT_E_INVALID_ARG;
  const int64_t n = c->p.n;
  const size_t bytes = sizeof(double) * (size_t)n;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const double* src[3] = {h, q, z};
  CK(cudaStreamSynchronize(c->stream));
  for (int k = 0; k < 3; ++k) {
    if (c->prec == ADOT_FP32) {
      CK(cudaMemcpyAsync(c->d_io + k * n, src[k], bytes, kind, c->stream));
      CK(launch_to_ff(c->d_io + k * n, (float2*)c->buf[0][k], n, c->stream));
    } else {
      CK(cudaMemcpyAsync(c->buf[0][k], src[k], bytes, kind, c->stream));
    }
  }
  memset(c->h_ctl, 0, sizeof(Ctl));
  c->h_ctl->s[0].t = t0;
  c->h_ctl->t_end = INFINITY;
  c->t_end_dev = INFINITY;
  CK(cudaMemcpyAsync(c->d_ctl, c->h_ctl, sizeof(Ctl), cudaMemcpyHostToDevice, c->stream));
  c->cur = 0;
  c->phase = 0;
  if (c->prec == ADOT_FP32)
    CK(launch_rho_f32(c->p, c->law, st32(c, 0), 0, c->stream));
  else
    CK(launch_rho_f64(c->p, c->law, st64(c, 0), 0, c->stream));
  adot_status st = read_ctl(c);
  if (st) return st;
  c->state_set = true;
  st = status_from_bits(c->h_ctl->status);
  if (st) return st;
  return choose_variant(c);
}

adot_status adot_get_state(adot_ctx* c, double* h, double* q, double* z, int on_device) {
  if (!c || !h || !q || !z) return ADOT_E_INVALID_ARG;
  const int64_t n = c->p.n;
  const size_t bytes = sizeof(double) * (size_t)n;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  double* dst[3] = {h, q, z};
  for (int k = 0; k < 3; ++k) {
    if (c->prec == ADOT_FP32) {
      CK(launch_from_ff((const float2*)c->buf[c->cur][k], c->d_io + k * n, n, c->stream));
      CK(cudaMemcpyAsync(dst[k], c->d_io + k * n, bytes, kind, c->stream));
    } else {
      CK(cudaMemcpyAsync(dst[k], c->buf[c->cur][k], bytes, kind, c->stream));
    }
  }
  CK(cudaStreamSynchronize(c->stream));
  return ADOT_OK;
}

adot_status adot_checkpoint_size(adot_ctx* c, int64_t* bytes_out) {
  if (!c || !bytes_out) return ADOT_E_INVALID_ARG;
  *bytes_out = checkpoint_bytes(c);
  return ADOT_OK;
}

adot_status adot_checkpoint_save(adot_ctx* c, void* buf, int64_t bytes, int on_device) {
  if (!c || !buf || !c->state_set || bytes < checkpoint_bytes(c)) return ADOT_E_INVALID_ARG;
  adot_status st = read_ctl(c);
  if (st) return st;
  const CtlSlot& s = c->h_ctl->s[c->phase % 3];
  CkptHeader hd;
  memset(&hd, 0, sizeof hd);
  hd.magic = kCkptMagic;
  hd.version = 1;
  hd.n_cells = c->p.n;
  hd.precision = c->prec;
  hd.law = c->law;
  hd.t = s.t;
  hd.dt = s.dt;
  hd.steps = s.steps;
  hd.rho_bits = s.rho_bits;
  hd.status = c->h_ctl->status;
  hd.state_words = 8;
  hd.fingerprint = config_fingerprint(c->cfg);
  const size_t row = (size_t)c->p.n * 8;
  unsigned char* out = static_cast<unsigned char*>(buf);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (on_device)
    CK(cudaMemcpyAsync(out, &hd, sizeof hd, cudaMemcpyHostToDevice, c->stream));
  else
    memcpy(out, &hd, sizeof hd);
  for (int k = 0; k < 3; ++k)
    CK(cudaMemcpyAsync(out + sizeof hd + k * row, c->buf[c->cur][k], row, kind, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return ADOT_OK;
}

adot_status adot_checkpoint_load(adot_ctx* c, const void* buf, int64_t bytes, int on_device) {
  if (!c || !buf || bytes < (int64_t)sizeof(CkptHeader)) return ADOT_E_INVALID_ARG;
  CkptHeader hd;
  const unsigned char* in = static_cast<const unsigned char*>(buf);
  CK(cudaStreamSynchronize(c->stream));
  if (on_device) {
    CK(cudaMemcpyAsync(&hd, in, sizeof hd, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  } else {
    memcpy(&hd, in, sizeof hd);
  }
  if (hd.magic != kCkptMagic || hd.version != 1 || hd.state_words != 8 || hd.n_cells != c->p.n ||
      hd.precision != c->prec || hd.law != c->law || hd.fingerprint != config_fingerprint(c->cfg) ||
      bytes < checkpoint_bytes(c) || !isfinite(hd.t))
    return ADOT_E_INVALID_ARG;
  const size_t row = (size_t)c->p.n * 8;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  for (int k = 0; k < 3; ++k)
    CK(cudaMemcpyAsync(c->buf[0][k], in + sizeof hd + k * row, row, kind, c->stream));
  memset(c->h_ctl, 0, sizeof(Ctl));
  c->h_ctl->s[0].t = hd.t;
  c->h_ctl->s[0].dt = hd.dt;
  c->h_ctl->s[0].steps = hd.steps;
  c->h_ctl->s[0].rho_bits = hd.rho_bits;
  c->h_ctl->status = hd.status;
  c->h_ctl->t_end = INFINITY;
  c->t_end_dev = INFINITY;
  CK(cudaMemcpyAsync(c->d_ctl, c->h_ctl, sizeof(Ctl), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->cur = 0;
  c->phase = 0;
  c->state_set = true;
  adot_status st = status_from_bits(hd.status);
  if (st) return st;
  return choose_variant(c);
}

adot_status adot_enqueue_steps(adot_ctx* c, int64_t n_steps) {
  if (!c || n_steps < 0 || !c->state_set) return ADOT_E_INVALID_ARG;
  adot_status st = set_t_end(c, INFINITY);
  if (st) return st;
  return enqueue(c, n_steps);
}

adot_status adot_query(adot_ctx* c, double* t_out, int64_t* steps_out, double* dt_last_out) {
  if (!c) return ADOT_E_INVALID_ARG;
  adot_status st = read_ctl(c);
  if (st) return st;
  const CtlSlot& s = c->h_ctl->s[c->phase % 3];
  if (t_out) *t_out = s.t;
  if (steps_out) *steps_out = s.steps;
  if (dt_last_out) *dt_last_out = s.dt;
  return status_from_bits(c->h_ctl->status);
}

adot_status adot_step(adot_ctx* c, int64_t n_steps, double* t_out, double* dt_last_out) {
  adot_status st = adot_enqueue_steps(c, n_steps);
  if (st) return st;
  return adot_query(c, t_out, nullptr, dt_last_out);
}

adot_status adot_run_to(adot_ctx* c, double t_end, int64_t* steps_out) {
  if (!c || !c->state_set || !isfinite(t_end)) return ADOT_E_INVALID_ARG;
  adot_status st = read_ctl(c);
  if (st) return st;
  const long long steps0 = c->h_ctl->s[c->phase % 3].steps;
  if (steps_out) *steps_out = 0;
  if (c->h_ctl->s[c->phase % 3].t >= t_end) return status_from_bits(c->h_ctl->status);
  st = set_t_end(c, t_end);
  if (st) return st;
  for (;;) {
    // align to the graph's phase with single steps, then replay whole graphs
    int64_t chunk = c->phase ? (6 - c->phase) : c->steps_per_graph;
    st = enqueue(c, chunk);
    if (st) return st;
    st = read_ctl(c);
    if (st) return st;
    const CtlSlot& s = c->h_ctl->s[c->phase % 3];
    if (steps_out) *steps_out = s.steps - steps0;
    adot_status dev = status_from_bits(c->h_ctl->status);
    if (dev) return dev;
    if (!(s.t < t_end)) break;
  }
  return ADOT_OK;
}

adot_status adot_fluctuations(adot_ctx* c, const double* WL, const double* WR, int64_t n,
                              double* Dminus, double* Dplus, double* rho_max_out, int on_device) {
  if (!c || n < 0) return ADOT_E_INVALID_ARG;
  if (n > 0 && (!WL || !WR || !Dminus || !Dplus)) return ADOT_E_INVALID_ARG;
  if (n == 0) {
    if (rho_max_out) *rho_max_out = 0.0;
    return ADOT_OK;
  }
  const double *wl = WL, *wr = WR;
  double *dm = Dminus, *dp = Dplus;
  const size_t bytes = sizeof(double) * 3 * (size_t)n;
  if (!on_device) {
    if (c->fl_cap < n) {
      if (c->d_fl) cudaFree(c->d_fl);
      c->d_fl = nullptr;
      c->fl_cap = 0;
      CK(cudaMalloc((void**)&c->d_fl, 4 * bytes));
      c->fl_cap = n;
    }
    double* base = c->d_fl;
    CK(cudaMemcpyAsync(base, WL, bytes, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(base + 3 * n, WR, bytes, cudaMemcpyHostToDevice, c->stream));
    wl = base;
    wr = base + 3 * n;
    dm = base + 6 * n;
    dp = base + 9 * n;
  }
  CK(cudaMemsetAsync(c->d_flrho, 0, 2 * sizeof(unsigned long long), c->stream));
  CK(launch_fluct(c->prec, c->law, c->p.lf, c->p.ld, wl, wr, n, dm, dp, c->d_flrho,
                  (unsigned*)(c->d_flrho + 1), c->stream));
  if (!on_device) {
    CK(cudaMemcpyAsync(Dminus, dm, bytes, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(Dplus, dp, bytes, cudaMemcpyDeviceToHost, c->stream));
  }
  CK(cudaMemcpyAsync(c->h_flrho, c->d_flrho, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                     c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (rho_max_out) {
    unsigned long long b = c->h_flrho[0];
    double r;
    memcpy(&r, &b, sizeof(r));
    *rho_max_out = r;
  }
  return status_from_bits((unsigned)(c->h_flrho[1] & 0xffffffffu));
}

adot_status adot_price_fluctuations(adot_ctx* c, const double* WL, const double* WR, int64_t n,
                                    double dt_over_dx, double* Dminus, double* Dplus,
                                    int on_device) {
  if (!c || n < 0 || !(dt_over_dx > 0.0) || !isfinite(dt_over_dx)) return ADOT_E_INVALID_ARG;
  if (n > 0 && (!WL || !WR || !Dminus || !Dplus)) return ADOT_E_INVALID_ARG;
  if (n == 0) return ADOT_OK;
  const double *wl = WL, *wr = WR;
  double *dm = Dminus, *dp = Dplus;
  const size_t bytes = sizeof(double) * 3 * (size_t)n;
  if (!on_device) {
    if (c->fl_cap < n) {
      if (c->d_fl) cudaFree(c->d_fl);
      c->d_fl = nullptr;
      c->fl_cap = 0;
      CK(cudaMalloc((void**)&c->d_fl, 4 * bytes));
      c->fl_cap = n;
    }
    double* base = c->d_fl;
    CK(cudaMemcpyAsync(base, WL, bytes, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(base + 3 * n, WR, bytes, cudaMemcpyHostToDevice, c->stream));
    wl = base;
    wr = base + 3 * n;
    dm = base + 6 * n;
    dp = base + 9 * n;
  }
  StepParams p = c->p;
  p.price_eps = c->cfg.price_eps;
  CK(launch_price_fluct(c->prec, c->law, p, dt_over_dx, wl, wr, n, dm, dp, c->stream));
  if (!on_device) {
    CK(cudaMemcpyAsync(Dminus, dm, bytes, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(Dplus, dp, bytes, cudaMemcpyDeviceToHost, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  return ADOT_OK;
}

adot_status adot_autotune(adot_ctx* c, int64_t trial_steps, int32_t* block_out,
                          int32_t* reg_cap_out, int32_t* step_kernel_out) {
  if (!c || !c->state_set || trial_steps < 1) return ADOT_E_INVALID_ARG;
  adot_status st = tune(c, trial_steps);
  if (st) return st;
  if (block_out) *block_out = c->var.block;
  if (reg_cap_out) *reg_cap_out = c->var.reg_cap ? c->var.reg_cap : -1;
  if (step_kernel_out) *step_kernel_out = c->var.warp_tiles ? 2 : 1;
  return ADOT_OK;
}

adot_status adot_set_surrogate(adot_ctx* c, adot_mlp* m, double fr_lo, double fr_hi) {
  if (!c) return ADOT_E_INVALID_ARG;
  if (m == nullptr) {
    c->mlp = nullptr;
    return build_graph(c);
  }
  if (c->prec != ADOT_FP32 || c->law != ADOT_LAW_GRASS || c->p.order == 2 || c->p.scheme != 0)
    return ADOT_E_UNSUPPORTED;
  if (!mlp_ready(m) || !(fr_lo <= fr_hi)) return ADOT_E_INVALID_ARG;
  CK(cudaStreamSynchronize(c->stream));
  if (!c->d_absA) {
    CK(cudaMalloc((void**)&c->d_absA, sizeof(float) * 9 * (size_t)(c->p.n + 1)));
    // [0]: fallbacks of the steps, [1]: fallbacks of adot_surrogate_eval
    CK(cudaMalloc((void**)&c->d_fb, 2 * sizeof(unsigned long long)));
    CK(cudaMemset(c->d_fb, 0, 2 * sizeof(unsigned long long)));
  }
  c->mlp = m;
  c->fr_lo = (float)fr_lo;
  c->fr_hi = (float)fr_hi;
  adot_status st = read_ctl(c);
  if (st) return st;
  c->sur_steps0 = c->h_ctl->s[c->phase % 3].steps;
  CK(cudaMemcpy(&c->fb0, c->d_fb, sizeof(unsigned long long), cudaMemcpyDeviceToHost));
  return build_graph(c);
}

adot_status adot_surrogate_stats(adot_ctx* c, int64_t* edges_out, int64_t* fallback_out) {
  if (!c) return ADOT_E_INVALID_ARG;
  adot_status st = read_ctl(c);
  if (st) return st;
  unsigned long long fb = 0;
  if (c->d_fb) CK(cudaMemcpy(&fb, c->d_fb, sizeof(unsigned long long), cudaMemcpyDeviceToHost));
  const long long steps = c->h_ctl->s[c->phase % 3].steps - c->sur_steps0;
  if (edges_out) *edges_out = c->mlp ? steps * (c->p.n + 1) : 0;
  if (fallback_out) *fallback_out = (int64_t)(fb - c->fb0);
  return ADOT_OK;
}

adot_status adot_surrogate_eval(adot_ctx* c, float* absA, int on_device, int64_t* fallback_out) {
  if (!c || !c->mlp || !c->state_set) return ADOT_E_INVALID_ARG;
  CK(cudaMemsetAsync(c->d_fb + 1, 0, sizeof(unsigned long long), c->stream));
  CK(launch_mlp_edges(c->mlp, c->p, st32(c, c->cur), c->phase % 3, (float)c->cfg.law.Ag, c->fr_lo,
                      c->fr_hi, c->d_absA, c->d_fb + 1, c->stream));
  if (absA)
    CK(cudaMemcpyAsync(absA, c->d_absA, sizeof(float) * 9 * (size_t)(c->p.n + 1),
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  unsigned long long fb = 0;
  if (fallback_out)
    CK(cudaMemcpyAsync(&fb, c->d_fb + 1, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
  adot_status st = read_ctl(c);  // waits for the stream
  if (st) return st;
  if (fallback_out) *fallback_out = (int64_t)fb;
  return status_from_bits(c->h_ctl->status);
}

adot_status adot_harvest(adot_ctx* c, int64_t n, uint64_t seed, float* X, float* T, int on_device) {
  if (!c || !c->state_set || n < 0 || (n > 0 && (!X || !T))) return ADOT_E_INVALID_ARG;
  if (c->law != ADOT_LAW_GRASS) return ADOT_E_UNSUPPORTED;
  if (n == 0) return ADOT_OK;
  float* dX = X;
  float* dT = T;
  if (!on_device) {
    CK(cudaMalloc((void**)&dX, sizeof(float) * 7 * (size_t)n));
    if (cudaMalloc((void**)&dT, sizeof(float) * 9 * (size_t)n) != cudaSuccess) {
      cudaFree(dX);
      return ADOT_E_CUDA;
    }
  }
  const int slot = c->phase % 3;
  cudaError_t e;
  if (c->prec == ADOT_FP32)
    e = launch_harvest_f32(c->p, st32(c, c->cur), slot, n, seed, (float)c->cfg.law.Ag, dX, dT, c->stream);
  else
    e = launch_harvest_f64(c->p, st64(c, c->cur), slot, n, seed, (float)c->cfg.law.Ag, dX, dT, c->stream);
  if (e == cudaSuccess && !on_device) {
    e = cudaMemcpyAsync(X, dX, sizeof(float) * 7 * (size_t)n, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(T, dT, sizeof(float) * 9 * (size_t)n, cudaMemcpyDeviceToHost, c->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (!on_device) {
    cudaFree(dX);
    cudaFree(dT);
  }
  if (e != cudaSuccess) return ADOT_E_CUDA;
  adot_status st = read_ctl(c);
  if (st) return st;
  return status_from_bits(c->h_ctl->status);
}

adot_status adot_precision_stats(adot_ctx* c, int64_t* nodes_out, int64_t* fp64_nodes_out) {
  if (!c || !c->state_set) return ADOT_E_INVALID_ARG;
  const int64_t ne = c->p.periodic ? c->p.n : c->p.n + 1;
  unsigned long long redo = 0;
  if (c->prec == ADOT_FP32) {
    CK(cudaMemsetAsync(c->d_flrho, 0, sizeof(unsigned long long), c->stream));
    CK(launch_redo_count_f32(c->p, c->law, st32(c, c->cur), c->phase % 3, c->d_flrho, c->stream));
    CK(cudaMemcpyAsync(c->h_flrho, c->d_flrho, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    redo = c->h_flrho[0];
  }
  if (nodes_out) *nodes_out = 3 * ne;
  if (fp64_nodes_out) *fp64_nodes_out = (int64_t)redo;
  return ADOT_OK;
}

adot_status adot_conserved_sums(adot_ctx* c, double sums_out[3]) {
  if (!c || !sums_out) return ADOT_E_INVALID_ARG;
  if (c->prec == ADOT_FP32)
    CK(launch_sums_f32(st32(c, c->cur), c->p.n, c->d_partial, c->d_sums, c->stream));
  else
    CK(launch_sums_f64(st64(c, c->cur), c->p.n, c->d_partial, c->d_sums, c->stream));
  CK(cudaMemcpyAsync(c->h_sums, c->d_sums, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  for (int i = 0; i < 3; ++i) sums_out[i] = c->h_sums[i];
  return ADOT_OK;
}

}  // extern "C"
