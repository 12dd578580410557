// Batched ensemble of independent channels (adot_ensemble_*).
//
// Every channel is its own first-order DOT problem (Eq. scheme, Grass law with
// its own A_g, transmissive ends) with its own dt = cfl dx_c / rho_c. The
// channels' cells lie end to end in one state array. One launch advances every
// running channel by one of its own steps:
//  - channels are cut into tiles of B-1 cells (block kernel: B threads
//    evaluate B edges and update the B-1 cells between them, D+ through shared
//    memory) or of 16 x 31 cells (persistent warp tiles: one warp takes the
//    tile's 31-cell sub-tiles in turn, 32 lanes, D+ by shuffle, no block
//    barrier, one control evaluation and one CFL atomic per tile); the tile
//    list is ordered longest channel first;
//  - a fixed grid (resident blocks x SMs) walks the tiles [0, A), where A is
//    one past the last tile of any channel that was running at the start of
//    the previous step (set by device atomics), so finished short channels
//    drop out of the walk without a host round trip;
//  - each channel has three rotating control slots (t, dt, steps, CFL max);
//    the channel's first tile ("leader") writes the next slot, the other tiles
//    only read the current one and fold their CFL maxima in with atomicMax;
//  - a channel that has reached t_end copies its state across once (so both
//    ping-pong buffers hold it; the global step of that copy is kept in fin[c])
//    and is skipped from then on.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "../../include/adot.h"
#include "adot_step_impl.cuh"

namespace adot {

struct EnsDev {
  // per channel, [3][C] rotating slots
  double* t;
  double* dt;
  long long* steps;
  unsigned long long* rho;
  // per channel, latest values written by the leader
  double* t_cur;
  double* dt_cur;
  long long* steps_cur;
  long long* fin;  // global step of the copy step after t_end (LLONG_MAX before)
  // global
  long long* gstep;  // [3]
  int* active;       // [3] tile bound
  double* t_end;     // scalar
  unsigned* status;  // scalar
  int* next;         // channel queue head of the persistent form
};

struct EnsParams {
  int C;
  int64_t n_tiles;
  double cfl;
  float g_f;
  double g_d;
  const int64_t* off;   // [C+1]
  const double* dx;     // [C]
  const float* K3f;     // [C] 3 xi A_g
  const double* K3d;    // [C]
  const int* tile_chan; // [T]
  const int* tile_e0;   // [T] first edge of the tile within its channel
  const int* chan_tile_end;  // [C] one past the channel's last tile
  EnsDev d;
};

// Control of channel c for this launch, evaluated by one lane: the mode (0 step,
// 1 copy on the first launch after t_end, 2 skip), nu = dt/dx, and, on the
// channel's first tile ("leader"), the next control slot (as in k_ens_step).
template <typename R>
__device__ __forceinline__ int ens_control(const EnsParams& p, int c, bool leader, int slot, int nx,
                                           int pv, long long k, double t_end, R& nu) {
  const int C = p.C;
  int mode;
  const long long fin = p.d.fin[c];
  const double t = p.d.t[slot * C + c];
  double dt = 0.0;
  double tn = t;
  if (k > fin) {
    mode = 2;
  } else if (!(t < t_end)) {
    mode = 1;
  } else {
    mode = 0;
    const double rho = Prec<R>::from_bits(p.d.rho[slot * C + c]);
    dt = p.cfl * p.dx[c] / rho;
    tn = t + dt;
    if (tn >= t_end) {
      dt = t_end - t;
      tn = t_end;
    }
  }
  nu = (mode == 0) ? R(dt / p.dx[c]) : R(0);
  if (leader && mode != 2) {
    const long long st = p.d.steps[slot * C + c] + (mode == 0 ? 1 : 0);
    p.d.t[nx * C + c] = tn;
    p.d.dt[nx * C + c] = (mode == 0) ? dt : p.d.dt[slot * C + c];
    p.d.steps[nx * C + c] = st;
    p.d.rho[pv * C + c] = 0ull;
    p.d.t_cur[c] = tn;
    p.d.steps_cur[c] = st;
    if (mode == 0) {
      p.d.dt_cur[c] = dt;
      atomicMax(&p.d.active[nx], p.chan_tile_end[c]);
    } else {
      p.d.rho[nx * C + c] = p.d.rho[slot * C + c];
      p.d.fin[c] = k;
    }
  }
  return mode;
}

template <typename R, int B>
__global__ void __launch_bounds__(B, 65536 / (B * 64))
    k_ens_step(const EnsParams p, const typename Prec<R>::State in,
               const typename Prec<R>::State out, const int slot) {
  using S = typename Prec<R>::S;
  __shared__ R sDp[3][B];
  __shared__ R sRed[B / 32];
  __shared__ R sNu;
  __shared__ int sMode;  // 0 step, 1 copy (first step after t_end), 2 skip

  const int tid = threadIdx.x;
  const int C = p.C;
  const int nx = (slot + 1) % 3, pv = (slot + 2) % 3;
  const int A = p.d.active[slot];
  const long long k = p.d.gstep[slot];
  const double t_end = *p.d.t_end;
  if (blockIdx.x == 0 && tid == 0) {
    p.d.active[pv] = 0;
    p.d.gstep[nx] = k + 1;
  }
  unsigned flags = 0;
  for (int64_t tile = blockIdx.x; tile < A; tile += gridDim.x) {
    const int c = p.tile_chan[tile];
    const int64_t e0 = p.tile_e0[tile];
    const int64_t base = p.off[c];
    const int64_t nc = p.off[c + 1] - base;
    const int64_t e = e0 + tid;
    // states on both sides of edge e (cells e-1 and e of the channel; copies at the ends)
    S wl[3], wr[3];
    const bool valid = e <= nc;
    if (valid) {
      const int64_t il = (e > 0) ? e - 1 : 0;
      const int64_t ir = (e < nc) ? e : nc - 1;
      wl[0] = in.h[base + il];
      wl[1] = in.q[base + il];
      wl[2] = in.z[base + il];
      wr[0] = in.h[base + ir];
      wr[1] = in.q[base + ir];
      wr[2] = in.z[base + ir];
    }
    if (tid == 0) {
      R nu = R(0);
      sMode = ens_control<R>(p, c, e0 == 0, slot, nx, pv, k, t_end, nu);
      sNu = nu;
    }
    __syncthreads();
    const int mode = sMode;
    const R nu = sNu;
    if (mode == 2) {
      __syncthreads();
      continue;
    }
    const int64_t i = e - 1;  // cell updated by this thread
    if (mode == 1) {
      if (tid >= 1 && i < nc) {
        out.h[base + i] = wl[0];
        out.q[base + i] = wl[1];
        out.z[base + i] = wl[2];
      }
      __syncthreads();
      continue;
    }
    StepParams lp;
    lp.lf = LawT<float>{p.g_f, p.K3f[c], 0.0f, 0.0f};
    lp.ld = LawT<double>{p.g_d, p.K3d[c], 0.0, 0.0};
    R dm[3] = {R(0), R(0), R(0)}, dp[3] = {R(0), R(0), R(0)};
    if (valid && e > 0 && e < nc) edge_fluct<R, LAW_GRASS, false>(lp, wl, wr, dm, dp, flags);
    sDp[0][tid] = dp[0];
    sDp[1][tid] = dp[1];
    sDp[2][tid] = dp[2];
    __syncthreads();
    R rho = R(0);
    if (tid >= 1 && i < nc) {
      const S nh = Prec<R>::add(wl[0], -nu * (dm[0] + sDp[0][tid - 1]));
      const S nq = Prec<R>::add(wl[1], -nu * (dm[1] + sDp[1][tid - 1]));
      const S nz = Prec<R>::add(wl[2], -nu * (dm[2] + sDp[2][tid - 1]));
      out.h[base + i] = nh;
      out.q[base + i] = nq;
      out.z[base + i] = nz;
      const R hh = Prec<R>::hi(nh);
      if (!(hh > R(0))) flags |= ST_DEPTH;
      if (!(Prec<R>::finite(nh) && Prec<R>::finite(nq) && Prec<R>::finite(nz))) {
        flags |= ST_NONFINITE;
      } else if (hh > R(0)) {
        rho = Prec<R>::template rho<LAW_GRASS>(lp, hh, Prec<R>::hi(nq));
        if (!(rho <= R(3.0e38))) {
          flags |= ST_NONFINITE;
          rho = R(0);
        }
      }
    }
    rho = warp_max(rho);
    if ((tid & 31) == 0) sRed[tid >> 5] = rho;
    __syncthreads();
    if (tid < 32) {
      rho = (tid < B / 32) ? sRed[tid] : R(0);
      rho = warp_max(rho);
      if (tid == 0 && rho > R(0)) atomicMax(&p.d.rho[nx * C + c], Prec<R>::bits(rho));
    }
  }
  if (flags) atomicOr(p.d.status, flags);
}

// One sub-tile of a channel: lane l evaluates edge e0 + l (cells e0 + l - 1
// and e0 + l, copies at the ends) and lanes 1..31 update cells e0 .. e0 + 30
// with D+ of the left edge by shuffle. mode 0 steps with nu = dt/dx and folds
// the new cells' CFL maxima into rho; mode 1 copies the cells across.
// State load: plain (L1-cached) or, when other SMs write the cells between
// steps of one launch (a cluster team), at L2 only.
template <bool CG, typename T>
__device__ __forceinline__ T ens_ld(const T* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

template <typename R, int CAP, bool CG = false>
__device__ __forceinline__ void ens_subtile(const StepParams& lp, const typename Prec<R>::State& in,
                                            const typename Prec<R>::State& out, const int64_t base,
                                            const int64_t nc, const int64_t e0, const int lane,
                                            const R nu, const int mode, R& rho, unsigned& flags) {
  using S = typename Prec<R>::S;
  const int64_t e = e0 + lane;
    // states of edge e: cells e-1 and e, each lane loading both (a right
    // state taken from the next lane by shuffle measured 4 % slower: every
    // lane then waits for its neighbour's load); transmissive ends copy the
    // adjacent cell, lanes past the channel's end read its last cell
    const bool valid = e <= nc;
    S wl[3], wr[3];
    const int64_t il = (e > 0) ? (e <= nc ? e - 1 : nc - 1) : 0;
    const int64_t ir = (e < nc) ? e : nc - 1;
    wl[0] = ens_ld<CG>(in.h + base + il);
    wl[1] = ens_ld<CG>(in.q + base + il);
    wl[2] = ens_ld<CG>(in.z + base + il);
    wr[0] = ens_ld<CG>(in.h + base + ir);
    wr[1] = ens_ld<CG>(in.q + base + ir);
    wr[2] = ens_ld<CG>(in.z + base + ir);
    const int64_t i = e - 1;  // cell updated by this lane (lanes 1..31)
    if (mode == 1) {
      if (lane >= 1 && i < nc) {
        out.h[base + i] = wl[0];
        out.q[base + i] = wl[1];
        out.z[base + i] = wl[2];
      }
      return;
    }
    R dm[3] = {R(0), R(0), R(0)}, dp[3] = {R(0), R(0), R(0)};
    // the paired-node float32 form where the register cap leaves it room
    if (valid && e > 0 && e < nc) edge_fluct<R, LAW_GRASS, (CAP >= 80)>(lp, wl, wr, dm, dp, flags);
    R dpl[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) dpl[r] = __shfl_up_sync(0xffffffffu, dp[r], 1);
    if (lane >= 1 && i < nc) {
      const S nh = Prec<R>::add(wl[0], -nu * (dm[0] + dpl[0]));
      const S nq = Prec<R>::add(wl[1], -nu * (dm[1] + dpl[1]));
      const S nz = Prec<R>::add(wl[2], -nu * (dm[2] + dpl[2]));
      out.h[base + i] = nh;
      out.q[base + i] = nq;
      out.z[base + i] = nz;
      const R hh = Prec<R>::hi(nh);
      if (!(hh > R(0))) flags |= ST_DEPTH;
      if (!(Prec<R>::finite(nh) && Prec<R>::finite(nq) && Prec<R>::finite(nz))) {
        flags |= ST_NONFINITE;
      } else if (hh > R(0)) {
        R r = Prec<R>::template rho<LAW_GRASS>(lp, hh, Prec<R>::hi(nq));
        if (!(r <= R(3.0e38))) {
          flags |= ST_NONFINITE;
          r = R(0);
        }
        rho = r > rho ? r : rho;
      }
    }
}

// A contiguous range of one channel's edges in chunks of 32 (as the
// single-channel warp kernel): lane l of the chunk starting at edge eb
// evaluates edge eb + l and updates cell eb + l - 1 with D+ of the previous
// edge from lane l - 1, or in lane 0 carried over from lane 31 of the previous
// chunk; rem = edges of the range after its first (the first edge's cell is
// not updated). The ends copy the adjacent cell (transmissive), so the end
// edges carry no fluctuation.
template <typename R, int CAP, bool CG = false>
__device__ __forceinline__ void ens_range(const StepParams& lp, const typename Prec<R>::State& in,
                                          const typename Prec<R>::State& out, const int64_t base,
                                          const int64_t nc, const int64_t e0, int rem, const R nu, R& rho,
                                          unsigned& flags) {
  using S = typename Prec<R>::S;
  const int lane = threadIdx.x & 31;
  R carry[3] = {R(0), R(0), R(0)};
  bool lead = lane >= 1;
  for (int64_t eb = e0; rem >= 0; eb += 32, rem -= 32) {
    const int64_t e = eb + lane;
    const bool in_range = lane <= rem;
    S wl[3];
    R dm[3] = {R(0), R(0), R(0)}, dp[3] = {R(0), R(0), R(0)};
    if (in_range) {
      S wr[3];
      const int64_t il = (e > 0) ? e - 1 : 0;
      const int64_t ir = (e < nc) ? e : nc - 1;
      wl[0] = ens_ld<CG>(in.h + base + il);
      wl[1] = ens_ld<CG>(in.q + base + il);
      wl[2] = ens_ld<CG>(in.z + base + il);
      wr[0] = ens_ld<CG>(in.h + base + ir);
      wr[1] = ens_ld<CG>(in.q + base + ir);
      wr[2] = ens_ld<CG>(in.z + base + ir);
      if (e > 0 && e < nc) edge_fluct<R, LAW_GRASS, (CAP >= 80)>(lp, wl, wr, dm, dp, flags);
    }
    R dl[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const R up = __shfl_sync(0xffffffffu, dp[r], (lane + 31) & 31);
      dl[r] = lane ? up : carry[r];
      carry[r] = up;  // lane 0: D+ of this chunk's last edge
    }
    if (lead && in_range) {
      const int64_t i = e - 1;
      const S nh = Prec<R>::add(wl[0], -nu * (dm[0] + dl[0]));
      const S nq = Prec<R>::add(wl[1], -nu * (dm[1] + dl[1]));
      const S nz = Prec<R>::add(wl[2], -nu * (dm[2] + dl[2]));
      out.h[base + i] = nh;
      out.q[base + i] = nq;
      out.z[base + i] = nz;
      const R hh = Prec<R>::hi(nh);
      if (!(hh > R(0))) flags |= ST_DEPTH;
      if (!(Prec<R>::finite(nh) && Prec<R>::finite(nq) && Prec<R>::finite(nz))) {
        flags |= ST_NONFINITE;
      } else if (hh > R(0)) {
        R v = Prec<R>::template rho<LAW_GRASS>(lp, hh, Prec<R>::hi(nq));
        if (!(v <= R(3.0e38))) {
          flags |= ST_NONFINITE;
          v = R(0);
        }
        rho = v > rho ? v : rho;
      }
    }
    lead = true;
  }
}

// One step of a channel of nc cells by `nw` warps (warp index w): the edges
// 0 .. nc in contiguous ranges of whole chunks, one per active warp (at least
// 31 cells each), consecutive ranges sharing one edge.
template <typename R, int CAP, bool CG = false>
__device__ __forceinline__ void ens_channel_sweep(const StepParams& lp, const typename Prec<R>::State& in,
                                                  const typename Prec<R>::State& out, const int64_t base,
                                                  const int64_t nc, const int64_t w, const int64_t nw,
                                                  const R nu, R& rho, unsigned& flags) {
  const int64_t nact = (nw < (nc + 30) / 31) ? nw : (nc + 30) / 31;
  if (w >= nact) return;
  const int64_t K = (nc + nact + 31) / 32;
  const int64_t kb = K / nact, kr = K % nact;
  const int64_t kw = kb + (w < kr ? 1 : 0);
  const int64_t e0 = 32 * (w * kb + (w < kr ? w : kr)) - w;
  const int64_t last = (e0 + 32 * kw - 1 < nc) ? e0 + 32 * kw - 1 : nc;
  ens_range<R, CAP, CG>(lp, in, out, base, nc, e0, (int)(last - e0), nu, rho, flags);
}

// Persistent warp tiles: each warp walks tiles of SUB x 31 cells of one
// channel (tile list in those units, longest channel first) with a grid-wide
// stride over the active bound. Lane 0 evaluates the channel's control once per
// tile and broadcasts it; the warp then takes the tile's SUB sub-tiles of 32
// edges / 31 cells in turn: lane l evaluates edge e0 + l and D+ of the left
// edge comes by shuffle, so no block barrier is taken. One CFL atomic per tile.
template <typename R, int B, int CAP, int SUB>
__global__ void __launch_bounds__(B, 65536 / (B * CAP))
    k_ens_step_warp(const EnsParams p, const typename Prec<R>::State in,
                    const typename Prec<R>::State out, const int slot) {
  const int lane = threadIdx.x & 31;
  const int C = p.C;
  const int nx = (slot + 1) % 3, pv = (slot + 2) % 3;
  const int A = p.d.active[slot];
  const long long k = p.d.gstep[slot];
  const double t_end = *p.d.t_end;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    p.d.active[pv] = 0;
    p.d.gstep[nx] = k + 1;
  }
  const int64_t warp0 = ((int64_t)blockIdx.x * B + threadIdx.x) >> 5;
  const int64_t n_warps = ((int64_t)gridDim.x * B) >> 5;
  unsigned flags = 0;
  for (int64_t tile = warp0; tile < A; tile += n_warps) {
    const int c = p.tile_chan[tile];
    const int64_t t0 = p.tile_e0[tile];
    const int64_t base = p.off[c];
    const int64_t nc = p.off[c + 1] - base;
    R nu = R(0);
    int mode = 0;
    if (lane == 0) mode = ens_control<R>(p, c, t0 == 0, slot, nx, pv, k, t_end, nu);
    mode = __shfl_sync(0xffffffffu, mode, 0);
    nu = __shfl_sync(0xffffffffu, nu, 0);
    if (mode == 2) continue;
    StepParams lp;
    lp.lf = LawT<float>{p.g_f, p.K3f[c], 0.0f, 0.0f};
    lp.ld = LawT<double>{p.g_d, p.K3d[c], 0.0, 0.0};
    R rho = R(0);
#pragma unroll 1
    for (int sub = 0; sub < SUB; ++sub) {
      const int64_t e0 = t0 + sub * 31;
      if (e0 >= nc) break;  // past the channel's last cell (warp-uniform)
      {
        const int64_t cn = e0 + 31 + lane;  // the next sub-tile's cells into L2 (+1.5 %)
        if (sub + 1 < SUB && cn < nc) {
          asm volatile("prefetch.global.L2 [%0];" ::"l"(in.h + base + cn));
          asm volatile("prefetch.global.L2 [%0];" ::"l"(in.q + base + cn));
          asm volatile("prefetch.global.L2 [%0];" ::"l"(in.z + base + cn));
        }
      }
      ens_subtile<R, CAP>(lp, in, out, base, nc, e0, lane, nu, mode, rho, flags);
    }
    if (mode == 0) {
      rho = warp_max(rho);
      if (lane == 0 && rho > R(0)) atomicMax(&p.d.rho[nx * C + c], Prec<R>::bits(rho));
    }
  }
  if (flags) atomicOr(p.d.status, flags);
}

// Persistent form (one launch per run_to chunk). Each CTA takes whole channels
// from a device queue, largest estimated work first (order[]; the head *next is
// zeroed by the host before the launch), and advances each one alone: the CFL
// maximum of its state, then up to max_steps of its own steps (dt and the
// landing on t_end exactly as ens_control), the CTA's warps taking the
// channel's 31-cell sub-tiles in turn and one block barrier (the CFL maximum of
// the new state) between steps. No CTA waits on another. When the channel
// stops, its state is copied into the other ping-pong buffer (so that both
// hold it) and its control is left as the per-step launches read it at slot
// `slot`: finished channels (t >= t_end) marked as copied before step
// gstep[slot], running ones added to the tile bound active[slot]. A non-finite
// value or non-positive depth (this CTA's or any other's, read from the status
// word) stops the channel after its step and the CTA takes no further channel.
struct EnsRun {
  const int* order;  // [C] channels, largest estimated work first
  int* next;         // queue head
  double t_end;
  long long max_steps;
  int slot;
};

template <typename R, int NW>
__device__ __forceinline__ R block_max(R v, R* red) {
  v = warp_max(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  R m = red[0];
#pragma unroll
  for (int w = 1; w < NW; ++w) m = d_max(m, red[w]);
  return m;
}

// One CTA steps channel c of the persistent form to t_end (at most max_steps
// steps), copies its state into the other buffer and leaves its control at
// slot `slot` (see k_ens_run). Returns whether a non-finite value or
// non-positive depth was met (the CTA then takes no further channel); the
// status bits stay in flags.
template <typename R, int B, int CAP>
__device__ __forceinline__ bool ens_run_channel(const EnsParams& p, const typename Prec<R>::State& b0,
                                                const typename Prec<R>::State& b1, const int c,
                                                const double t_end, const long long max_steps,
                                                const int slot, R* sRed, unsigned& flags) {
  constexpr int NW = B / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int C = p.C;
  const int64_t base = p.off[c];
  const int64_t nc = p.off[c + 1] - base;
  StepParams lp;
  lp.lf = LawT<float>{p.g_f, p.K3f[c], 0.0f, 0.0f};
  lp.ld = LawT<double>{p.g_d, p.K3d[c], 0.0, 0.0};
  // CFL maximum of the channel's current state (as k_ens_rho)
  R rho = R(0);
  for (int64_t i = threadIdx.x; i < nc; i += B) {
    const auto h = b0.h[base + i], q = b0.q[base + i], z = b0.z[base + i];
    const R hh = Prec<R>::hi(h);
    if (!(Prec<R>::finite(h) && Prec<R>::finite(q) && Prec<R>::finite(z))) {
      flags |= ST_NONFINITE;
      continue;
    }
    if (!(hh > R(0))) {
      flags |= ST_DEPTH;
      continue;
    }
    const R v = Prec<R>::template rho<LAW_GRASS>(lp, hh, Prec<R>::hi(q));
    if (!(v <= R(3.0e38))) {
      flags |= ST_NONFINITE;
      continue;
    }
    rho = d_max(rho, v);
  }
  rho = block_max<R, NW>(rho, sRed);
  double t = p.d.t_cur[c];
  long long st = p.d.steps_cur[c];
  double dt_last = p.d.dt_cur[c];
  const double dx = p.dx[c];
  int cur = 0;
  bool stop = __syncthreads_or(flags != 0 || (threadIdx.x == 0 && *(volatile unsigned*)p.d.status != 0));
  for (long long ns = 0; !stop && t < t_end && ns < max_steps; ++ns) {
    double dt = p.cfl * dx / (double)rho;
    double tn = t + dt;
    if (tn >= t_end) {
      dt = t_end - t;
      tn = t_end;
    }
    const R nu = R(dt / dx);
    const typename Prec<R>::State& in = cur ? b1 : b0;
    const typename Prec<R>::State& out = cur ? b0 : b1;
    R rr = R(0);
    ens_channel_sweep<R, CAP>(lp, in, out, base, nc, warp, NW, nu, rr, flags);
    rho = block_max<R, NW>(rr, sRed);
    t = tn;
    ++st;
    dt_last = dt;
    cur ^= 1;
    stop = __syncthreads_or(flags != 0 || (threadIdx.x == 0 && *(volatile unsigned*)p.d.status != 0));
  }
  // both buffers hold the channel's state
  {
    const typename Prec<R>::State& src = cur ? b1 : b0;
    const typename Prec<R>::State& dst = cur ? b0 : b1;
    for (int64_t i = threadIdx.x; i < nc; i += B) {
      dst.h[base + i] = src.h[base + i];
      dst.q[base + i] = src.q[base + i];
      dst.z[base + i] = src.z[base + i];
    }
  }
  if (threadIdx.x == 0) {
    const int s0 = slot, s1 = (slot + 1) % 3;
    p.d.t[s0 * C + c] = t;
    p.d.dt[s0 * C + c] = dt_last;
    p.d.steps[s0 * C + c] = st;
    p.d.rho[s0 * C + c] = rho > R(0) ? Prec<R>::bits(rho) : 0ull;
    p.d.rho[s1 * C + c] = 0ull;
    p.d.t_cur[c] = t;
    p.d.steps_cur[c] = st;
    p.d.dt_cur[c] = dt_last;
    const bool done = !(t < t_end);
    p.d.fin[c] = done ? p.d.gstep[s0] - 1 : 0x7fffffffffffffffLL;
    if (!done) atomicMax(&p.d.active[s0], p.chan_tile_end[c]);
  }
  return stop;
}

template <typename R, int B, int CAP>
__global__ void __launch_bounds__(B, 65536 / (B * CAP))
    k_ens_run(const EnsParams p, const typename Prec<R>::State b0, const typename Prec<R>::State b1,
              const EnsRun r) {
  constexpr int NW = B / 32;
  __shared__ R sRed[NW];
  __shared__ int sJ;
  unsigned flags = 0;
  bool stop = false;
  while (!stop) {
    __syncthreads();
    if (threadIdx.x == 0) sJ = atomicAdd(r.next, 1);
    __syncthreads();
    const int j = sJ;
    if (j >= p.C) break;
    stop = ens_run_channel<R, B, CAP>(p, b0, b1, r.order[j], r.t_end, r.max_steps, r.slot, sRed, flags);
    if (flags) {
      atomicOr(p.d.status, flags);
      flags = 0;
    }
  }
}

// ---- cluster teams: a long channel stepped by the CTAs of one cluster -------
// Thread block clusters of CL CTAs (one CTA of 768 threads per SM). For each of
// its assigned long channels a cluster steps the channel as one team: the CL x
// 24 warps take the channel's 31-cell sub-tiles in turn, and each step ends
// with a team exchange of the CFL maximum and an error bit. Each CTA writes its
// value into its own shared memory (double-buffered by step parity), arrives
// on every team member's mbarrier through distributed shared memory (release
// at cluster scope, after a block barrier and a device fence that order the
// step's cell writes), waits on its own (acquire; at most ~2^31 cycles, then
// the team aborts with ST_TIMEOUT) and reads the members' values remotely.
// A member can run at most one exchange ahead of another (it needs every
// member's arrival to finish an exchange), so the two value buffers and the
// barrier's phase parity suffice. Team members read cells that other SMs wrote
// in the previous step, so their state loads bypass L1 (ld.global.cg). Every
// decision that shapes the control flow (the channel list, t, dt, the step
// count, the stop bit) is the same in all members, so all of them make the
// same exchanges. After the long channels each CTA takes the short ones from
// the dynamic queue alone (ens_run_channel), and a final cluster barrier keeps
// every CTA's shared memory alive until no member can read it.

__device__ __forceinline__ uint32_t cl_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cl_id() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t sh_addr(const void* ptr) {
  return (uint32_t)__cvta_generic_to_shared(ptr);
}
// address of the same shared-memory variable in cluster CTA `rank`
__device__ __forceinline__ uint32_t cl_map(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
// all threads of every CTA of the cluster
__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

struct EnsTeamRun {
  const int* big_ptr;   // [clusters + 1]: cluster k runs big_list[big_ptr[k] .. big_ptr[k+1])
  const int* big_list;  // the long channels, cluster by cluster
  const int* order;     // [n_small] the other channels, largest estimated work first
  int n_small;
  int* next;            // queue head of those
  double t_end;
  long long max_steps;
  int slot;
  int fault;  // test hook: 1 = cluster 0's CTA 1 does not arrive at its first exchange
};

struct TeamSmem {
  uint64_t bar;                    // CL arrivals per exchange
  unsigned long long val[2][2];    // [parity][rho bits, stop bit] of this CTA
  unsigned long long out_rho;      // the exchange's results, for the whole CTA
  int out_stop;                    // 0 go on, 1 stop (an error bit), 2 timed out
};

// Thread 0: publishes (rho_bits, stop) for exchange k, arrives at every member,
// waits for all of them and combines; false if the wait ran out.
template <int CL>
__device__ __forceinline__ bool team_exchange(TeamSmem& ts, int k, unsigned long long rho_bits,
                                              unsigned long long stop, unsigned long long& rmax,
                                              unsigned long long& sany, bool withhold) {
  const int par = k & 1;
  ts.val[par][0] = rho_bits;
  ts.val[par][1] = stop;
  __threadfence();
  const uint32_t bar = sh_addr(&ts.bar);
  if (!withhold) {
#pragma unroll
    for (int q = 0; q < CL; ++q)
      asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cl_map(bar, (uint32_t)q))
                   : "memory");
  }
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"((uint32_t)par)
        : "memory");
    if (done) break;
    if (clock64() - t0 > (1ll << 31)) return false;
  }
  __threadfence();
  rmax = 0ull;
  sany = 0ull;
  const uint32_t va = sh_addr(&ts.val[par][0]);
#pragma unroll
  for (int q = 0; q < CL; ++q) {
    const uint32_t ra = cl_map(va, (uint32_t)q);
    unsigned long long a, b;
    asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(a) : "r"(ra) : "memory");
    asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(b) : "r"(ra + 8u) : "memory");
    rmax = a > rmax ? a : rmax;
    sany |= b;
  }
  return true;
}

template <typename R, int B, int CAP, int CL>
__global__ void __launch_bounds__(B, 65536 / (B * CAP))
    k_ens_run_team(const EnsParams p, const typename Prec<R>::State b0, const typename Prec<R>::State b1,
                   const EnsTeamRun r) {
  constexpr int NW = B / 32;
  __shared__ R sRed[NW];
  __shared__ int sJ;
  __shared__ __align__(16) TeamSmem ts;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t rank = cl_rank();
  const int C = p.C;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sh_addr(&ts.bar)), "r"(CL) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  cl_sync();  // every member's barrier is initialised before anyone arrives
  unsigned flags = 0;
  bool quit = false;
  int xk = 0;  // exchanges so far
  const uint32_t cid = cl_id();
  // team exchange of this CTA's (rho, error) by all threads; results in ts
  auto exchange = [&](R rho_cta, bool err) {
    if (threadIdx.x == 0) {
      unsigned long long rm = 0ull, sa = 0ull;
      const bool st_err = err || *(volatile unsigned*)p.d.status != 0;
      const bool withhold = r.fault == 1 && cid == 0 && rank == 1 && xk == 0;
      if (!team_exchange<CL>(ts, xk, rho_cta > R(0) ? Prec<R>::bits(rho_cta) : 0ull, st_err ? 1ull : 0ull, rm,
                             sa, withhold)) {
        atomicOr(p.d.status, ST_TIMEOUT);
        ts.out_stop = 2;
      } else {
        ts.out_rho = rm;
        ts.out_stop = sa ? 1 : 0;
      }
    }
    ++xk;
    __syncthreads();
  };

  for (int k = r.big_ptr[cid]; !quit && k < r.big_ptr[cid + 1]; ++k) {
    const int c = r.big_list[k];
    const int64_t base = p.off[c];
    const int64_t nc = p.off[c + 1] - base;
    StepParams lp;
    lp.lf = LawT<float>{p.g_f, p.K3f[c], 0.0f, 0.0f};
    lp.ld = LawT<double>{p.g_d, p.K3d[c], 0.0, 0.0};
    // CFL maximum of the current state over this member's cells
    R rho = R(0);
    for (int64_t i = (int64_t)rank * B + threadIdx.x; i < nc; i += (int64_t)CL * B) {
      const auto h = ens_ld<true>(b0.h + base + i), q = ens_ld<true>(b0.q + base + i),
                 z = ens_ld<true>(b0.z + base + i);
      const R hh = Prec<R>::hi(h);
      if (!(Prec<R>::finite(h) && Prec<R>::finite(q) && Prec<R>::finite(z))) {
        flags |= ST_NONFINITE;
        continue;
      }
      if (!(hh > R(0))) {
        flags |= ST_DEPTH;
        continue;
      }
      const R v = Prec<R>::template rho<LAW_GRASS>(lp, hh, Prec<R>::hi(q));
      if (!(v <= R(3.0e38))) {
        flags |= ST_NONFINITE;
        continue;
      }
      rho = d_max(rho, v);
    }
    rho = block_max<R, NW>(rho, sRed);
    exchange(rho, __syncthreads_or(flags != 0));
    int stop = ts.out_stop;
    rho = (R)Prec<R>::from_bits(ts.out_rho);
    double t = p.d.t_cur[c];
    long long st = p.d.steps_cur[c];
    double dt_last = p.d.dt_cur[c];
    const double dx = p.dx[c];
    int cur = 0;
    for (long long ns = 0; stop == 0 && t < r.t_end && ns < r.max_steps; ++ns) {
      double dt = p.cfl * dx / (double)rho;
      double tn = t + dt;
      if (tn >= r.t_end) {
        dt = r.t_end - t;
        tn = r.t_end;
      }
      const R nu = R(dt / dx);
      const typename Prec<R>::State& in = cur ? b1 : b0;
      const typename Prec<R>::State& out = cur ? b0 : b1;
      R rr = R(0);
      ens_channel_sweep<R, CAP, true>(lp, in, out, base, nc, (int64_t)rank * NW + warp, (int64_t)CL * NW, nu,
                                      rr, flags);
      rr = block_max<R, NW>(rr, sRed);
      exchange(rr, __syncthreads_or(flags != 0));
      stop = ts.out_stop;
      rho = (R)Prec<R>::from_bits(ts.out_rho);
      t = tn;
      ++st;
      dt_last = dt;
      cur ^= 1;
    }
    if (stop == 2) {
      quit = true;
      break;
    }
    // both buffers hold the channel's state (each member copies its own cells)
    {
      const typename Prec<R>::State& src = cur ? b1 : b0;
      const typename Prec<R>::State& dst = cur ? b0 : b1;
      for (int64_t i = (int64_t)rank * B + threadIdx.x; i < nc; i += (int64_t)CL * B) {
        dst.h[base + i] = ens_ld<true>(src.h + base + i);
        dst.q[base + i] = ens_ld<true>(src.q + base + i);
        dst.z[base + i] = ens_ld<true>(src.z + base + i);
      }
    }
    if (rank == 0 && threadIdx.x == 0) {
      const int s0 = r.slot, s1 = (r.slot + 1) % 3;
      p.d.t[s0 * C + c] = t;
      p.d.dt[s0 * C + c] = dt_last;
      p.d.steps[s0 * C + c] = st;
      p.d.rho[s0 * C + c] = rho > R(0) ? Prec<R>::bits(rho) : 0ull;
      p.d.rho[s1 * C + c] = 0ull;
      p.d.t_cur[c] = t;
      p.d.steps_cur[c] = st;
      p.d.dt_cur[c] = dt_last;
      const bool done = !(t < r.t_end);
      p.d.fin[c] = done ? p.d.gstep[s0] - 1 : 0x7fffffffffffffffLL;
      if (!done) atomicMax(&p.d.active[s0], p.chan_tile_end[c]);
    }
    if (stop) quit = true;
  }
  // the short channels, one CTA each
  while (!quit) {
    __syncthreads();
    if (threadIdx.x == 0) sJ = atomicAdd(r.next, 1);
    __syncthreads();
    const int j = sJ;
    if (j >= r.n_small) break;
    quit = ens_run_channel<R, B, CAP>(p, b0, b1, r.order[j], r.t_end, r.max_steps, r.slot, sRed, flags);
  }
  if (flags) atomicOr(p.d.status, flags);
  cl_sync();  // no member reads this CTA's shared memory after it exits
}


// Initial CFL maxima of every channel into slot 0 (grid-stride over cells).
template <typename R>
__global__ void __launch_bounds__(256) k_ens_rho(const EnsParams p, const typename Prec<R>::State st,
                                                  int64_t n_total) {
  unsigned flags = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_total;
       i += (int64_t)gridDim.x * blockDim.x) {
    // channel of cell i by binary search over the offsets
    int lo = 0, hi = p.C - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (p.off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    const int c = lo;
    const auto h = st.h[i], q = st.q[i], z = st.z[i];
    const R hh = Prec<R>::hi(h);
    if (!(Prec<R>::finite(h) && Prec<R>::finite(q) && Prec<R>::finite(z))) {
      flags |= ST_NONFINITE;
      continue;
    }
    if (!(hh > R(0))) {
      flags |= ST_DEPTH;
      continue;
    }
    StepParams lp;
    lp.lf = LawT<float>{p.g_f, p.K3f[c], 0.0f, 0.0f};
    lp.ld = LawT<double>{p.g_d, p.K3d[c], 0.0, 0.0};
    const R r = Prec<R>::template rho<LAW_GRASS>(lp, hh, Prec<R>::hi(q));
    if (!(r <= R(3.0e38))) {
      flags |= ST_NONFINITE;
      continue;
    }
    atomicMax(&p.d.rho[c], Prec<R>::bits(r));
  }
  if (flags) atomicOr(p.d.status, flags);
}

}  // namespace adot

using namespace adot;

namespace {

// Step kernel variants: block kernel (tile = block - 1 cells, 64-register cap)
// or persistent warp tiles (31 cells per tile) at a register cap.
struct EnsVariant {
  int block;
  int cap;
  bool warp;
};
constexpr EnsVariant kEnsVariants[] = {{256, 64, false}, {128, 64, false}, {512, 64, false},
                                       {256, 64, true},  {256, 80, true}};
constexpr int kNumEnsVariants = sizeof(kEnsVariants) / sizeof(kEnsVariants[0]);
// Threads per CTA of the persistent form when block_threads = 0: on the 4096-channel
// ensemble (float32, N_c log-uniform in [1e3, 1e5], t_end 0.02 and 0.1 s) 256 x 80:
// 3.99e10, 384 x 80: 5.12e10, 512 x 64: 4.6-4.7e10 cell-updates/s (per-step warp
// tiles: 4.36e10). With 256 threads the 456 CTAs hold less work each than the
// largest channel alone.
constexpr int kRunBlockDefault = 384;
// Persistent shapes tried when block_threads = 0 (threads, register cap), and the
// per-step form's measured speed relative to a balanced persistent run (4.36e10
// against 5.13e10 cell-updates/s): the per-step form is used when the persistent
// form's estimated imbalance exceeds 1 / kPerStepRel.
constexpr int kRunBlocks[] = {384, 768};
constexpr int kNumRunBlocks = 2;
constexpr double kPerStepRel = 0.85;
// 31-cell sub-tiles per warp tile (one control evaluation each; on the 4096-channel
// ensemble with scalar nodes 4: 2.99e10, 8: 3.15e10, 16: 3.19e10 cell-updates/s)
constexpr int kEnsSub = 16;

struct HostCtl {
  long long gstep[3];
  int active[3];
  unsigned status;
};

}  // namespace

struct adot_ensemble {
  int C;
  int prec;
  int device;
  int block;
  int cap;       // register cap of the warp-tile kernel
  bool warp;     // persistent warp tiles (31 cells) instead of block tiles (block - 1 cells)
  int step_kernel_cfg;  // 0 chosen per state, 1 block, 2 warp tiles, 3 persistent, 4 per-step autotuned
  int run_block_cfg;    // configured threads per CTA of the persistent form (0 = chosen)
  int n_sms;
  int run_occ[kNumRunBlocks];  // resident CTAs per SM of each persistent shape
  // how run_to (plan[0]) and step (plan[1]) advance the channels
  struct Plan {
    bool persistent;
    int block;       // threads per CTA of k_ens_run / k_ens_run_team
    int grid;        // resident CTAs (at most one per channel without teams)
    double imbalance;  // estimated list-scheduling makespan / mean CTA load
    int* d_order;    // [C] channel queue (the short channels with teams), largest estimated work first
    int cluster;     // 1: one CTA per channel; 2 or 4: long channels stepped by cluster teams
    int n_big;       // channels run by teams
    int n_small;     // channels in the queue
    int* d_team;     // [clusters + 1 + C]: big_ptr, then big_list
  } plan[2];
  int team_clusters[2];  // resident clusters of k_ens_run_team with 2 and 4 CTAs (0: not launchable)
  int fault;             // test hook for the next team launch (adot_ensemble_inject_fault)
  int block_cfg;        // configured block_threads (0 = any)
  bool tuned;
  int steps_per_graph;
  double cfl, g, xi;
  int64_t n_total;
  std::vector<int64_t> n_cells;
  std::vector<int64_t> off;
  std::vector<int> order;  // channels, longest first
  std::vector<double> length;
  cudaStream_t stream;
  bool own_stream;
  cudaStream_t cap_stream;
  // device
  void* buf[2][3];
  int cur;
  int phase;
  int64_t* d_off;
  double* d_dx;
  float* d_K3f;
  double* d_K3d;
  int* d_tile_chan;
  int* d_tile_e0;
  int* d_chan_tile_end;
  int64_t n_tiles;
  int grid;
  void* d_ctl_mem;  // all EnsDev arrays in one allocation
  size_t ctl_bytes;
  EnsDev dev;
  double* d_io;
  cudaGraphExec_t graph;
  bool graph_ready;
  bool state_set;
  double t_end_dev;
};

namespace {

#define CKE(expr)                               \
  do {                                          \
    cudaError_t _e = (expr);                    \
    if (_e != cudaSuccess) return ADOT_E_CUDA;  \
  } while (0)

adot_status ens_status(unsigned bits) {
  if (bits & ST_NONFINITE) return ADOT_E_NONFINITE;
  if (bits & ST_DEPTH) return ADOT_E_NONPOSITIVE_DEPTH;
  if (bits & ST_NONHYPERBOLIC) return ADOT_E_NONHYPERBOLIC;
  if (bits & ST_TIMEOUT) return ADOT_E_TIMEOUT;
  return ADOT_OK;
}

EnsParams ens_params(const adot_ensemble* e) {
  EnsParams p;
  p.C = e->C;
  p.n_tiles = e->n_tiles;
  p.cfl = e->cfl;
  p.g_f = (float)e->g;
  p.g_d = e->g;
  p.off = e->d_off;
  p.dx = e->d_dx;
  p.K3f = e->d_K3f;
  p.K3d = e->d_K3d;
  p.tile_chan = e->d_tile_chan;
  p.tile_e0 = e->d_tile_e0;
  p.chan_tile_end = e->d_chan_tile_end;
  p.d = e->dev;
  return p;
}

template <typename R>
typename Prec<R>::State ens_state(adot_ensemble* e, int which) {
  using S = typename Prec<R>::S;
  return typename Prec<R>::State{(S*)e->buf[which][0], (S*)e->buf[which][1], (S*)e->buf[which][2]};
}

template <typename R>
cudaError_t ens_launch_t(adot_ensemble* e, int block, int grid, cudaStream_t s, int cur, int phase) {
  const EnsParams p = ens_params(e);
  const auto in = ens_state<R>(e, cur), out = ens_state<R>(e, 1 - cur);
  const int slot = phase % 3;
  if (e->warp) {
    if (block == 256 && e->cap == 64) k_ens_step_warp<R, 256, 64, kEnsSub><<<grid, 256, 0, s>>>(p, in, out, slot);
    else if (block == 256 && e->cap == 80) k_ens_step_warp<R, 256, 80, kEnsSub><<<grid, 256, 0, s>>>(p, in, out, slot);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
  }
  switch (block) {
    case 128: k_ens_step<R, 128><<<grid, 128, 0, s>>>(p, in, out, slot); break;
    case 256: k_ens_step<R, 256><<<grid, 256, 0, s>>>(p, in, out, slot); break;
    case 512: k_ens_step<R, 512><<<grid, 512, 0, s>>>(p, in, out, slot); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t ens_launch(adot_ensemble* e, cudaStream_t s, int cur, int phase) {
  if (e->prec == ADOT_FP32) return ens_launch_t<float>(e, e->block, e->grid, s, cur, phase);
  return ens_launch_t<double>(e, e->block, e->grid, s, cur, phase);
}

int resident_grid(adot_ensemble* e, int block) {
  int per_sm = 1, sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, e->device);
  cudaError_t err;
  if (e->warp) {
    const bool c80 = e->cap == 80;
    if (e->prec == ADOT_FP32)
      err = c80 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ens_step_warp<float, 256, 80, kEnsSub>, 256, 0)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ens_step_warp<float, 256, 64, kEnsSub>, 256, 0);
    else
      err = c80 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ens_step_warp<double, 256, 80, kEnsSub>, 256, 0)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ens_step_warp<double, 256, 64, kEnsSub>, 256, 0);
  } else if (e->prec == ADOT_FP32) {
    if (block == 128) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ens_step<float, 128>, 128, 0);
    else if (block == 256) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ens_step<float, 256>, 256, 0);
    else err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ens_step<float, 512>, 512, 0);
  } else {
    if (block == 128) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ens_step<double, 128>, 128, 0);
    else if (block == 256) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ens_step<double, 256>, 256, 0);
    else err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ens_step<double, 512>, 512, 0);
  }
  if (err != cudaSuccess || per_sm < 1) per_sm = 1;
  int64_t g = (int64_t)sms * per_sm;
  return (int)g;
}

// Launch of the persistent form with `block` threads per CTA on `grid` CTAs, or
// (grid = 0) the resident CTAs per SM of that shape into *per_sm.
template <typename R, int B, int CAP>
cudaError_t ens_run_launch_t(adot_ensemble* e, const EnsRun& r, int grid, int* per_sm) {
  if (grid == 0) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_ens_run<R, B, CAP>, B, 0);
  k_ens_run<R, B, CAP><<<grid, B, 0, e->stream>>>(ens_params(e), ens_state<R>(e, e->cur),
                                                  ens_state<R>(e, 1 - e->cur), r);
  return cudaGetLastError();
}

template <typename R>
cudaError_t ens_run_dispatch(adot_ensemble* e, const EnsRun& r, int block, int grid, int* per_sm) {
  if (block == 256) return ens_run_launch_t<R, 256, 80>(e, r, grid, per_sm);
  if (block == 384) return ens_run_launch_t<R, 384, 80>(e, r, grid, per_sm);
  if (block == 512) return ens_run_launch_t<R, 512, 64>(e, r, grid, per_sm);
  if (block == 768) return ens_run_launch_t<R, 768, 80>(e, r, grid, per_sm);
  return cudaErrorInvalidValue;
}

cudaError_t ens_run_call(adot_ensemble* e, const EnsRun& r, int block, int grid, int* per_sm = nullptr) {
  if (e->prec == ADOT_FP32) return ens_run_dispatch<float>(e, r, block, grid, per_sm);
  return ens_run_dispatch<double>(e, r, block, grid, per_sm);
}

// Launch of the cluster-team form (768 threads, 80 registers, CL CTAs per
// cluster) on `clusters` clusters, or (clusters = 0) the resident clusters into *n.
template <typename R, int CL>
cudaError_t ens_team_launch_t(adot_ensemble* e, const EnsTeamRun& r, int clusters, int* n) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(768, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = e->stream;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (clusters == 0) {
    cfg.gridDim = dim3((unsigned)((e->n_sms / CL) * CL), 1, 1);
    return cudaOccupancyMaxActiveClusters(n, (void*)k_ens_run_team<R, 768, 80, CL>, &cfg);
  }
  cfg.gridDim = dim3((unsigned)(clusters * CL), 1, 1);
  return cudaLaunchKernelEx(&cfg, k_ens_run_team<R, 768, 80, CL>, ens_params(e), ens_state<R>(e, e->cur),
                            ens_state<R>(e, 1 - e->cur), r);
}

cudaError_t ens_team_call(adot_ensemble* e, const EnsTeamRun& r, int cl, int clusters, int* n = nullptr) {
  if (e->prec == ADOT_FP32)
    return cl == 2 ? ens_team_launch_t<float, 2>(e, r, clusters, n) : ens_team_launch_t<float, 4>(e, r, clusters, n);
  return cl == 2 ? ens_team_launch_t<double, 2>(e, r, clusters, n) : ens_team_launch_t<double, 4>(e, r, clusters, n);
}

// Resident grid of a persistent shape (at most one CTA per channel).
int ens_run_grid(adot_ensemble* e, int block) {
  int per_sm = 0, sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, e->device);
  if (ens_run_call(e, EnsRun{}, block, 0, &per_sm) != cudaSuccess || per_sm < 1) per_sm = 1;
  return (int)std::min<int64_t>((int64_t)sms * per_sm, e->C);
}

// Tile list of a variant: channels longest first, tiles of block - 1 cells
// (block kernel) or 31 cells (warp tiles).
adot_status build_tiles(adot_ensemble* e, EnsVariant v) {
  std::vector<int> tc, te;
  std::vector<int> tend(e->C);
  const int64_t cells = v.warp ? 31 * kEnsSub : v.block - 1;
  for (int c : e->order) {
    const int64_t nt = (e->n_cells[c] + cells - 1) / cells;
    for (int64_t j = 0; j < nt; ++j) {
      tc.push_back(c);
      te.push_back((int)(j * cells));
    }
    tend[c] = (int)tc.size();
  }
  if (tc.size() > 0x7fffffff) return ADOT_E_INVALID_ARG;
  if (e->d_tile_chan) cudaFree(e->d_tile_chan);
  if (e->d_tile_e0) cudaFree(e->d_tile_e0);
  e->d_tile_chan = nullptr;
  e->d_tile_e0 = nullptr;
  e->n_tiles = (int64_t)tc.size();
  CKE(cudaMalloc((void**)&e->d_tile_chan, sizeof(int) * tc.size()));
  CKE(cudaMalloc((void**)&e->d_tile_e0, sizeof(int) * te.size()));
  CKE(cudaMemcpy(e->d_tile_chan, tc.data(), sizeof(int) * tc.size(), cudaMemcpyHostToDevice));
  CKE(cudaMemcpy(e->d_tile_e0, te.data(), sizeof(int) * te.size(), cudaMemcpyHostToDevice));
  CKE(cudaMemcpy(e->d_chan_tile_end, tend.data(), sizeof(int) * e->C, cudaMemcpyHostToDevice));
  e->block = v.block;
  e->cap = v.cap;
  e->warp = v.warp;
  int g = resident_grid(e, v.block);
  const int64_t need = v.warp ? (e->n_tiles * 32 + v.block - 1) / v.block : e->n_tiles;  // one warp per tile
  e->grid = (int)std::min<int64_t>(g, std::max<int64_t>(1, need));
  return ADOT_OK;
}

adot_status ens_build_graph(adot_ensemble* e) {
  if (e->graph_ready) {
    cudaGraphExecDestroy(e->graph);
    e->graph_ready = false;
  }
  cudaGraph_t g = nullptr;
  CKE(cudaStreamBeginCapture(e->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t err = cudaSuccess;
  for (int k = 0; k < e->steps_per_graph && err == cudaSuccess; ++k)
    err = ens_launch(e, e->cap_stream, k & 1, k % 6);
  cudaError_t e2 = cudaStreamEndCapture(e->cap_stream, &g);
  if (err != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return ADOT_E_CUDA;
  }
  err = cudaGraphInstantiate(&e->graph, g, 0);
  cudaGraphDestroy(g);
  if (err != cudaSuccess) return ADOT_E_CUDA;
  e->graph_ready = true;
  return ADOT_OK;
}

adot_status ens_enqueue(adot_ensemble* e, int64_t n) {
  while (n > 0) {
    if (e->phase == 0 && n >= e->steps_per_graph) {
      CKE(cudaGraphLaunch(e->graph, e->stream));
      n -= e->steps_per_graph;
    } else {
      CKE(ens_launch(e, e->stream, e->cur, e->phase));
      e->cur ^= 1;
      e->phase = (e->phase + 1) % 6;
      --n;
    }
  }
  return ADOT_OK;
}

adot_status ens_read(adot_ensemble* e, HostCtl* h) {
  CKE(cudaMemcpyAsync(h->gstep, e->dev.gstep, sizeof(h->gstep), cudaMemcpyDeviceToHost, e->stream));
  CKE(cudaMemcpyAsync(h->active, e->dev.active, sizeof(h->active), cudaMemcpyDeviceToHost, e->stream));
  CKE(cudaMemcpyAsync(&h->status, e->dev.status, sizeof(unsigned), cudaMemcpyDeviceToHost, e->stream));
  CKE(cudaStreamSynchronize(e->stream));
  return ADOT_OK;
}

adot_status ens_set_t_end(adot_ensemble* e, double t_end) {
  if (e->t_end_dev == t_end) return ADOT_OK;
  CKE(cudaStreamSynchronize(e->stream));
  CKE(cudaMemcpy(e->dev.t_end, &t_end, sizeof(double), cudaMemcpyHostToDevice));
  e->t_end_dev = t_end;
  return ADOT_OK;
}

// Resets every control array: all channels at t0 = 0, nothing finished, the
// whole tile list active, the previous-step slot at -inf.
adot_status ens_reset_ctl(adot_ensemble* e) {
  const int C = e->C;
  CKE(cudaMemsetAsync(e->d_ctl_mem, 0, e->ctl_bytes, e->stream));
  std::vector<long long> fin(C, 0x7fffffffffffffffLL);
  CKE(cudaMemcpyAsync(e->dev.fin, fin.data(), sizeof(long long) * C, cudaMemcpyHostToDevice, e->stream));
  int act[3] = {(int)e->n_tiles, 0, 0};
  CKE(cudaMemcpyAsync(e->dev.active, act, sizeof(act), cudaMemcpyHostToDevice, e->stream));
  double inf = INFINITY;
  CKE(cudaMemcpyAsync(e->dev.t_end, &inf, sizeof(double), cudaMemcpyHostToDevice, e->stream));
  CKE(cudaStreamSynchronize(e->stream));
  e->t_end_dev = INFINITY;
  e->cur = 0;
  e->phase = 0;
  return ADOT_OK;
}

// Variants allowed by the configuration (block_threads, step_kernel).
bool ens_candidate(const adot_ensemble* e, EnsVariant v) {
  if (e->step_kernel_cfg == 1 && v.warp) return false;
  if (e->step_kernel_cfg == 2 && !v.warp) return false;
  if (e->block_cfg && v.block != e->block_cfg) return false;
  return true;
}

// Trial steps of each variant on the current state (no state advance:
// with t_end = inf no channel finishes; the written slot and the tile bound
// are reset afterwards).
adot_status ens_tune(adot_ensemble* e, int trial) {
  cudaEvent_t a, b;
  CKE(cudaEventCreate(&a));
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return ADOT_E_CUDA;
  }
  float best = 0.0f;
  EnsVariant best_v{e->block, e->cap, e->warp};
  bool have = false;
  cudaError_t err = cudaSuccess;
  for (int i = 0; i < kNumEnsVariants && err == cudaSuccess; ++i) {
    const EnsVariant v = kEnsVariants[i];
    if (!ens_candidate(e, v)) continue;
    if (build_tiles(e, v) != ADOT_OK) {
      err = cudaErrorUnknown;
      break;
    }
    int act[3] = {(int)e->n_tiles, 0, 0};
    err = cudaMemcpy(e->dev.active, act, sizeof(act), cudaMemcpyHostToDevice);
    for (int k = 0; k < 1 + trial && err == cudaSuccess; ++k) {
      if (k == 1) err = cudaEventRecord(a, e->stream);
      if (err == cudaSuccess) err = ens_launch(e, e->stream, e->cur, e->phase);
    }
    if (err == cudaSuccess) err = cudaEventRecord(b, e->stream);
    if (err == cudaSuccess) err = cudaEventSynchronize(b);
    float ms = 0.0f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, a, b);
    if (err == cudaSuccess && (!have || ms < best)) {
      best = ms;
      best_v = v;
      have = true;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (err != cudaSuccess) return ADOT_E_CUDA;
  adot_status st = build_tiles(e, best_v);
  if (st) return st;
  // undo what the trials wrote: slot 1 (CFL maxima, times) and the tile bounds
  const int C = e->C;
  CKE(cudaMemsetAsync(e->dev.rho + C, 0, sizeof(unsigned long long) * C, e->stream));
  int act[3] = {(int)e->n_tiles, 0, 0};
  CKE(cudaMemcpyAsync(e->dev.active, act, sizeof(act), cudaMemcpyHostToDevice, e->stream));
  long long g0[3] = {0, 0, 0};
  CKE(cudaMemcpyAsync(e->dev.gstep, g0, sizeof(g0), cudaMemcpyHostToDevice, e->stream));
  CKE(cudaMemsetAsync(e->dev.t_cur, 0, sizeof(double) * C, e->stream));
  CKE(cudaMemsetAsync(e->dev.dt_cur, 0, sizeof(double) * C, e->stream));
  CKE(cudaMemsetAsync(e->dev.steps_cur, 0, sizeof(long long) * C, e->stream));
  CKE(cudaStreamSynchronize(e->stream));
  e->tuned = true;
  return ens_build_graph(e);
}

// Longest-processing-time list scheduling of the work items w (sorted in
// decreasing order) onto g equal workers: makespan / (sum w / g).
double lpt_imbalance(const std::vector<double>& w_sorted, int g) {
  if (g < 1 || w_sorted.empty()) return 1.0;
  std::vector<double> load((size_t)g, 0.0);  // min-heap of worker loads
  auto cmp = [](double a, double b) { return a > b; };
  double total = 0.0;
  for (double x : w_sorted) {
    std::pop_heap(load.begin(), load.end(), cmp);
    load.back() += x;
    std::push_heap(load.begin(), load.end(), cmp);
    total += x;
  }
  const double mk = *std::max_element(load.begin(), load.end());
  return total > 0.0 ? mk / (total / g) : 1.0;
}

// A team plan: channels with work >= thr (the long ones, in decreasing order)
// go to the cluster with the least team work, counted as work / (CL x
// kTeamEff); the others to the CTA with the least load, every CTA starting at
// its cluster's team work. Returns the makespan / (total work / CTAs); fills
// the per-cluster lists and the short-channel order when asked.
constexpr double kTeamEff = 0.95;  // a team of CL CTAs steps a channel ~CL x this faster than one CTA

double team_plan(const std::vector<double>& ws, const std::vector<int>& ord, int n_cl, int cl, double thr,
                 std::vector<int>* ptr, std::vector<int>* list, std::vector<int>* small, int* n_big) {
  const int C = (int)ws.size();
  if (n_cl < 1) return INFINITY;
  std::vector<double> cload((size_t)n_cl, 0.0);
  std::vector<std::vector<int>> lists((size_t)n_cl);
  double total = 0.0;
  int nb = 0;
  for (int i = 0; i < C; ++i) total += ws[i];
  for (; nb < C && ws[nb] >= thr; ++nb) {
    int best = 0;
    for (int k = 1; k < n_cl; ++k)
      if (cload[k] < cload[best]) best = k;
    cload[best] += ws[nb] / (cl * kTeamEff);
    lists[best].push_back(ord[nb]);
  }
  if (nb == 0) return INFINITY;
  const int n_cta = n_cl * cl;
  std::vector<double> load((size_t)n_cta);
  for (int k = 0; k < n_cta; ++k) load[k] = cload[k / cl];
  auto cmp = [](double a, double b) { return a > b; };
  std::make_heap(load.begin(), load.end(), cmp);
  for (int i = nb; i < C; ++i) {
    std::pop_heap(load.begin(), load.end(), cmp);
    load.back() += ws[i];
    std::push_heap(load.begin(), load.end(), cmp);
  }
  const double mk = *std::max_element(load.begin(), load.end());
  if (ptr) {
    ptr->assign(1, 0);
    list->clear();
    for (int k = 0; k < n_cl; ++k) {
      list->insert(list->end(), lists[k].begin(), lists[k].end());
      ptr->push_back((int)list->size());
    }
    small->assign(ord.begin() + nb, ord.end());
    *n_big = nb;
  }
  return total > 0.0 ? mk / (total / n_cta) : 1.0;
}

// Plans of run_to (k = 0) and step (k = 1). A channel's work is N_c times its
// steps: for run_to N_c rho_c / dx_c (steps per unit time, from the first CFL
// maxima in slot 0), for step N_c. Each CTA of the persistent form steps one
// channel at a time, so its time is that of the list schedule of the channels,
// largest first, onto the resident CTAs; the shape with the smaller estimated
// imbalance is taken (or the configured one). Team plans put the channels
// above a work threshold (1/2, 1 or 2 mean CTA loads) on clusters of 2 or 4
// CTAs and are taken when they beat the one-CTA shapes by 3 %. With
// step_kernel = 0 the per-step form runs instead when the best imbalance
// exceeds 1 / kPerStepRel; step_kernel 3 takes the best persistent plan, 5 the
// best team plan.
adot_status ens_plan(adot_ensemble* e) {
  const int C = e->C;
  std::vector<unsigned long long> bits(C);
  CKE(cudaMemcpyAsync(bits.data(), e->dev.rho, sizeof(unsigned long long) * C, cudaMemcpyDeviceToHost,
                      e->stream));
  CKE(cudaStreamSynchronize(e->stream));
  for (int k = 0; k < 2; ++k) {
    std::vector<double> w(C);
    for (int c = 0; c < C; ++c) {
      const double n = (double)e->n_cells[c];
      if (k == 1) {
        w[c] = n;
        continue;
      }
      double rho;
      if (e->prec == ADOT_FP32) {
        const unsigned u = (unsigned)bits[c];
        float f;
        memcpy(&f, &u, sizeof(f));
        rho = f;
      } else {
        memcpy(&rho, &bits[c], sizeof(rho));
      }
      w[c] = n * n * rho / e->length[c];
    }
    std::vector<int> ord(C);
    for (int c = 0; c < C; ++c) ord[c] = c;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return w[a] > w[b]; });
    std::vector<double> ws(C);
    double total = 0.0;
    for (int i = 0; i < C; ++i) {
      ws[i] = w[ord[i]];
      total += ws[i];
    }
    adot_ensemble::Plan& pl = e->plan[k];
    pl.imbalance = INFINITY;
    pl.cluster = 1;
    for (int i = 0; i < kNumRunBlocks; ++i) {
      const int blk = kRunBlocks[i];
      if (e->run_block_cfg && blk != e->run_block_cfg) continue;
      const int g = (int)std::min<int64_t>((int64_t)e->n_sms * e->run_occ[i], C);
      const double imb = lpt_imbalance(ws, g);
      if (imb < pl.imbalance) {
        pl.imbalance = imb;
        pl.block = blk;
        pl.grid = g;
      }
    }
    if (e->run_block_cfg && !(pl.imbalance < INFINITY)) {  // a configured shape outside kRunBlocks
      pl.block = e->run_block_cfg;
      pl.grid = ens_run_grid(e, pl.block);
      pl.imbalance = lpt_imbalance(ws, pl.grid);
    }
    // team plans (768-thread CTAs)
    double best_team = INFINITY;
    int team_cl = 0;
    double team_thr = 0.0;
    if (e->run_block_cfg == 0 || e->run_block_cfg == 768) {
      for (int ci = 0; ci < 2; ++ci) {
        const int cl = ci == 0 ? 2 : 4;
        const int n_cl = e->team_clusters[ci];
        if (n_cl < 1) continue;
        for (double f : {0.5, 1.0, 2.0}) {
          const double thr = f * total / (n_cl * cl);
          const double imb = team_plan(ws, ord, n_cl, cl, thr, nullptr, nullptr, nullptr, nullptr);
          if (imb < best_team) {
            best_team = imb;
            team_cl = cl;
            team_thr = thr;
          }
        }
      }
    }
    const bool want_team = team_cl > 0 && (e->step_kernel_cfg == 5 || best_team < 0.97 * pl.imbalance);
    std::vector<int> small = ord;
    pl.n_big = 0;
    if (want_team) {
      std::vector<int> ptr, list;
      const int n_cl = e->team_clusters[team_cl == 2 ? 0 : 1];
      team_plan(ws, ord, n_cl, team_cl, team_thr, &ptr, &list, &small, &pl.n_big);
      pl.cluster = team_cl;
      pl.block = 768;
      pl.grid = n_cl * team_cl;
      pl.imbalance = best_team;
      std::vector<int> tbuf(ptr);
      tbuf.insert(tbuf.end(), list.begin(), list.end());
      CKE(cudaMemcpyAsync(pl.d_team, tbuf.data(), sizeof(int) * tbuf.size(), cudaMemcpyHostToDevice,
                          e->stream));
      CKE(cudaStreamSynchronize(e->stream));
    }
    pl.n_small = (int)small.size();
    pl.persistent = e->step_kernel_cfg == 3 || e->step_kernel_cfg == 5 || pl.imbalance * kPerStepRel <= 1.0;
    if (!small.empty())
      CKE(cudaMemcpyAsync(pl.d_order, small.data(), sizeof(int) * small.size(), cudaMemcpyHostToDevice,
                          e->stream));
  }
  CKE(cudaStreamSynchronize(e->stream));
  return ADOT_OK;
}

// Persistent form: launches of at most kRunChunk steps per channel (the host
// reads the status word between launches) until every channel has reached
// t_end, or every channel has taken n_steps steps (n_steps >= 0, t_end = inf).
constexpr long long kRunChunk = 1 << 14;

adot_status ens_run(adot_ensemble* e, const adot_ensemble::Plan& pl, double t_end, long long n_steps,
                    int64_t* launches_out) {
  int64_t launches = 0;
  long long left = n_steps;
  for (;;) {
    if (n_steps >= 0 && left <= 0) break;
    const long long m = (n_steps >= 0) ? std::min(left, kRunChunk) : kRunChunk;
    CKE(cudaMemsetAsync(e->dev.next, 0, sizeof(int), e->stream));
    CKE(cudaMemsetAsync(e->dev.active, 0, sizeof(int) * 3, e->stream));
    const int slot = e->phase % 3;
    if (pl.cluster > 1) {
      EnsTeamRun r;
      r.big_ptr = pl.d_team;
      r.big_list = pl.d_team + pl.grid / pl.cluster + 1;
      r.order = pl.d_order;
      r.n_small = pl.n_small;
      r.next = e->dev.next;
      r.t_end = t_end;
      r.max_steps = m;
      r.slot = slot;
      r.fault = e->fault;
      e->fault = 0;
      CKE(ens_team_call(e, r, pl.cluster, pl.grid / pl.cluster));
    } else {
      EnsRun r;
      r.order = pl.d_order;
      r.next = e->dev.next;
      r.t_end = t_end;
      r.max_steps = m;
      r.slot = slot;
      CKE(ens_run_call(e, r, pl.block, pl.grid));
    }
    ++launches;
    left -= m;
    HostCtl hc;
    adot_status st = ens_read(e, &hc);
    if (st) return st;
    st = ens_status(hc.status);
    if (st) return st;
    if (hc.active[slot] == 0) break;  // every channel at t_end
  }
  if (launches_out) *launches_out = launches;
  return ADOT_OK;
}

void ens_free(adot_ensemble* e) {
  if (!e) return;
  if (e->graph_ready) cudaGraphExecDestroy(e->graph);
  for (int b = 0; b < 2; ++b)
    for (int k = 0; k < 3; ++k)
      if (e->buf[b][k]) cudaFree(e->buf[b][k]);
  if (e->d_off) cudaFree(e->d_off);
  if (e->d_dx) cudaFree(e->d_dx);
  if (e->d_K3f) cudaFree(e->d_K3f);
  if (e->d_K3d) cudaFree(e->d_K3d);
  if (e->d_tile_chan) cudaFree(e->d_tile_chan);
  if (e->d_tile_e0) cudaFree(e->d_tile_e0);
  if (e->d_chan_tile_end) cudaFree(e->d_chan_tile_end);
  for (int k = 0; k < 2; ++k) {
    if (e->plan[k].d_order) cudaFree(e->plan[k].d_order);
    if (e->plan[k].d_team) cudaFree(e->plan[k].d_team);
  }
  if (e->d_ctl_mem) cudaFree(e->d_ctl_mem);
  if (e->d_io) cudaFree(e->d_io);
  if (e->cap_stream) cudaStreamDestroy(e->cap_stream);
  if (e->own_stream && e->stream) cudaStreamDestroy(e->stream);
  delete e;
}

}  // namespace

extern "C" {

adot_status adot_ensemble_create(const adot_ensemble_config* cfg, void* cuda_stream,
                                 adot_ensemble** out) {
  if (!out) return ADOT_E_INVALID_ARG;
  *out = nullptr;
  if (!cfg || cfg->n_channels < 1 || !cfg->n_cells || !cfg->length || !cfg->Ag) return ADOT_E_INVALID_ARG;
  if (!(cfg->g > 0.0) || !(cfg->xi > 0.0) || !(cfg->cfl > 0.0 && cfg->cfl <= 1.0)) return ADOT_E_INVALID_ARG;
  if (cfg->precision != ADOT_FP64 && cfg->precision != ADOT_FP32) return ADOT_E_INVALID_ARG;
  if (cfg->step_kernel < 0 || cfg->step_kernel > 5) return ADOT_E_INVALID_ARG;
  if (cfg->step_kernel == 5 && cfg->block_threads != 0 && cfg->block_threads != 768) return ADOT_E_INVALID_ARG;
  if (cfg->step_kernel == 0 || cfg->step_kernel == 3 || cfg->step_kernel == 5) {
    if (cfg->block_threads != 0 && cfg->block_threads != 256 && cfg->block_threads != 384 &&
        cfg->block_threads != 512 && cfg->block_threads != 768)
      return ADOT_E_INVALID_ARG;
  } else if (cfg->block_threads != 0 && cfg->block_threads != 128 && cfg->block_threads != 256 &&
             cfg->block_threads != 512) {
    return ADOT_E_INVALID_ARG;
  }
  if (cfg->step_kernel == 2 && cfg->block_threads != 0 && cfg->block_threads != 256) return ADOT_E_INVALID_ARG;
  if (cfg->steps_per_graph < 0 || cfg->device < -1) return ADOT_E_INVALID_ARG;
  const int C = cfg->n_channels;
  int64_t total = 0;
  for (int c = 0; c < C; ++c) {
    if (cfg->n_cells[c] < 1 || cfg->n_cells[c] > 0x7fff0000LL) return ADOT_E_INVALID_ARG;
    if (!(cfg->length[c] > 0.0) || !isfinite(cfg->Ag[c])) return ADOT_E_INVALID_ARG;
    total += cfg->n_cells[c];
  }
  if (cfg->device >= 0 && cudaSetDevice(cfg->device) != cudaSuccess) return ADOT_E_CUDA;
  adot_ensemble* e = new adot_ensemble();
  memset(e->buf, 0, sizeof(e->buf));
  e->C = C;
  e->prec = cfg->precision;
  cudaGetDevice(&e->device);
  e->cfl = cfg->cfl;
  e->g = cfg->g;
  e->xi = cfg->xi;
  e->n_total = total;
  e->n_cells.assign(cfg->n_cells, cfg->n_cells + C);
  e->length.assign(cfg->length, cfg->length + C);
  e->off.resize(C + 1);
  e->off[0] = 0;
  for (int c = 0; c < C; ++c) e->off[c + 1] = e->off[c] + e->n_cells[c];
  e->order.resize(C);
  for (int c = 0; c < C; ++c) e->order[c] = c;
  std::stable_sort(e->order.begin(), e->order.end(),
                   [&](int a, int b) { return e->n_cells[a] > e->n_cells[b]; });
  int spg = cfg->steps_per_graph ? cfg->steps_per_graph : 48;
  e->steps_per_graph = ((spg + 5) / 6) * 6;
  e->step_kernel_cfg = cfg->step_kernel;
  const bool may_persist = cfg->step_kernel == 0 || cfg->step_kernel == 3 || cfg->step_kernel == 5;
  e->block_cfg = may_persist ? 0 : cfg->block_threads;
  e->run_block_cfg = may_persist ? cfg->block_threads : 0;
  e->t_end_dev = INFINITY;

  std::vector<double> dx(C), K3d(C);
  std::vector<float> K3f(C);
  for (int c = 0; c < C; ++c) {
    dx[c] = cfg->length[c] / (double)e->n_cells[c];
    K3d[c] = 3.0 * cfg->xi * cfg->Ag[c];
    K3f[c] = (float)K3d[c];
  }
  cudaError_t err = cudaSuccess;
  if (cuda_stream) {
    e->stream = (cudaStream_t)cuda_stream;
  } else {
    err = cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking);
    e->own_stream = true;
  }
  if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&e->cap_stream, cudaStreamNonBlocking);
  const size_t elem = (e->prec == ADOT_FP32) ? sizeof(float2) : sizeof(double);
  for (int b = 0; b < 2 && err == cudaSuccess; ++b)
    for (int k = 0; k < 3 && err == cudaSuccess; ++k) err = cudaMalloc(&e->buf[b][k], elem * (size_t)total);
  if (err == cudaSuccess) err = cudaMalloc((void**)&e->d_off, sizeof(int64_t) * (C + 1));
  if (err == cudaSuccess) err = cudaMalloc((void**)&e->d_dx, sizeof(double) * C);
  if (err == cudaSuccess) err = cudaMalloc((void**)&e->d_K3f, sizeof(float) * C);
  if (err == cudaSuccess) err = cudaMalloc((void**)&e->d_K3d, sizeof(double) * C);
  if (err == cudaSuccess) err = cudaMalloc((void**)&e->d_chan_tile_end, sizeof(int) * C);
  if (err == cudaSuccess && e->prec == ADOT_FP32) err = cudaMalloc((void**)&e->d_io, sizeof(double) * (size_t)total);
  // control arrays in one allocation
  const size_t slots = 3 * (size_t)C;
  e->ctl_bytes = slots * (sizeof(double) * 2 + sizeof(long long) + sizeof(unsigned long long)) +
                 (size_t)C * (sizeof(double) * 2 + sizeof(long long) * 2) + sizeof(long long) * 3 +
                 sizeof(int) * 4 + sizeof(double) + sizeof(unsigned) + sizeof(int) + 64;
  if (err == cudaSuccess) err = cudaMalloc(&e->d_ctl_mem, e->ctl_bytes);
  if (err == cudaSuccess) {
    char* m = (char*)e->d_ctl_mem;
    auto take = [&](size_t bytes) {
      char* r = m;
      m += (bytes + 7) & ~(size_t)7;
      return r;
    };
    e->dev.t = (double*)take(sizeof(double) * slots);
    e->dev.dt = (double*)take(sizeof(double) * slots);
    e->dev.steps = (long long*)take(sizeof(long long) * slots);
    e->dev.rho = (unsigned long long*)take(sizeof(unsigned long long) * slots);
    e->dev.t_cur = (double*)take(sizeof(double) * C);
    e->dev.dt_cur = (double*)take(sizeof(double) * C);
    e->dev.steps_cur = (long long*)take(sizeof(long long) * C);
    e->dev.fin = (long long*)take(sizeof(long long) * C);
    e->dev.gstep = (long long*)take(sizeof(long long) * 3);
    e->dev.active = (int*)take(sizeof(int) * 4);
    e->dev.t_end = (double*)take(sizeof(double));
    e->dev.status = (unsigned*)take(sizeof(unsigned));
    e->dev.next = (int*)take(sizeof(int));
  }
  e->n_sms = 152;
  cudaDeviceGetAttribute(&e->n_sms, cudaDevAttrMultiProcessorCount, e->device);
  for (int k = 0; k < 2 && err == cudaSuccess; ++k) {
    err = cudaMalloc((void**)&e->plan[k].d_order, sizeof(int) * C);
    if (err == cudaSuccess)
      err = cudaMalloc((void**)&e->plan[k].d_team, sizeof(int) * ((size_t)e->n_sms + 1 + C));
    if (err == cudaSuccess)
      err = cudaMemcpy(e->plan[k].d_order, e->order.data(), sizeof(int) * C, cudaMemcpyHostToDevice);
    // until the first set_state: the configured form, persistent at the default shape
    e->plan[k].persistent = may_persist;
    e->plan[k].block = (e->run_block_cfg && e->run_block_cfg != 768) ? e->run_block_cfg : kRunBlockDefault;
    e->plan[k].grid = ens_run_grid(e, e->plan[k].block);
    e->plan[k].imbalance = 1.0;
    e->plan[k].cluster = 1;
    e->plan[k].n_big = 0;
    e->plan[k].n_small = C;
  }
  for (int ci = 0; ci < 2; ++ci) {
    int n = 0;
    if (ens_team_call(e, EnsTeamRun{}, ci == 0 ? 2 : 4, 0, &n) != cudaSuccess || n < 0) n = 0;
    e->team_clusters[ci] = std::min(n, e->n_sms / (ci == 0 ? 2 : 4));
  }
  cudaGetLastError();  // an unsupported cluster query leaves no error behind
  for (int i = 0; i < kNumRunBlocks; ++i) {
    int per_sm = 0;
    if (ens_run_call(e, EnsRun{}, kRunBlocks[i], 0, &per_sm) != cudaSuccess || per_sm < 1) per_sm = 1;
    e->run_occ[i] = per_sm;
  }
  if (err == cudaSuccess) err = cudaMemcpy(e->d_off, e->off.data(), sizeof(int64_t) * (C + 1), cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemcpy(e->d_dx, dx.data(), sizeof(double) * C, cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemcpy(e->d_K3f, K3f.data(), sizeof(float) * C, cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemcpy(e->d_K3d, K3d.data(), sizeof(double) * C, cudaMemcpyHostToDevice);
  // the first allowed variant; tuned at the first set_state unless it is the only one
  int n_cand = 0;
  EnsVariant v0{256, 64, false};
  for (int i = kNumEnsVariants - 1; i >= 0; --i)
    if (ens_candidate(e, kEnsVariants[i])) {
      v0 = kEnsVariants[i];
      ++n_cand;
    }
  e->tuned = n_cand == 1 || cfg->step_kernel == 3 || cfg->step_kernel == 5;
  if (err != cudaSuccess || build_tiles(e, v0) != ADOT_OK ||
      ens_reset_ctl(e) != ADOT_OK || ens_build_graph(e) != ADOT_OK) {
    ens_free(e);
    return ADOT_E_CUDA;
  }
  *out = e;
  return ADOT_OK;
}

void adot_ensemble_destroy(adot_ensemble* e) {
  if (!e) return;
  cudaStreamSynchronize(e->stream);
  ens_free(e);
}

adot_status adot_ensemble_set_state(adot_ensemble* e, const double* h, const double* q,
                                    const double* z, int on_device) {
  if (!e || !h || !q || !z) return ADOT_E_INVALID_ARG;
  const int64_t n = e->n_total;
  const size_t bytes = sizeof(double) * (size_t)n;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const double* src[3] = {h, q, z};
  CKE(cudaStreamSynchronize(e->stream));
  adot_status st = ens_reset_ctl(e);
  if (st) return st;
  for (int k = 0; k < 3; ++k) {
    if (e->prec == ADOT_FP32) {
      CKE(cudaMemcpyAsync(e->d_io, src[k], bytes, kind, e->stream));
      CKE(launch_to_ff(e->d_io, (float2*)e->buf[0][k], n, e->stream));
    } else {
      CKE(cudaMemcpyAsync(e->buf[0][k], src[k], bytes, kind, e->stream));
    }
  }
  // previous-step slot (2) at -inf so that no channel reads as already finished
  std::vector<double> neg(e->C, -INFINITY);
  CKE(cudaMemcpyAsync(e->dev.t + 2 * (size_t)e->C, neg.data(), sizeof(double) * e->C,
                      cudaMemcpyHostToDevice, e->stream));
  const EnsParams p = ens_params(e);
  int64_t g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  if (e->prec == ADOT_FP32)
    k_ens_rho<float><<<(unsigned)g, 256, 0, e->stream>>>(p, ens_state<float>(e, 0), n);
  else
    k_ens_rho<double><<<(unsigned)g, 256, 0, e->stream>>>(p, ens_state<double>(e, 0), n);
  CKE(cudaGetLastError());
  HostCtl hc;
  st = ens_read(e, &hc);
  if (st) return st;
  st = ens_status(hc.status);
  if (st) return st;
  e->state_set = true;
  if (e->step_kernel_cfg == 0 || e->step_kernel_cfg == 3 || e->step_kernel_cfg == 5) {
    st = ens_plan(e);
    if (st) return st;
  }
  if (!e->tuned && !(e->plan[0].persistent && e->plan[1].persistent)) return ens_tune(e, 2);
  return ADOT_OK;
}

adot_status adot_ensemble_get_state(adot_ensemble* e, double* h, double* q, double* z, int on_device) {
  if (!e || !h || !q || !z) return ADOT_E_INVALID_ARG;
  const int64_t n = e->n_total;
  const size_t bytes = sizeof(double) * (size_t)n;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  double* dst[3] = {h, q, z};
  for (int k = 0; k < 3; ++k) {
    if (e->prec == ADOT_FP32) {
      CKE(launch_from_ff((const float2*)e->buf[e->cur][k], e->d_io, n, e->stream));
      CKE(cudaMemcpyAsync(dst[k], e->d_io, bytes, kind, e->stream));
      CKE(cudaStreamSynchronize(e->stream));
    } else {
      CKE(cudaMemcpyAsync(dst[k], e->buf[e->cur][k], bytes, kind, e->stream));
    }
  }
  CKE(cudaStreamSynchronize(e->stream));
  return ADOT_OK;
}

adot_status adot_ensemble_run_to(adot_ensemble* e, double t_end, int64_t* launches_out) {
  if (!e || !e->state_set || !isfinite(t_end)) return ADOT_E_INVALID_ARG;
  adot_status st = ens_set_t_end(e, t_end);
  if (st) return st;
  if (e->plan[0].persistent) return ens_run(e, e->plan[0], t_end, -1, launches_out);
  int64_t launches = 0;
  for (;;) {
    const int64_t chunk = e->phase ? (6 - e->phase) : e->steps_per_graph;
    st = ens_enqueue(e, chunk);
    if (st) return st;
    launches += chunk;
    HostCtl hc;
    st = ens_read(e, &hc);
    if (st) return st;
    st = ens_status(hc.status);
    if (st) return st;
    if (hc.active[e->phase % 3] == 0) break;  // every channel finished and copied across
  }
  if (launches_out) *launches_out = launches;
  return ADOT_OK;
}

adot_status adot_ensemble_step(adot_ensemble* e, int64_t n_steps) {
  if (!e || !e->state_set || n_steps < 0) return ADOT_E_INVALID_ARG;
  adot_status st = ens_set_t_end(e, INFINITY);
  if (st) return st;
  if (e->plan[1].persistent) return ens_run(e, e->plan[1], INFINITY, n_steps, nullptr);
  st = ens_enqueue(e, n_steps);
  if (st) return st;
  HostCtl hc;
  st = ens_read(e, &hc);
  if (st) return st;
  return ens_status(hc.status);
}

adot_status adot_ensemble_query(adot_ensemble* e, double* t_out, int64_t* steps_out,
                                int64_t* cell_updates_out) {
  if (!e) return ADOT_E_INVALID_ARG;
  std::vector<long long> steps(e->C);
  CKE(cudaMemcpyAsync(steps.data(), e->dev.steps_cur, sizeof(long long) * e->C,
                      cudaMemcpyDeviceToHost, e->stream));
  if (t_out)
    CKE(cudaMemcpyAsync(t_out, e->dev.t_cur, sizeof(double) * e->C, cudaMemcpyDeviceToHost, e->stream));
  HostCtl hc;
  adot_status st = ens_read(e, &hc);
  if (st) return st;
  int64_t cu = 0;
  for (int c = 0; c < e->C; ++c) {
    if (steps_out) steps_out[c] = steps[c];
    cu += steps[c] * e->n_cells[c];
  }
  if (cell_updates_out) *cell_updates_out = cu;
  return ens_status(hc.status);
}

adot_status adot_ensemble_info(adot_ensemble* e, int32_t* block_out, int64_t* tiles_out,
                               int32_t* grid_out, int32_t* step_kernel_out) {
  if (!e) return ADOT_E_INVALID_ARG;
  if (e->plan[0].persistent) {
    if (step_kernel_out) *step_kernel_out = 3;
    if (block_out) *block_out = e->plan[0].block;
    if (tiles_out) *tiles_out = e->C;
    if (grid_out) *grid_out = e->plan[0].grid;
    return ADOT_OK;
  }
  if (step_kernel_out) *step_kernel_out = e->warp ? 2 : 1;
  if (block_out) *block_out = e->block;
  if (tiles_out) *tiles_out = e->n_tiles;
  if (grid_out) *grid_out = e->grid;
  return ADOT_OK;
}

adot_status adot_ensemble_inject_fault(adot_ensemble* e, int32_t kind) {
  if (!e || kind < 0 || kind > 1) return ADOT_E_INVALID_ARG;
  e->fault = kind;
  return ADOT_OK;
}

adot_status adot_ensemble_plan(adot_ensemble* e, int32_t which, int32_t* form_out, int32_t* block_out,
                               int32_t* cluster_out, int32_t* grid_out, int32_t* teamed_out,
                               double* imbalance_out) {
  if (!e || which < 0 || which > 1) return ADOT_E_INVALID_ARG;
  const adot_ensemble::Plan& pl = e->plan[which];
  if (form_out) *form_out = pl.persistent ? 3 : (e->warp ? 2 : 1);
  if (block_out) *block_out = pl.persistent ? pl.block : e->block;
  if (cluster_out) *cluster_out = pl.persistent ? pl.cluster : 1;
  if (grid_out) *grid_out = pl.persistent ? pl.grid : e->grid;
  if (teamed_out) *teamed_out = pl.persistent ? pl.n_big : 0;
  if (imbalance_out) *imbalance_out = pl.imbalance;
  return ADOT_OK;
}

}  // extern "C"
