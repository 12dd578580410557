// Second-order time step: MUSCL-Hancock in path-conservative form, on the
// same DOT edge (Eq. DOTjumpN) as the first-order kernels. The paper applies
// A-DOT to the first-order scheme and notes (Sec. 6) that nothing restricts the
// order; this is the reconstruction-of-states form of Castro, Gallardo & Pares
// (2006) with a Hancock half-step predictor. Per cell i:
//   1. minmod slopes of (eta = h + z, q, z) against both neighbours, turned
//      into slopes of (h, q, z) (the h slope is the eta slope minus the z
//      slope); boundary values W-+_i = W_i -+ slope/2;
//   2. predictor: both values move by -dt/(2 dx) A(W_i) (W+_i - W-_i);
//   3. a cell whose reconstructed or predicted depth is not positive keeps
//      zero slopes;
//   4. W_i <- W_i - dt/dx (D-(W+_i, W-_{i+1}) + D+(W+_{i-1}, W-_i) + I_i) with
//      I_i = sum_k w_k A(Psi_k) (W+_i - W-_i) on the segment inside the cell.
// Ghost cells are the first-order kernels' ghosts with zero slopes.
//
// Launch geometry: persistent warp tiles of 30 cells. Lane l of tile t holds
// cell c = 30 t - 1 + l (cells 30t-1 .. 30t+30), takes its neighbours' states by
// shuffle (lanes 0 and 31 load one more), evaluates the edge between its cell
// and the next lane's (lanes 0..30), and lanes 1..30 update cells 30t .. 30t+29
// with their own D- and the left lane's D+. One edge in 31 and two boundary
// values in 32 are evaluated twice.
#pragma once

#include "adot_step_impl.cuh"

namespace adot {

// One-lane shuffles of a state word (float-float pair or double).
__device__ __forceinline__ float2 shfl_up_s(float2 v) {
  return make_float2(__shfl_up_sync(0xffffffffu, v.x, 1), __shfl_up_sync(0xffffffffu, v.y, 1));
}
__device__ __forceinline__ double shfl_up_s(double v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ float2 shfl_down_s(float2 v) {
  return make_float2(__shfl_down_sync(0xffffffffu, v.x, 1), __shfl_down_sync(0xffffffffu, v.y, 1));
}
__device__ __forceinline__ double shfl_down_s(double v) {
  return __shfl_down_sync(0xffffffffu, v, 1);
}

__device__ __forceinline__ float minmod(float a, float b) {
  return (a > 0.0f && b > 0.0f) ? fminf(a, b) : ((a < 0.0f && b < 0.0f) ? fmaxf(a, b) : 0.0f);
}
__device__ __forceinline__ double minmod(double a, double b) {
  return (a > 0.0 && b > 0.0) ? fmin(a, b) : ((a < 0.0 && b < 0.0) ? fmax(a, b) : 0.0);
}

// State of cell c with the periodic wrap, or the ghost beyond an end (c < 0:
// left, c >= n: right). Reads only cells 0 .. n-1.
template <typename R>
__device__ __forceinline__ void load_cell2(const StepParams& p, const typename Prec<R>::State& st,
                                           int64_t c, int slot, typename Prec<R>::S w[3]) {
  const int64_t n = p.n;
  if (c >= 0 && c < n) {
    w[0] = st.h[c];
    w[1] = st.q[c];
    w[2] = st.z[c];
  } else if (p.periodic) {
    const int64_t k = ((c % n) + n) % n;
    w[0] = st.h[k];
    w[1] = st.q[k];
    w[2] = st.z[k];
  } else {
    const bool left = c < 0;
    const int64_t a = left ? 0 : n - 1;
    const int64_t b = (n > 1) ? (left ? 1 : n - 2) : a;
    typename Prec<R>::S adj[3] = {st.h[a], st.q[a], st.z[a]};
    ghost_state<R>(left ? p.bc_left : p.bc_right, left ? p.bcl : p.bcr, p.ctl->s[slot].t, adj,
                   st.z[b], w);
  }
}

// A dW at a state (h, q) with 1/h, u, c^2: (dq, (c^2 - u^2) dh + 2u dq + c^2 dz, a dh + b dq).
template <typename R, int LAW>
__device__ __forceinline__ void A_times(const LawT<R>& L, R h, R q, const R d[3], R out[3]) {
  const R inv_h = R(1) / h;
  const R u = q * inv_h, c2 = L.g * h;
  R a, b;
  sediment_derivs<R, LAW>(L, h, q, inv_h, u, a, b);
  out[0] = d[1];
  out[1] = (c2 - u * u) * d[0] + R(2) * u * d[1] + c2 * d[2];
  out[2] = a * d[0] + b * d[1];
}

template <typename R, int LAW, int B, int CAP>
__global__ void __launch_bounds__(B, MinBlocks<B, CAP>::value)
    k_step2_warp(const StepParams p, const typename Prec<R>::State in,
                 const typename Prec<R>::State out, const int slot) {
  using S = typename Prec<R>::S;
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * B + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * B) >> 5;
  const int64_t n = p.n;
  const int64_t n_tiles = (n + 29) / 30;
  const LawT<R>& L = Prec<R>::law(p);

  R nu;
  bool done;
  warp_step_size<R>(p, slot, lane, gw == 0, nu, done);
  const R half = R(0.5) * nu;

  unsigned flags = 0;
  R rho_run = R(0);
  for (int64_t t = gw; t < n_tiles; t += nwarps) {
    const int64_t c = 30 * t - 1 + lane;
    // a lane beyond the ghost on the right (last tile) repeats the ghost
    const int64_t cl = (!p.periodic && c > n) ? n : c;
    const bool ghost = !p.periodic && (cl < 0 || cl >= n);
    S w[3], wm[3], wp[3];
    load_cell2<R>(p, in, cl, slot, w);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      wm[r] = shfl_up_s(w[r]);
      wp[r] = shfl_down_s(w[r]);
    }
    if (lane == 0) load_cell2<R>(p, in, cl - 1, slot, wm);
    if (lane == 31) load_cell2<R>(p, in, (!p.periodic && cl + 1 > n) ? n : cl + 1, slot, wp);

    // 1. slopes in (h, q, z) from minmod slopes of (eta, q, z)
    R sw[3] = {R(0), R(0), R(0)};
    if (!ghost) {
      const R mh = Prec<R>::diff(w[0], wm[0]), mq = Prec<R>::diff(w[1], wm[1]);
      const R mz = Prec<R>::diff(w[2], wm[2]);
      const R ph = Prec<R>::diff(wp[0], w[0]), pq = Prec<R>::diff(wp[1], w[1]);
      const R pz = Prec<R>::diff(wp[2], w[2]);
      const R se = minmod(mh + mz, ph + pz);
      sw[2] = minmod(mz, pz);
      sw[1] = minmod(mq, pq);
      sw[0] = se - sw[2];
    }
    // 2.-3. boundary values (offsets from W_i) after the half-step predictor
    const R h0 = Prec<R>::hi(w[0]), q0 = Prec<R>::hi(w[1]);
    R dL[3], dR[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      dL[r] = -R(0.5) * sw[r];
      dR[r] = R(0.5) * sw[r];
    }
    const bool sloped = sw[0] != R(0) || sw[1] != R(0) || sw[2] != R(0);
    bool flat = !(h0 + dL[0] > R(0)) || !(h0 + dR[0] > R(0));
    if (sloped && !flat) {
      R Ad[3];
      A_times<R, LAW>(L, h0, q0, sw, Ad);
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        dL[r] -= half * Ad[r];
        dR[r] -= half * Ad[r];
      }
      flat = !(h0 + dL[0] > R(0)) || !(h0 + dR[0] > R(0));
    }
    if (flat || !sloped) {
#pragma unroll
      for (int r = 0; r < 3; ++r) sw[r] = dL[r] = dR[r] = R(0);
    }
    // 4a. path integral of A inside the cell: W+ - W- = slope
    R I[3] = {R(0), R(0), R(0)};
    if (sloped && !flat) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const R sk = (k == 0) ? R(GL3_S0) : ((k == 1) ? R(0.5) : R(GL3_S2));
        const R wk = (k == 1) ? R(GL3_W1) : R(GL3_W0);
        R Ak[3];
        A_times<R, LAW>(L, h0 + dL[0] + sk * sw[0], q0 + dL[1] + sk * sw[1], sw, Ak);
#pragma unroll
        for (int r = 0; r < 3; ++r) I[r] += wk * Ak[r];
      }
    }
    // 4b. the edge to the next lane's cell: W+ here, W- there
    S wlb[3], wrb[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      wlb[r] = Prec<R>::add(w[r], dR[r]);
      wrb[r] = shfl_down_s(Prec<R>::add(w[r], dL[r]));
    }
    R dm[3] = {R(0), R(0), R(0)}, dp[3] = {R(0), R(0), R(0)};
    const bool has_edge = lane < 31 && (p.periodic || (c >= -1 && c + 1 <= n));
    if (has_edge) edge_fluct<R, LAW>(p, wlb, wrb, dm, dp, flags);
    R dl[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) dl[r] = __shfl_up_sync(0xffffffffu, dp[r], 1);
    // 4c. update of cells 30t .. 30t+29
    if (lane >= 1 && lane <= 30 && c >= 0 && c < n) {
      S nh = w[0], nq = w[1], nz = w[2];
      if (!done) {
        nh = Prec<R>::add(w[0], -nu * (dm[0] + dl[0] + I[0]));
        nq = Prec<R>::add(w[1], -nu * (dm[1] + dl[1] + I[1]));
        nz = Prec<R>::add(w[2], -nu * (dm[2] + dl[2] + I[2]));
      }
      out.h[c] = nh;
      out.q[c] = nq;
      out.z[c] = nz;
      if (!done) {
        const R hh = Prec<R>::hi(nh);
        if (!(hh > R(0))) flags |= ST_DEPTH;
        if (!(Prec<R>::finite(nh) && Prec<R>::finite(nq) && Prec<R>::finite(nz))) {
          flags |= ST_NONFINITE;
        } else if (hh > R(0)) {
          R r;
          if constexpr (std::is_same<R, float>::value)
            r = spectral_radius_f32<LAW, true>(p.lf, hh, Prec<R>::hi(nq), rho_run);  // 0: below rho_run
          else
            r = Prec<R>::template rho<LAW>(p, hh, Prec<R>::hi(nq));
          if (!(r <= R(3.0e38))) {
            flags |= ST_NONFINITE;
            r = R(0);
          }
          rho_run = d_max(rho_run, r);
        }
      }
    }
  }
  rho_run = warp_max(rho_run);
  if (lane == 0 && !done && rho_run > R(0))
    atomicMax(&p.ctl->s[(slot + 1) % 3].rho_bits, Prec<R>::bits(rho_run));
  if (flags) atomicOr(&p.ctl->status, flags);
}

template <typename R, int LAW>
cudaError_t launch_step2_law(const StepParams& p, StepVariant v, typename Prec<R>::State in,
                             typename Prec<R>::State out, int slot, cudaStream_t s) {
  if (p.ctl == nullptr || p.n < 1 || !v.warp_tiles) return cudaErrorInvalidValue;
  int sms = 152, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t per_sm = v.reg_cap ? 65536 / (v.block * v.reg_cap) : 1;
  const int64_t tiles = (p.n + 29) / 30;
  const int64_t wpb = v.block / 32;
  int64_t gg = (tiles + wpb - 1) / wpb;
  if (gg > sms * per_sm) gg = sms * per_sm;
#define ADOT_STEP2_CASE(BB, CC)                                                   \
  if (v.block == BB && v.reg_cap == CC) {                                         \
    k_step2_warp<R, LAW, BB, CC><<<(unsigned)gg, BB, 0, s>>>(p, in, out, slot); \
    return cudaGetLastError();                                                    \
  }
  ADOT_STEP2_CASE(256, 64)
  ADOT_STEP2_CASE(128, 64)
  ADOT_STEP2_CASE(128, 72)
  ADOT_STEP2_CASE(256, 80)
#undef ADOT_STEP2_CASE
  return cudaErrorInvalidValue;
}

template <typename R>
cudaError_t launch_step2_impl(const StepParams& p, int law, StepVariant v,
                              typename Prec<R>::State in, typename Prec<R>::State out, int slot,
                              cudaStream_t s) {
  if (law == LAW_GRASS) return launch_step2_law<R, LAW_GRASS>(p, v, in, out, slot, s);
  if (law == LAW_MPM) return launch_step2_law<R, LAW_MPM>(p, v, in, out, slot, s);
  if (law == LAW_GRASS_THR || law == LAW_POWER)
    return launch_step2_law<R, LAW_GRASS_THR>(p, v, in, out, slot, s);
  return cudaErrorInvalidValue;
}

}  // namespace adot
