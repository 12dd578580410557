// Fused time-step kernel of the A-DOT scheme, shared by the float32 and
// float64 translation units.
//
// Launch geometry: block b owns edges e = b*(B-1) + t, t = 0..B-1 (edge e
// joins cells e-1 and e; edges 0..n), and updates cells e-1 for t >= 1, i.e.
// B-1 cells per block, so one edge per block is evaluated twice and no other
// work is repeated. Per thread:
//   1. load cells e-1 and e (or a ghost / the periodic wrap at the ends);
//   2. D-/+ of edge e = 1/2 sum_k w_k (A_k dW -/+ |A_k| dW) over the three
//      Gauss-Legendre nodes of the segment path (Eq. path, Eq. DOTjumpN);
//   3. publish D+ in shared memory; after one barrier, cell e-1 takes its own
//      edge's D- and the left neighbour thread's D+ (Eq. scheme):
//      W_{e-1} <- W_{e-1} - dt/dx (D-_e + D+_{e-1});
//   4. spectral radius of the new state, block max, one 64-bit atomicMax
//      into the control slot that the next step reads for its dt.
// dt is formed once per block by thread 0 from the control slot:
// dt = cfl dx / rho_max, clipped so that t lands on t_end; once t >= t_end the
// kernel copies the state unchanged (the ping-pong buffers stay consistent).
#pragma once

#include <float.h>

#include <algorithm>
#include <type_traits>

#include "adot_internal.h"
#include "adot_math_x2.cuh"

namespace adot {

template <typename R>
struct Prec;

template <>
struct Prec<float> {
  using S = float2;
  using State = StateF32;
  __device__ static __forceinline__ float diff(S a, S b) { return ff_diff(a, b); }
  __device__ static __forceinline__ float hi(S a) { return a.x; }
  __device__ static __forceinline__ S add(S a, float d) { return ff_add(a, d); }
  __device__ static __forceinline__ S from_double(double d) { return ff_from_double(d); }
  __device__ static __forceinline__ unsigned long long bits(float r) {
    return (unsigned long long)__float_as_uint(r);
  }
  __device__ static __forceinline__ double from_bits(unsigned long long b) {
    return (double)__uint_as_float((unsigned)b);
  }
  // A NaN or infinity in the low word reaches the high word: set_state stores
  // lo = (float)(d - hi) of a finite d, and ff_add forms hi = s + lo.
  __device__ static __forceinline__ bool finite(S a) { return isfinite(a.x); }
  __device__ static __forceinline__ const LawT<float>& law(const StepParams& p) { return p.lf; }
  template <int LAW>
  __device__ static __forceinline__ float rho(const StepParams& p, float h, float q) {
    return spectral_radius_f32<LAW>(p.lf, h, q);
  }
};

template <>
struct Prec<double> {
  using S = double;
  using State = StateF64;
  __device__ static __forceinline__ double diff(S a, S b) { return a - b; }
  __device__ static __forceinline__ double hi(S a) { return a; }
  __device__ static __forceinline__ S add(S a, double d) { return a + d; }
  __device__ static __forceinline__ S from_double(double d) { return d; }
  __device__ static __forceinline__ unsigned long long bits(double r) {
    return (unsigned long long)__double_as_longlong(r);
  }
  __device__ static __forceinline__ double from_bits(unsigned long long b) {
    return __longlong_as_double((long long)b);
  }
  __device__ static __forceinline__ bool finite(S a) { return isfinite(a); }
  __device__ static __forceinline__ const LawT<double>& law(const StepParams& p) { return p.ld; }
  template <int LAW>
  __device__ static __forceinline__ double rho(const StepParams& p, double h, double q) {
    return spectral_radius<double, LAW>(p.ld, h, q);
  }
};

// Ghost state beyond one end: adj = the cell next to the end, nxt = the one
// after it (adj itself when the domain has one cell). BC_INFLOW_QS and
// BC_OUTFLOW_HS continue the bed slope, z_g = 2 z_adj - z_nxt, so a uniform
// flow on a constant slope meets the same bed step at the end edge as inside.
template <typename R, bool EXT = true>
__device__ __forceinline__ void ghost_state(int kind, const double v[3], double t,
                                            const typename Prec<R>::S adj[3],
                                            const typename Prec<R>::S& z_nxt,
                                            typename Prec<R>::S out[3]) {
  out[0] = adj[0];
  out[1] = adj[1];
  out[2] = adj[2];
  if (kind == BC_INFLOW_Q) {
    out[1] = Prec<R>::from_double(v[0]);
  } else if (kind == BC_OUTFLOW_H) {
    out[0] = Prec<R>::from_double(v[0]);
  } else if (kind == BC_INFLOW_QZ) {
    out[1] = Prec<R>::from_double(v[0]);
    out[2] = Prec<R>::from_double(v[1] - v[2] * t);
  } else if (EXT && (kind == BC_INFLOW_QS || kind == BC_OUTFLOW_HS)) {
    if (kind == BC_INFLOW_QS)
      out[1] = Prec<R>::from_double(v[0]);
    else
      out[0] = Prec<R>::from_double(v[0]);
    out[2] = Prec<R>::add(adj[2], Prec<R>::diff(adj[2], z_nxt));
  }
}

// States on both sides of edge e (joins cells e-1 and e), 0 <= e <= n. EXT:
// the slope-continuing ghosts are compiled in (the plain step kernels run only
// configurations without them).
template <typename R, bool EXT = true>
__device__ __forceinline__ void load_edge(const StepParams& p, const typename Prec<R>::State& st,
                                          int64_t e, int slot, typename Prec<R>::S wl[3],
                                          typename Prec<R>::S wr[3]) {
  const int64_t n = p.n;
  if (e > 0 && e < n) {
    wl[0] = st.h[e - 1];
    wl[1] = st.q[e - 1];
    wl[2] = st.z[e - 1];
    wr[0] = st.h[e];
    wr[1] = st.q[e];
    wr[2] = st.z[e];
  } else if (p.periodic) {
    const int64_t il = (e == 0) ? n - 1 : e - 1;
    const int64_t ir = (e == n) ? 0 : e;
    wl[0] = st.h[il];
    wl[1] = st.q[il];
    wl[2] = st.z[il];
    wr[0] = st.h[ir];
    wr[1] = st.q[ir];
    wr[2] = st.z[ir];
  } else if (e == 0) {
    wr[0] = st.h[0];
    wr[1] = st.q[0];
    wr[2] = st.z[0];
    if constexpr (EXT)
      ghost_state<R>(p.bc_left, p.bcl, p.ctl->s[slot].t, wr, st.z[n > 1 ? 1 : 0], wl);
    else
      ghost_state<R, false>(p.bc_left, p.bcl, p.ctl->s[slot].t, wr, wr[2], wl);
  } else {
    wl[0] = st.h[n - 1];
    wl[1] = st.q[n - 1];
    wl[2] = st.z[n - 1];
    if constexpr (EXT)
      ghost_state<R>(p.bc_right, p.bcr, p.ctl->s[slot].t, wl, st.z[n > 1 ? n - 2 : 0], wr);
    else
      ghost_state<R, false>(p.bc_right, p.bcr, p.ctl->s[slot].t, wl, wl[2], wr);
  }
}

// Sediment feed through an end (Sec. 5.1): the bed row of Eq. scheme is
// z_i -= dt/dx (F_{i+1/2} - F_{i-1/2}) with the edge discharge
// F_{i+1/2} = xi q_s(W_i) + D-_{i+1/2} = xi q_s(W_{i+1}) - D+_{i+1/2}; a feeding
// end's edge discharge is the imposed xi q_s,in, so the bed gains exactly what
// is fed. Edge 0: bed row of D+ = xi q_s(W_0) - xi q_s,in; edge n: bed row of
// D- = xi q_s,in - xi q_s(W_{n-1}). The h and q rows keep the edge against the
// ghost.
template <typename R, int LAW>
__device__ __forceinline__ void feed_edge(const StepParams& p, int64_t e,
                                          const typename Prec<R>::S wl[3],
                                          const typename Prec<R>::S wr[3], R dm[3], R dp[3]) {
  if (p.periodic) return;
  if (e == 0 && p.bc_left == BC_INFLOW_QS)
    dp[2] = sediment_xqs<R, LAW>(Prec<R>::law(p), Prec<R>::hi(wr[0]), Prec<R>::hi(wr[1])) -
            R(p.feed_l);
  if (e == p.n && p.bc_right == BC_INFLOW_QS)
    dm[2] = R(p.feed_r) -
            sediment_xqs<R, LAW>(Prec<R>::law(p), Prec<R>::hi(wl[0]), Prec<R>::hi(wl[1]));
}

// Momentum source of Eq. SV-Ex2 times dt at the step's starting state:
// -dt g h s_f, Strickler s_f = q|q| / (K_s^2 h^(10/3)) (Sec. 2), i.e.
// -dt (g / K_s^2) q|q| h^(-7/3).
template <typename R>
__device__ __forceinline__ R friction_dt(const StepParams& p, R dt, R h, R q) {
  const R ih = R(1) / h;
  return -dt * R(p.fric) * q * d_abs(q) * (ih * ih * d_rcbrt(h));
}

__device__ __forceinline__ int64_t d_min_i64(int64_t a, int64_t b) { return a < b ? a : b; }

template <typename R>
__device__ __forceinline__ R warp_max(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = d_max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Whether float32 edges evaluate the two outer Gauss-Legendre nodes in paired
// float32x2 instructions. Building with -DADOT_SCALAR_NODES gives the all-scalar
// form, whose per-opcode instruction counters (which do not count paired
// instructions) give the kernels' executed float32 flops; the arithmetic is the
// same, only the rounding order of the outer nodes differs.
#ifdef ADOT_SCALAR_NODES
constexpr bool kPairedNodes = false;
#else
constexpr bool kPairedNodes = true;
#endif

// D-/+ of one edge from its two states. PAIRED: float32 edges take the
// paired-instruction form of the two outer nodes (fewer issue slots, more
// registers); the ensemble kernel, held to 64 registers, keeps the scalar form.
// All-scalar float32 edge (as edge_fluct_f32x2_core with every node scalar):
// D-/+ in float32 and whether the edge needs the float64 redo.
template <int LAW>
__device__ __forceinline__ bool edge_fluct_f32_scalar_core(const LawT<float>& L, const float2 wl[3],
                                                           const float2 wr[3], float dm[3], float dp[3]) {
  const float dh = ff_diff(wr[0], wl[0]), dq = ff_diff(wr[1], wl[1]), dz = ff_diff(wr[2], wl[2]);
  const float h0 = wl[0].x, q0 = wl[1].x;
  float ya[3] = {0.0f, 0.0f, 0.0f}, xa[3] = {0.0f, 0.0f, 0.0f};
  bool redo = false;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float sk = (k == 0) ? (float)GL3_S0 : ((k == 1) ? 0.5f : (float)GL3_S2);
    const float w = (k == 1) ? (float)GL3_W1 : (float)GL3_W0;
    Eig<float> e;
    node_eig<float, LAW>(L, h0 + sk * dh, q0 + sk * dq, e);
    redo = redo || !(fmaf(-e.arg, e.arg, 1.0f) >= TAU_FP64_FALLBACK);
    float y[3], x[3];
    A_times(e, dh, dq, dz, y[0], y[1], y[2]);
    abs_A_times_proj(e, dh, dq, dz, y, x);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      ya[r] += w * y[r];
      xa[r] += w * x[r];
    }
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    dm[r] = 0.5f * (ya[r] - xa[r]);
    dp[r] = 0.5f * (ya[r] + xa[r]);
  }
  return redo;
}

// Float32 edge without the float64 redo: D-/+ from the float32 nodes and
// whether the edge needs float64 (the step kernel then leaves the two cells of
// the edge to k_fixup).
template <int LAW, bool PAIRED = kPairedNodes>
__device__ __forceinline__ bool edge_fluct_deferred(const StepParams& p, const float2 wl[3],
                                                    const float2 wr[3], float dm[3], float dp[3]) {
  if constexpr (PAIRED) return edge_fluct_f32x2_core<LAW>(p.lf, wl, wr, dm, dp);
  else return edge_fluct_f32_scalar_core<LAW>(p.lf, wl, wr, dm, dp);
}

template <typename R, int LAW, bool PAIRED = kPairedNodes>
__device__ __forceinline__ void edge_fluct(const StepParams& p, const typename Prec<R>::S wl[3],
                                           const typename Prec<R>::S wr[3], R dm[3], R dp[3],
                                           unsigned& flags) {
  if constexpr (PAIRED && std::is_same<R, float>::value) {
    edge_fluct_f32x2<LAW>(p.lf, p.ld, wl, wr, dm, dp, flags);
    return;
  } else if constexpr (std::is_same<R, float>::value) {
    // all-scalar float32 nodes; as in edge_fluct_f32x2, an edge with a node
    // whose roots nearly coalesce is redone in float64 as a whole
    if (edge_fluct_f32_scalar_core<LAW>(p.lf, wl, wr, dm, dp)) {
      const EdgeD d = edge_fluct_f64_redo<LAW>(p.ld, wl[0], wl[1], wl[2], wr[0], wr[1], wr[2]);
      flags |= d.flags;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        dm[r] = d.dm[r];
        dp[r] = d.dp[r];
      }
    }
  } else {
    const R dh = Prec<R>::diff(wr[0], wl[0]);
    const R dq = Prec<R>::diff(wr[1], wl[1]);
    const R dz = Prec<R>::diff(wr[2], wl[2]);
    const R h0 = Prec<R>::hi(wl[0]), q0 = Prec<R>::hi(wl[1]);
    R ya[3] = {R(0), R(0), R(0)}, xa[3] = {R(0), R(0), R(0)};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const R s = (k == 0) ? R(GL3_S0) : ((k == 1) ? R(0.5) : R(GL3_S2));
      const R w = (k == 1) ? R(GL3_W1) : R(GL3_W0);
      R y[3], x[3];
      node_f64<LAW>(p.ld, h0 + s * dh, q0 + s * dq, dh, dq, dz, y, x, flags);
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        ya[r] += w * y[r];
        xa[r] += w * x[r];
      }
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      dm[r] = R(0.5) * (ya[r] - xa[r]);
      dp[r] = R(0.5) * (ya[r] + xa[r]);
    }
  }
}

// D-/+ of one float32 edge whose |A|_Psi (row-major 3x3) comes from the
// surrogate: |A|_Psi dW replaces sum_k w_k |A_k| dW, and sum_k w_k A_k dW keeps
// its analytic form (Eq. DOTjumpN, segment path).
template <int LAW>
__device__ __forceinline__ void edge_fluct_sur(const StepParams& p, const float2 wl[3],
                                               const float2 wr[3], const float M[9], float dm[3],
                                               float dp[3]) {
  const float dh = ff_diff(wr[0], wl[0]), dq = ff_diff(wr[1], wl[1]), dz = ff_diff(wr[2], wl[2]);
  const float h0 = wl[0].x, q0 = wl[1].x;
  float ya[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float sk = (k == 0) ? (float)GL3_S0 : ((k == 1) ? 0.5f : (float)GL3_S2);
    const float w = (k == 1) ? (float)GL3_W1 : (float)GL3_W0;
    const float h = h0 + sk * dh, q = q0 + sk * dq;
    const float inv_h = __fdividef(1.0f, h);
    const float u = q * inv_h, c2 = p.lf.g * h;
    float a, b;
    sediment_derivs<float, LAW>(p.lf, h, q, inv_h, u, a, b);
    ya[0] += w * dq;
    ya[1] += w * ((c2 - u * u) * dh + 2.0f * u * dq + c2 * dz);
    ya[2] += w * (a * dh + b * dq);
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float x = M[3 * r] * dh + M[3 * r + 1] * dq + M[3 * r + 2] * dz;
    dm[r] = 0.5f * (ya[r] - x);
    dp[r] = 0.5f * (ya[r] + x);
  }
}

// PRICE-C fluctuations of one edge (Sec. 3.2, Eq. PRICEjump, AiPRICE, Apsi,
// Im): D-/+ = 1/4 [2 A^Psi -/+ (dx/dt) I_eps -/+ (dt/dx) (A^Psi)^2] dW. A^Psi is
// the 3-point Gauss-Legendre mean of A(Psi(s)) along the segment path, whose
// first row is (0, 1, 0) and whose other rows hold five entries:
//   row 1: (mean of c^2 - u^2, mean of 2u, mean of c^2),  row 2: (mean of a, mean of b, 0).
// The products are taken matrix-free: y = A^Psi dW, zz = A^Psi y = (A^Psi)^2 dW.
// nu = dt/dx and inv_nu = dx/dt come from the step; eps is p.price_eps. No
// eigen-solve: the per-node work is u, c^2 and the transport derivatives.
template <typename R, int LAW>
__device__ __forceinline__ void edge_fluct_price(const StepParams& p, R nu, R inv_nu,
                                                 const typename Prec<R>::S wl[3],
                                                 const typename Prec<R>::S wr[3], R dm[3], R dp[3]) {
  const R dh = Prec<R>::diff(wr[0], wl[0]);
  const R dq = Prec<R>::diff(wr[1], wl[1]);
  const R dz = Prec<R>::diff(wr[2], wl[2]);
  const R h0 = Prec<R>::hi(wl[0]), q0 = Prec<R>::hi(wl[1]);
  const auto& L = Prec<R>::law(p);
  R m10 = R(0), m11 = R(0), m12 = R(0), m20 = R(0), m21 = R(0);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const R sk = (k == 0) ? R(GL3_S0) : ((k == 1) ? R(0.5) : R(GL3_S2));
    const R w = (k == 1) ? R(GL3_W1) : R(GL3_W0);
    const R h = h0 + sk * dh, q = q0 + sk * dq;
    const R inv_h = R(1) / h;
    const R u = q * inv_h, c2 = L.g * h;
    R a, b;
    sediment_derivs<R, LAW>(L, h, q, inv_h, u, a, b);
    m10 += w * (c2 - u * u);
    m11 += w * (R(2) * u);
    m12 += w * c2;
    m20 += w * a;
    m21 += w * b;
  }
  const R y0 = dq;
  const R y1 = m10 * dh + m11 * dq + m12 * dz;
  const R y2 = m20 * dh + m21 * dq;
  const R z0 = y1;
  const R z1 = m10 * y0 + m11 * y1 + m12 * y2;
  const R z2 = m20 * y0 + m21 * y1;
  const R y[3] = {y0, y1, y2};
  const R zz[3] = {z0, z1, z2};
  const R v[3] = {dh, dq, R(p.price_eps) * dz};
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const R dis = R(0.25) * (inv_nu * v[r] + nu * zz[r]);
    dm[r] = R(0.5) * y[r] - dis;
    dp[r] = R(0.5) * y[r] + dis;
  }
}

// Resident blocks per SM requested from the register allocator: CAP registers
// per thread out of the SM's 65536, or no request (CAP = 0).
template <int B, int CAP>
struct MinBlocks {
  static constexpr int value = CAP ? 65536 / (B * CAP) : 1;
};

// EXT: the friction source and the sediment feed are compiled in (configs that
// use neither run the EXT = false kernels, whose register allocation they would
// otherwise share).
template <typename R, int LAW, int B, int CAP, bool SUR = false, bool EXT = false>
__global__ void __launch_bounds__(B, MinBlocks<B, CAP>::value) k_step(const StepParams p, const typename Prec<R>::State in,
                                            const typename Prec<R>::State out, const int slot) {
  using S = typename Prec<R>::S;
  __shared__ R sDp[3][B];
  __shared__ R sRed[B / 32];
  __shared__ R sNu;
  __shared__ int sDone;

  const int tid = threadIdx.x;
  const int64_t n = p.n;
  const int64_t e = (int64_t)blockIdx.x * (B - 1) + tid;
  Ctl* ctl = p.ctl;

  if (tid == 0) {
    const CtlSlot cs = ctl->s[slot];
    const double t_end = ctl->t_end;
    const bool done = !(cs.t < t_end);
    const double rho = Prec<R>::from_bits(cs.rho_bits);
    double dt = p.cfl * p.dx / rho;
    double tn = cs.t + dt;
    if (tn >= t_end) {
      dt = t_end - cs.t;
      tn = t_end;
    }
    sNu = done ? R(0) : R(dt / p.dx);
    sDone = done ? 1 : 0;
    if (blockIdx.x == 0) {
      CtlSlot& nx = ctl->s[(slot + 1) % 3];
      nx.t = done ? cs.t : tn;
      nx.dt = done ? cs.dt : dt;
      nx.steps = cs.steps + (done ? 0 : 1);
      if (done) nx.rho_bits = cs.rho_bits;
      ctl->s[(slot + 2) % 3].rho_bits = 0ull;
    }
  }

  unsigned flags = 0;
  S wl[3];
  R dm[3] = {R(0), R(0), R(0)}, dp[3] = {R(0), R(0), R(0)};
  if (e <= n) {
    S wr[3];
    load_edge<R, EXT>(p, in, e, slot, wl, wr);
    if constexpr (SUR) {
      float M[9];
#pragma unroll
      for (int r = 0; r < 9; ++r) M[r] = p.absA[(int64_t)r * (n + 1) + e];
      if (isnan(M[0]))
        edge_fluct<R, LAW>(p, wl, wr, dm, dp, flags);
      else
        edge_fluct_sur<LAW>(p, wl, wr, M, dm, dp);
    } else {
      edge_fluct<R, LAW>(p, wl, wr, dm, dp, flags);
    }
    if constexpr (EXT) feed_edge<R, LAW>(p, e, wl, wr, dm, dp);
  }
  sDp[0][tid] = dp[0];
  sDp[1][tid] = dp[1];
  sDp[2][tid] = dp[2];
  __syncthreads();

  const R nu = sNu;
  const bool done = sDone != 0;
  R rho = R(0);
  const int64_t i = e - 1;
  if (tid >= 1 && i < n) {
    S nh = wl[0], nq = wl[1], nz = wl[2];
    if (!done) {
      R iq = -nu * (dm[1] + sDp[1][tid - 1]);
      if constexpr (EXT)
        if (p.fric != 0.0)
          iq += friction_dt<R>(p, nu * R(p.dx), Prec<R>::hi(wl[0]), Prec<R>::hi(wl[1]));
      nh = Prec<R>::add(wl[0], -nu * (dm[0] + sDp[0][tid - 1]));
      nq = Prec<R>::add(wl[1], iq);
      nz = Prec<R>::add(wl[2], -nu * (dm[2] + sDp[2][tid - 1]));
    }
    out.h[i] = nh;
    out.q[i] = nq;
    out.z[i] = nz;
    if (!done) {
      const R hh = Prec<R>::hi(nh);
      if (!(hh > R(0))) flags |= ST_DEPTH;
      if (!(Prec<R>::finite(nh) && Prec<R>::finite(nq) && Prec<R>::finite(nz))) {
        flags |= ST_NONFINITE;
      } else if (hh > R(0)) {
        rho = Prec<R>::template rho<LAW>(p, hh, Prec<R>::hi(nq));
        if (!(rho <= R(3.0e38))) {
          flags |= ST_NONFINITE;
          rho = R(0);
        }
      }
    }
  }

  rho = warp_max(rho);
  if ((tid & 31) == 0) sRed[tid >> 5] = rho;
  __syncthreads();
  if (tid < 32) {
    rho = (tid < B / 32) ? sRed[tid] : R(0);
    rho = warp_max(rho);
    if (tid == 0 && !done && rho > R(0))
      atomicMax(&ctl->s[(slot + 1) % 3].rho_bits, Prec<R>::bits(rho));
  }
  if (flags) atomicOr(&ctl->status, flags);
}

// Step size of a warp-tile kernel: lane 0 forms dt = cfl dx / rho from the
// control slot (clipped to land on t_end) and the first warp of the grid writes
// the next slot; every warp gets nu = dt/dx and whether the run is done.
template <typename R>
__device__ __forceinline__ void warp_step_size(const StepParams& p, int slot, int lane,
                                               bool first_warp, R& nu, bool& done) {
  Ctl* ctl = p.ctl;
  R nu0 = R(0);
  int done0 = 0;
  if (lane == 0) {
    const CtlSlot cs = ctl->s[slot];
    const double t_end = ctl->t_end;
    const bool d = !(cs.t < t_end);
    const double rho = Prec<R>::from_bits(cs.rho_bits);
    double dt = p.cfl * p.dx / rho;
    double tn = cs.t + dt;
    if (tn >= t_end) {
      dt = t_end - cs.t;
      tn = t_end;
    }
    nu0 = d ? R(0) : R(dt / p.dx);
    done0 = d ? 1 : 0;
    if (first_warp) {
      CtlSlot& nx = ctl->s[(slot + 1) % 3];
      nx.t = d ? cs.t : tn;
      nx.dt = d ? cs.dt : dt;
      nx.steps = cs.steps + (d ? 0 : 1);
      if (d) nx.rho_bits = cs.rho_bits;
      ctl->s[(slot + 2) % 3].rho_bits = 0ull;
    }
  }
  nu = __shfl_sync(0xffffffffu, nu0, 0);
  done = __shfl_sync(0xffffffffu, done0, 0) != 0;
}

// Share of a warp's chunks taken as one static contiguous range (in eighths)
// and the chunks per pool group, per jump function. Measured on the 1e7-cell
// smooth workload with the split formed on the host (cell-updates/s):
//  DOT: 3/8 6.01e10, 4/8 6.03e10, 5/8 5.81e10, 6/8 5.61e10, 7/8 5.28e10 (groups
//  of 2 chunks); at 5/8 groups of 1, 2, 4 chunks 5.54, 5.81, 5.84e10; 4/8 with 3
//  or 4 chunks 6.00e10 or 5.96e10; 3/8 with 3 chunks 6.03e10 (4/8 with 2 chunks
//  measured 6.02-6.03e10 in the same runs).
//  PRICE-C: 4/8 with groups of 2 or 4 chunks 8.19e10 or 9.64e10, 5/8 8.62e10 or
//  9.32e10, 6/8 8.56e10 (2 chunks); a pool of single chunks loses to
//  contention on the counter at PRICE-C's rate (6.6e10 at 5/8).
// Static groups interleaved over the warps instead of contiguous ranges
// measured at most 4.97e10 (DOT, before the host-side split). Measurement
// builds may set other values (-DADOT_STATIC_EIGHTHS=k, -DADOT_POOL_CHUNKS=c,
// -DADOT_PRICE_STATIC_EIGHTHS=k, -DADOT_PRICE_POOL_CHUNKS=c).
#ifndef ADOT_STATIC_EIGHTHS
#define ADOT_STATIC_EIGHTHS 4
#endif
#ifndef ADOT_POOL_CHUNKS
#define ADOT_POOL_CHUNKS 2
#endif
#ifndef ADOT_PRICE_STATIC_EIGHTHS
#define ADOT_PRICE_STATIC_EIGHTHS 4
#endif
#ifndef ADOT_PRICE_POOL_CHUNKS
#define ADOT_PRICE_POOL_CHUNKS 4
#endif
template <int SCHEME>
struct SplitShape {
  static constexpr int eighths = SCHEME == 1 ? ADOT_PRICE_STATIC_EIGHTHS : ADOT_STATIC_EIGHTHS;
  static constexpr int pool_chunks = SCHEME == 1 ? ADOT_PRICE_POOL_CHUNKS : ADOT_POOL_CHUNKS;
};

// Programmatic dependent launch: the float32 warp-tile step and k_fixup are
// launched with programmatic stream serialisation, so that each can be
// scheduled while the kernel before it drains. griddep_wait() blocks until the
// kernel before has completed and its writes are visible (a no-op for a normal
// launch), and comes before a kernel's first read of the control block or the
// state; griddep_launch() lets the next kernel be scheduled.
#ifndef ADOT_PDL
#define ADOT_PDL 1
#endif
__device__ __forceinline__ void griddep_wait() {
#if ADOT_PDL
  asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}
__device__ __forceinline__ void griddep_launch() {
#if ADOT_PDL
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), unsigned grid, unsigned block, cudaStream_t s,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = ADOT_PDL;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// The split of a warp-tile launch, the same for every warp: cells per static
// range, the cells [0, n_s) the static ranges cover, and the pool's groups.
// Formed on the host per launch: the kernel formed it with three 64-bit
// divisions at every pool group (5.50 -> 5.58e10 cell-updates/s at 1e7 cells
// when they left the kernel).
struct WarpSplit {
  int64_t cs, n_s, n_groups;
};

template <int SCHEME>
inline WarpSplit warp_split(int64_t n, int64_t nwarps) {
  WarpSplit w;
  int64_t ks = (((n + 31) / 32) * SplitShape<SCHEME>::eighths / 8) / nwarps;
  if (ks < 2) ks = 0;
  w.cs = 32 * ks - 1;
  w.n_s = ks ? std::min<int64_t>(nwarps, n / w.cs) * w.cs : 0;
  constexpr int64_t kGroup = 32 * SplitShape<SCHEME>::pool_chunks - 1;
  w.n_groups = (n - w.n_s + kGroup - 1) / kGroup;
  return w;
}

// Persistent warp-tile variant of the time step. A warp processes ranges of
// consecutive edges in chunks of 32 (one per lane): the edge of lane l in
// chunk j of a range starting at edge E is E + 32 j + l, and the lane updates
// cell e - 1 with D- of its own edge and D+ of edge e - 1, taken from lane
// l - 1 by a shuffle or, in lane 0, carried over from lane 31 of the previous
// chunk. A range of k chunks updates 32 k - 1 cells, and consecutive ranges
// share one edge (the only edge evaluated twice).
//  - static part: with W warps and K = n / 32 chunks, each warp first takes a
//    contiguous range of k_s = floor((e/8) K / W) chunks (none when k_s < 2;
//    e = SplitShape<SCHEME>::eighths, 4 for both jump functions),
//    so cells [0, N_s) with N_s = W' (32 k_s - 1), W' <= W; warp w of block b
//    takes range w G + b (G blocks), so neighbouring ranges run on different
//    SMs;
//  - work pool: cells [N_s, n) in groups of 32 c - 1 cells (c chunks: 2 for the
//    DOT edge, 4 for PRICE-C's cheaper one), handed out by
//    an atomic counter in the control block; a warp asks for its next group
//    before it computes the current one, so the atomic's latency is hidden.
// The pool evens out the warps' finishing times: with static ranges alone the
// schedulers were active 92.6 % of a step at N = 1e7 (SM active cycles from
// 391k to 426k of 430k), waiting for the slowest ranges. Every warp's
// requests end with exactly one that finds the pool empty, so a launch takes
// n_groups + W tickets; the warp holding the last one puts the counter back to
// 0 for the next launch. Warps never wait for
// one another; each keeps its CFL maximum in a register and folds it into the
// control slot once at the end. Which warp evaluates an edge does not change
// its value, so the results do not depend on the split.
//
// SCHEME 0 evaluates the DOT edge of Eq. DOTjumpN; SCHEME 1 the PRICE-C edge
// (edge_fluct_price), everything else unchanged.
template <typename R, int LAW, int B, int CAP, bool EXT = false, int SCHEME = 0, bool DEFER = false>
__global__ void __launch_bounds__(B, MinBlocks<B, CAP>::value)
    k_step_warp(const StepParams p, const typename Prec<R>::State in,
                const typename Prec<R>::State out, const int slot, const WarpSplit ws) {
  using S = typename Prec<R>::S;
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * B + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * B) >> 5;
  const int64_t n = p.n;
  Ctl* ctl = p.ctl;

  griddep_wait();  // the previous kernel's state, control slot and counters
  // first pool ticket, asked for before anything else (used after the static range)
  unsigned ticket = 0u;
  if (lane == 0) ticket = atomicAdd(&ctl->grab, 1u);

  R nu;
  bool done;
  warp_step_size<R>(p, slot, lane, gw == 0, nu, done);
  const R inv_nu = (SCHEME == 1 && !done) ? R(1) / nu : R(0);  // dx/dt of Eq. AiPRICE

  // Lane 0 carries D+ of the previous chunk's last edge: in registers, or with
  // the friction/feed/ghost extension compiled in, in shared memory (lane 0 is
  // the only reader), which frees three registers at the 64 cap and costs the
  // plain kernel a shared-memory round trip per chunk.
  constexpr bool kSharedCarry = EXT;
  __shared__ R s_carry[kSharedCarry ? B / 32 : 1][3];
  R carry[3] = {R(0), R(0), R(0)};

  unsigned flags = 0;
  R rho_run = R(0);
  bool carry_rd = false;  // DEFER: lane 0's flag of the previous chunk's last edge
  // the split (warp_split): static ranges of ws.cs cells over cells [0, ws.n_s),
  // then ws.n_groups pool groups
  constexpr int64_t kGroup = 32 * SplitShape<SCHEME>::pool_chunks - 1;  // cells per pool group
  // current range: next chunk's first edge eb, rem = edges after it (< 2^31;
  // negative when the range is finished)
  int64_t eb = 0;
  int rem = -1;
  {
    // range ri = w G + b for warp w of block b (G blocks): consecutive ranges
    // belong to different blocks, so to different SMs, and a run of expensive
    // cells (edges redone in float64 near critical flow) is spread over the GPU
    const int64_t ri = (int64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x;
    if ((ri + 1) * ws.cs <= ws.n_s) {
      eb = ri * ws.cs;
      rem = (int)ws.cs;
    }
  }
  bool lead = lane >= 1;  // the lane's cell is in the range (all lanes after the first chunk)
  for (;;) {
    if (rem < 0) {
      // next range from the pool
      const int64_t g = (int64_t)__shfl_sync(0xffffffffu, ticket, 0);
      if (g >= ws.n_groups) {
        // the launch's last ticket: every other request has been served
        if (lane == 0 && g == ws.n_groups + nwarps - 1) atomicExch(&ctl->grab, 0u);
        break;
      }
      if (lane == 0) ticket = atomicAdd(&ctl->grab, 1u);
      eb = ws.n_s + g * kGroup;
      rem = (int)d_min_i64(kGroup, n - eb);
      lead = lane >= 1;
    }
    const int64_t e = eb + lane;
    const bool in_range = lane <= rem;
    {
      // the range's next chunk into L2 while this one is computed
      const int64_t cn = e + 31;
      if (rem >= 32 && cn < n) {
        // (into L1 instead, or also the next pool group's first chunk at a
        // range's last one: no gain, or 0.5 % and 2 % (PRICE-C) slower at 1e7 cells)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(in.h + cn));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(in.q + cn));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(in.z + cn));
      }
    }
    S wl[3];
    R dm[3] = {R(0), R(0), R(0)}, dp[3] = {R(0), R(0), R(0)};
    bool rd = false;  // DEFER: this edge needs the float64 redo
    if (in_range) {
      S wr[3];
      load_edge<R, EXT>(p, in, e, slot, wl, wr);
      if constexpr (SCHEME == 1)
        edge_fluct_price<R, LAW>(p, nu, inv_nu, wl, wr, dm, dp);
      else if constexpr (DEFER && std::is_same<R, float>::value)
        rd = edge_fluct_deferred<LAW>(p, wl, wr, dm, dp);
      else
        edge_fluct<R, LAW>(p, wl, wr, dm, dp, flags);
      if constexpr (EXT) feed_edge<R, LAW>(p, e, wl, wr, dm, dp);
    }
    R dl[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const R up = __shfl_sync(0xffffffffu, dp[r], (lane + 31) & 31);
      if constexpr (kSharedCarry) {
        dl[r] = up;
        if (lane == 0) {
          R* sc = s_carry[threadIdx.x >> 5];
          if (lead) dl[r] = sc[r];
          sc[r] = up;  // D+ of this chunk's last edge
        }
      } else {
        dl[r] = lane ? up : carry[r];
        carry[r] = up;  // lane 0: D+ of this chunk's last edge
      }
    }
    const int64_t i = e - 1;
    // DEFER: a cell with an edge that needs the float64 redo (its own, or the
    // previous lane's / previous chunk's) is not written here but listed for
    // k_fixup, which recomputes it from the same input state
    bool fix = false;
    if constexpr (DEFER) {
      const bool up_rd = __shfl_sync(0xffffffffu, rd, (lane + 31) & 31);
      const bool rd_left = lane ? up_rd : carry_rd;
      carry_rd = up_rd;
      fix = !done && (rd || rd_left);
      const unsigned m = __ballot_sync(0xffffffffu, lead && in_range && fix);
      if (m) {
        unsigned base = 0u;
        if (lane == 0) base = atomicAdd(&ctl->fix_count, (unsigned)__popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (lead && in_range && fix) p.fix_list[base + __popc(m & ((1u << lane) - 1u))] = (unsigned)i;
      }
    }
    if (lead && in_range && !fix) {
      S nh = wl[0], nq = wl[1], nz = wl[2];
      if (!done) {
        R iq = -nu * (dm[1] + dl[1]);
        if constexpr (EXT)
          if (p.fric != 0.0)
            iq += friction_dt<R>(p, nu * R(p.dx), Prec<R>::hi(wl[0]), Prec<R>::hi(wl[1]));
        nh = Prec<R>::add(wl[0], -nu * (dm[0] + dl[0]));
        nq = Prec<R>::add(wl[1], iq);
        nz = Prec<R>::add(wl[2], -nu * (dm[2] + dl[2]));
      }
      out.h[i] = nh;
      out.q[i] = nq;
      out.z[i] = nz;
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
    lead = true;
    eb += 32;
    rem -= 32;
  }
  griddep_launch();  // k_fixup may be scheduled (it waits for this grid to complete)
  rho_run = warp_max(rho_run);
  if (lane == 0 && !done && rho_run > R(0))
    atomicMax(&ctl->s[(slot + 1) % 3].rho_bits, Prec<R>::bits(rho_run));
  if (flags) atomicOr(&ctl->status, flags);
}

// The cells the float32 warp-tile step left (an edge of theirs needs the
// float64 redo): each is recomputed from the step's input state, both of its
// edges evaluated as the step evaluates an edge (float32 nodes, or, when
// flagged, the three nodes in float64 as edge_fluct_f64_redo forms them) with
// the step's nu, and written; its CFL radius goes into the next slot. Spread
// over the grid and over one lane per node, the float64 work no longer queues
// up in the warps whose ranges cross a near-critical region. The last block to
// finish puts the list's counters back to 0 for the next step.
template <int LAW, bool EXT>
__global__ void __launch_bounds__(256) k_fixup(const StepParams p, const StateF32 in, const StateF32 out,
                                               const int slot) {
  __shared__ float sRed[8];
  Ctl* ctl = p.ctl;
  griddep_wait();    // the step kernel has completed: its list and counters are visible
  griddep_launch();  // the next step may be scheduled (it waits for this grid to complete)
  const unsigned count = ctl->fix_count;
  // nothing listed (the usual step): the counters are already 0. Otherwise every
  // block reads the same count, since the reset below waits for all of them.
  if (count == 0u) return;
  // nu and done exactly as warp_step_size forms them
  const CtlSlot cs = ctl->s[slot];
  const double t_end = ctl->t_end;
  const bool done = !(cs.t < t_end);
  double dt = p.cfl * p.dx / Prec<float>::from_bits(cs.rho_bits);
  if (cs.t + dt >= t_end) dt = t_end - cs.t;
  const float nu = done ? 0.0f : (float)(dt / p.dx);
  unsigned flags = 0;
  float rho_run = 0.0f;
  // six lanes per listed cell (five cells per warp, lanes 30 and 31 idle): lane
  // 6 c + 3 side + k takes edge i + side of cell c (the left edge i, or the right
  // edge i + 1) and Gauss-Legendre node k. The three lanes of an edge each
  // evaluate its float32 nodes; when the edge needs the float64 redo, each
  // evaluates its own node in float64 and the first gathers the three (the
  // accumulation of edge_fluct_f64_redo, in the same order), so a cell waits
  // for one float64 node, not an edge's three in turn. Lane 6 c updates the
  // cell. The loop is warp-uniform; warp w of block b takes the cells of slot
  // w G + b (G blocks), so neighbouring slots run on different SMs.
  const int lane = threadIdx.x & 31;
  const int cl = lane / 6, side = (lane % 6) / 3, k = lane % 3;
  const unsigned long long n_c = done ? 0ull : (unsigned long long)count;
  const unsigned long long stride = (unsigned long long)gridDim.x * (blockDim.x >> 5) * 5ull;
  const unsigned long long slot0 = (unsigned long long)(threadIdx.x >> 5) * gridDim.x + blockIdx.x;
  for (unsigned long long c0 = slot0 * 5ull; c0 < n_c; c0 += stride) {
    const unsigned long long c = c0 + (unsigned long long)cl;
    const bool active = lane < 30 && c < n_c;
    int64_t i = 0;
    float2 wa[3], wb[3];
    float dm[3] = {0.0f, 0.0f, 0.0f}, dp[3] = {0.0f, 0.0f, 0.0f};
    bool rd = false;
    int64_t e = 0;
    if (active) {
      i = p.fix_list[c];
      e = i + side;  // left edge i (cells i - 1 | i) or right edge i + 1 (cells i | i + 1)
      load_edge<float, EXT>(p, in, e, slot, wa, wb);
      rd = edge_fluct_deferred<LAW>(p, wa, wb, dm, dp);
    }
    if (__any_sync(0xffffffffu, rd)) {
      double y[3] = {0.0, 0.0, 0.0}, x[3] = {0.0, 0.0, 0.0};
      if (rd) {
        const double hl = ff_to_double(wa[0]), ql = ff_to_double(wa[1]), zl = ff_to_double(wa[2]);
        const double dh = ff_to_double(wb[0]) - hl, dq = ff_to_double(wb[1]) - ql,
                     dz = ff_to_double(wb[2]) - zl;
        const double sk = (k == 0) ? GL3_S0 : ((k == 1) ? 0.5 : GL3_S2);
        node_f64<LAW>(p.ld, hl + sk * dh, ql + sk * dq, dh, dq, dz, y, x, flags);
      }
      double y1[3], y2[3], x1[3], x2[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        y1[r] = __shfl_down_sync(0xffffffffu, y[r], 1);
        y2[r] = __shfl_down_sync(0xffffffffu, y[r], 2);
        x1[r] = __shfl_down_sync(0xffffffffu, x[r], 1);
        x2[r] = __shfl_down_sync(0xffffffffu, x[r], 2);
      }
      if (rd && k == 0) {
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          double ya = 0.0, xa = 0.0;
          ya += GL3_W0 * y[r];
          xa += GL3_W0 * x[r];
          ya += GL3_W1 * y1[r];
          xa += GL3_W1 * x1[r];
          ya += GL3_W0 * y2[r];
          xa += GL3_W0 * x2[r];
          dm[r] = (float)(0.5 * (ya - xa));
          dp[r] = (float)(0.5 * (ya + xa));
        }
      }
    }
    if constexpr (EXT)
      if (active) feed_edge<float, LAW>(p, e, wa, wb, dm, dp);
    // D- of the right edge (lane 6 c + 3) to the cell's lane 6 c
    float dmR[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) dmR[r] = __shfl_down_sync(0xffffffffu, dm[r], 3);
    if (active && side == 0 && k == 0) {
      // the step kernel's update of cell i: state wb (the left edge's right cell),
      // D+ of the left edge (dp) and D- of the right edge (dmR)
      float iq = -nu * (dmR[1] + dp[1]);
      if constexpr (EXT)
        if (p.fric != 0.0) iq += friction_dt<float>(p, nu * float(p.dx), wb[0].x, wb[1].x);
      const float2 nh = Prec<float>::add(wb[0], -nu * (dmR[0] + dp[0]));
      const float2 nq = Prec<float>::add(wb[1], iq);
      const float2 nz = Prec<float>::add(wb[2], -nu * (dmR[2] + dp[2]));
      out.h[i] = nh;
      out.q[i] = nq;
      out.z[i] = nz;
      const float hh = nh.x;
      if (!(hh > 0.0f)) flags |= ST_DEPTH;
      if (!(Prec<float>::finite(nh) && Prec<float>::finite(nq) && Prec<float>::finite(nz))) {
        flags |= ST_NONFINITE;
      } else if (hh > 0.0f) {
        float r = Prec<float>::template rho<LAW>(p, hh, nq.x);
        if (!(r <= 3.0e38f)) {
          flags |= ST_NONFINITE;
          r = 0.0f;
        }
        rho_run = d_max(rho_run, r);
      }
    }
  }
  rho_run = warp_max(rho_run);
  if ((threadIdx.x & 31) == 0) sRed[threadIdx.x >> 5] = rho_run;
  __syncthreads();
  if (threadIdx.x < 32) {
    float r = (threadIdx.x < 8) ? sRed[threadIdx.x] : 0.0f;
    r = warp_max(r);
    if (threadIdx.x == 0 && r > 0.0f) atomicMax(&ctl->s[(slot + 1) % 3].rho_bits, Prec<float>::bits(r));
  }
  if (flags) atomicOr(&ctl->status, flags);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&ctl->fix_done, 1u) == gridDim.x - 1) {
      ctl->fix_count = 0u;
      ctl->fix_done = 0u;
      __threadfence();
    }
  }
}
#ifndef ADOT_FIXUP_BLOCKS
#define ADOT_FIXUP_BLOCKS 304
#endif
// k_fixup blocks: 2 per SM (measurement builds: -DADOT_FIXUP_BLOCKS=n)
constexpr unsigned kFixupBlocks = ADOT_FIXUP_BLOCKS;

// CFL maximum and admissibility of a state (grid-stride).
template <typename R, int LAW>
__global__ void __launch_bounds__(256) k_rho(const StepParams p, const typename Prec<R>::State st,
                                             const int slot) {
  __shared__ R sRed[8];
  unsigned flags = 0;
  R rho = R(0);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.n;
       i += (int64_t)gridDim.x * blockDim.x) {
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
    R r = Prec<R>::template rho<LAW>(p, hh, Prec<R>::hi(q));
    if (!(r <= R(3.0e38))) {
      flags |= ST_NONFINITE;
      continue;
    }
    rho = d_max(rho, r);
  }
  rho = warp_max(rho);
  if ((threadIdx.x & 31) == 0) sRed[threadIdx.x >> 5] = rho;
  __syncthreads();
  if (threadIdx.x < 32) {
    rho = (threadIdx.x < 8) ? sRed[threadIdx.x] : R(0);
    rho = warp_max(rho);
    if (threadIdx.x == 0 && rho > R(0)) atomicMax(&p.ctl->s[slot].rho_bits, Prec<R>::bits(rho));
  }
  if (flags) atomicOr(&p.ctl->status, flags);
}

template <typename R, int LAW, bool EXT>
cudaError_t launch_step_law(const StepParams& p, StepVariant v, typename Prec<R>::State in,
                            typename Prec<R>::State out, int slot, cudaStream_t s) {
  if (p.ctl == nullptr || p.n < 1) return cudaErrorInvalidValue;
  // edges 0..n, B-1 new edges per block: ceil((n+1)/(B-1)) blocks
  const int64_t cells = v.block - 1;
  const int64_t g = (p.n + 1 + cells - 1) / cells;
  if (g > 0x7fffffffLL) return cudaErrorInvalidValue;
  const unsigned G = (unsigned)g;
  if (v.warp_tiles) {
    // resident grid: blocks per SM from the register cap, times the SM count
    int sms = 152, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t per_sm = v.reg_cap ? 65536 / (v.block * v.reg_cap) : 1;  // = MinBlocks
    const int64_t tiles = (p.n + 30) / 31;
    const int64_t wpb = v.block / 32;
    int64_t gg = (tiles + wpb - 1) / wpb;
    if (gg > sms * per_sm) gg = sms * per_sm;
    // float32: the deferred form (flagged cells listed for k_fixup, launched
    // right after); float64 evaluates every edge in place
    constexpr bool kDefer = std::is_same<R, float>::value;
    if (kDefer && p.fix_list == nullptr) return cudaErrorInvalidValue;
    const WarpSplit ws = warp_split<0>(p.n, gg * (v.block / 32));
    cudaError_t e = cudaErrorInvalidValue;
    if (v.block == 256 && v.reg_cap == 64) {
      e = launch_pdl(k_step_warp<R, LAW, 256, 64, EXT, 0, kDefer>, (unsigned)gg, 256u, s, p, in, out, slot, ws);
    } else if (v.block == 128 && v.reg_cap == 64) {
      e = launch_pdl(k_step_warp<R, LAW, 128, 64, EXT, 0, kDefer>, (unsigned)gg, 128u, s, p, in, out, slot, ws);
    } else if (v.block == 128 && v.reg_cap == 72) {
      e = launch_pdl(k_step_warp<R, LAW, 128, 72, EXT, 0, kDefer>, (unsigned)gg, 128u, s, p, in, out, slot, ws);
    } else if (v.block == 256 && v.reg_cap == 80) {
      e = launch_pdl(k_step_warp<R, LAW, 256, 80, EXT, 0, kDefer>, (unsigned)gg, 256u, s, p, in, out, slot, ws);
    }
    if constexpr (kDefer) {
      if (e == cudaSuccess) {
        e = launch_pdl(k_fixup<LAW, EXT>, kFixupBlocks, 256u, s, p, in, out, slot);
      }
    }
    return e;
  }
#define ADOT_STEP_CASE(BB, CC)                                       \
  if (v.block == BB && v.reg_cap == CC) {                            \
    k_step<R, LAW, BB, CC, false, EXT><<<G, BB, 0, s>>>(p, in, out, slot); \
    return cudaGetLastError();                                       \
  }
  ADOT_STEP_CASE(128, 0)
  ADOT_STEP_CASE(128, 64)
  ADOT_STEP_CASE(256, 0)
  ADOT_STEP_CASE(256, 64)
  ADOT_STEP_CASE(512, 0)
  ADOT_STEP_CASE(512, 64)
#undef ADOT_STEP_CASE
  return cudaErrorInvalidValue;
}

template <typename R, bool EXT>
cudaError_t launch_step_impl(const StepParams& p, int law, StepVariant v, typename Prec<R>::State in,
                             typename Prec<R>::State out, int slot, cudaStream_t s) {
  if (law == LAW_GRASS) return launch_step_law<R, LAW_GRASS, EXT>(p, v, in, out, slot, s);
  if (law == LAW_MPM) return launch_step_law<R, LAW_MPM, EXT>(p, v, in, out, slot, s);
  if (law == LAW_GRASS_THR || law == LAW_POWER)
    return launch_step_law<R, LAW_GRASS_THR, EXT>(p, v, in, out, slot, s);
  return cudaErrorInvalidValue;
}

template <typename R>
cudaError_t launch_rho_impl(const StepParams& p, int law, typename Prec<R>::State st, int slot,
                            cudaStream_t s) {
  if (p.ctl == nullptr || p.n < 1) return cudaErrorInvalidValue;
  int64_t g = (p.n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  if (g < 1) g = 1;
  if (law == LAW_GRASS)
    k_rho<R, LAW_GRASS><<<(unsigned)g, 256, 0, s>>>(p, st, slot);
  else if (law == LAW_MPM)
    k_rho<R, LAW_MPM><<<(unsigned)g, 256, 0, s>>>(p, st, slot);
  else if (law == LAW_GRASS_THR || law == LAW_POWER)
    k_rho<R, LAW_GRASS_THR><<<(unsigned)g, 256, 0, s>>>(p, st, slot);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace adot
