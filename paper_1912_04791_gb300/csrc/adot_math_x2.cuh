// Float32 edge fluctuations with paired instructions: the two outer
// Gauss-Legendre nodes s0 and s2 of Eq. DOTjumpN (equal weights) are evaluated
// together, one per half of a float2, through the paired float32 add, multiply
// and fused multiply-add of this architecture (__fadd2_rn, __fmul2_rn,
// __ffma2_rn: one issue slot for two lanes of work). The reciprocal, square
// root, arccos and sincos steps and the choice of the root taken from the
// product of the roots stay per lane. The midpoint node takes the scalar path.
// The arithmetic is that of the scalar nodes (Eq. charPol/lambda, Eq. RR, RR-1,
// Eq. asbA through one spectral projector), with the same identities; an edge
// with a node whose roots nearly coalesce is redone in float64 as a whole.
#pragma once

#include "adot_math.cuh"

namespace adot {

__device__ __forceinline__ float2 p2(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as one paired instruction (a negated operand would cost two scalar ones)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 abs2(float2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
__device__ __forceinline__ float2 rcp2(float2 a) {
  return make_float2(__fdividef(1.0f, a.x), __fdividef(1.0f, a.y));
}
__device__ __forceinline__ float2 nrcp2(float2 a) {  // -1/a
  return make_float2(__fdividef(-1.0f, a.x), __fdividef(-1.0f, a.y));
}

// Eigen-data of A at two states (one per lane); see Eig.
struct Eig2 {
  float2 u, c2, inv_c2, na, b;  // na = -a
  float2 l1, l2, l3;
  float2 arg;
};

// Steps 1-3 of node_eig for two states.
template <int LAW>
__device__ __forceinline__ void node_eig_x2(const LawT<float>& L, float2 h, float2 q, Eig2& e) {
  const float2 inv_h = make_float2(1.0f / h.x, 1.0f / h.y);
  const float2 u = mul2(q, inv_h);
  const float2 c2 = mul2(p2(L.g), h);
  const float2 rc = make_float2(rsqrtf(c2.x), rsqrtf(c2.y));  // 1/c
  const float2 c = mul2(c2, rc);
  const float2 Fr = mul2(u, rc);
  float2 na, b;  // na = -a = -dq_s/dh, b = dq_s/dq
  if constexpr (LAW == LAW_GRASS) {
    b = mul2(mul2(mul2(p2(L.K3), u), u), inv_h);
    na = mul2(b, u);
  } else {
    float ax, ay;
    sediment_derivs<float, LAW>(L, h.x, q.x, inv_h.x, u.x, ax, b.x);
    sediment_derivs<float, LAW>(L, h.y, q.y, inv_h.y, u.y, ay, b.y);
    na = make_float2(-ax, -ay);
  }
  const float2 Fr2 = mul2(Fr, Fr);
  const float2 k1 = fma2(p2(3.0f), b, fma2(Fr, Fr, p2(3.0f)));
  // k2 = Fr (18 (1 + b) - 2 Fr^2) + 27 a / c
  const float2 k2 = fma2(Fr, fma2(p2(18.0f), b, fma2(p2(-2.0f), Fr2, p2(18.0f))),
                         mul2(p2(-27.0f), mul2(na, rc)));
  const float2 rk = make_float2(rsqrtf(k1.x), rsqrtf(k1.y));
  const float2 arg = mul2(mul2(p2(0.5f), k2), mul2(mul2(rk, rk), rk));
  const float ax = fminf(fmaxf(arg.x, -1.0f), 1.0f), ay = fminf(fmaxf(arg.y, -1.0f), 1.0f);
  float2 S, C;
#ifdef ADOT_ACOS_LIBRARY
  __sincosf(acos_third(ax), &S.x, &C.x);
  __sincosf(acos_third(ay), &S.y, &C.y);
#else
  {
    // acos_third of both lanes with the polynomial in paired instructions
    const float2 aa = make_float2(fabsf(ax), fabsf(ay));
    float2 pp = p2(acos3_coef(7));
#pragma unroll
    for (int i = 6; i >= 0; --i) pp = fma2(pp, aa, p2(acos3_coef(i)));
    const float2 sq = make_float2(sqrtf(1.0f - aa.x), sqrtf(1.0f - aa.y));
    const float2 r = mul2(sq, pp);
    __sincosf(ax >= 0.0f ? r.x : kPi3 - r.x, &S.x, &C.x);
    __sincosf(ay >= 0.0f ? r.y : kPi3 - r.y, &S.y, &C.y);
  }
#endif
  const float2 k1rk = mul2(k1, rk);                               // sqrt(k1)
  const float2 m = mul2(p2((float)(2.0 / 3.0)), k1rk);            // (2/3) sqrt(k1)
  const float2 nm = mul2(p2((float)(-2.0 / 3.0)), k1rk);
  const float2 F = mul2(p2((float)(2.0 / 3.0)), Fr);
  const float2 hc = mul2(p2(0.5f), C);
  const float2 hs = mul2(p2(0.86602540378443864676f), S);  // (sqrt 3 / 2) S
  const float2 l1 = mul2(c, fma2(nm, add2(hc, hs), F));  // cos(phi/3 - pi/3) = C/2 + (sqrt3/2) S
  const float2 l2 = mul2(c, fma2(nm, sub2(hc, hs), F));  // cos(phi/3 + pi/3) = C/2 - (sqrt3/2) S
  const float2 l3 = mul2(c, fma2(m, C, F));
  e.u = u;
  e.c2 = c2;
  e.inv_c2 = mul2(rc, rc);
  e.na = na;
  e.b = b;
  e.l1 = l1;
  e.l2 = l2;
  e.l3 = l3;
  e.arg = arg;
}

// A(W) dW for two states and one dW (Eq. W&A_definition).
__device__ __forceinline__ void A_times_x2(const Eig2& e, float dh, float dq, float dz, float2 y[3]) {
  y[0] = p2(dq);
  const float2 t = fma2(add2(e.u, e.u), p2(dq), mul2(e.c2, p2(dz)));
  y[1] = fma2(sub2(e.c2, mul2(e.u, e.u)), p2(dh), t);
  y[2] = fma2(e.na, p2(-dh), mul2(e.b, p2(dq)));
}

// The projector's root of one lane when it is the root of smallest magnitude
// (see abs_A_times_proj): from the product of the roots, l1 l2 l3 = c^2 a,
// unless l2 l_f = 0.
__device__ __forceinline__ float small_root(float lk, float l2, float lf, float c2, float na) {
  const float pr = l2 * lf;
  return (pr != 0.0f) ? -(c2 * na) / pr : lk;
}

// |A| dW for two states through one projector each, as abs_A_times_proj: the
// projector's root (l1 or l3), the sign and the small-root case are chosen per
// lane; one reciprocal per lane serves both quotients.
__device__ __forceinline__ void abs_A_times_proj_x2(const Eig2& e, float dh, float dq, float dz,
                                                    const float2 y[3], float2 x[3]) {
  const bool lox = e.l2.x >= 0.0f, loy = e.l2.y >= 0.0f;
  float2 lk = make_float2(lox ? e.l1.x : e.l3.x, loy ? e.l1.y : e.l3.y);
  const float2 lf = make_float2(lox ? e.l3.x : e.l1.x, loy ? e.l3.y : e.l1.y);
  const bool smx = fabsf(lk.x) <= fabsf(e.l2.x), smy = fabsf(lk.y) <= fabsf(e.l2.y);
  if (smx) lk.x = small_root(lk.x, e.l2.x, lf.x, e.c2.x, e.na.x);
  if (smy) lk.y = small_root(lk.y, e.l2.y, lf.y, e.c2.y, e.na.y);
  const float2 m2 = make_float2(lox ? -2.0f * fminf(lk.x, 0.0f) : -2.0f * fmaxf(lk.x, 0.0f),
                                loy ? -2.0f * fminf(lk.y, 0.0f) : -2.0f * fmaxf(lk.y, 0.0f));
  const float2 sg = make_float2(lox ? 1.0f : -1.0f, loy ? 1.0f : -1.0f);
  const float2 dk = mul2(sub2(lk, e.l2), sub2(lk, lf));
  // (l_k . dW) d_k = (l_k (l_k - 2u) - c^2 b) dh + l_k dq + c^2 dz
  const float2 ntu = mul2(e.u, p2(-2.0f));
  const float2 czb = mul2(e.c2, fma2(e.b, p2(-dh), p2(dz)));
  const float2 pk = fma2(mul2(lk, add2(lk, ntu)), p2(dh), fma2(lk, p2(dq), czb));
  const float2 mp = mul2(m2, pk);
  // small root: coef = m p_k / d_k, third entry of r_k = (u - l_k)^2 / c^2 - 1;
  // otherwise coef = m p_k l_k / (d_k l_k), coef r_k = m p_k (b l_k + a) / (d_k l_k)
  const float2 den = make_float2(smx ? dk.x : dk.x * lk.x, smy ? dk.y : dk.y * lk.y);
  const float2 inv = rcp2(den);
  const float2 coef = mul2(mp, make_float2(smx ? inv.x : lk.x * inv.x, smy ? inv.y : lk.y * inv.y));
  const float2 vk = sub2(e.u, lk);
  const float2 rdirect = fma2(mul2(vk, vk), e.inv_c2, p2(-1.0f));
  const float2 rquot = mul2(mul2(mp, fma2(e.b, lk, mul2(e.na, p2(-1.0f)))), inv);
  const float2 c2nd = make_float2(smx ? coef.x * rdirect.x : rquot.x,
                                  smy ? coef.y * rdirect.y : rquot.y);
  x[0] = mul2(sg, add2(y[0], coef));
  x[1] = mul2(sg, fma2(coef, lk, y[1]));
  x[2] = mul2(sg, add2(y[2], c2nd));
}

// Fluctuations of one edge, all in float64 (see edge_fluct_f32x2).
struct EdgeD {
  float dm[3], dp[3];
  unsigned flags;
};

// The float64 redo of a float32 edge: the float-float states summed to
// float64, the three nodes of Eq. DOTjumpN by node_f64 (the Newton form near
// coalescence, the non-hyperbolic flag), D-/+ rounded to float32. Kept out of
// line and called from one place, after the float32 nodes, with the states
// passed by value and the result returned by value, so that the float32 path
// around it keeps its values in registers.
template <int LAW>
__device__ __noinline__ EdgeD edge_fluct_f64_redo(const LawT<double>& Ld, float2 l0, float2 l1,
                                                  float2 l2, float2 r0, float2 r1, float2 r2) {
  const double hl = ff_to_double(l0), ql = ff_to_double(l1), zl = ff_to_double(l2);
  const double dh = ff_to_double(r0) - hl, dq = ff_to_double(r1) - ql, dz = ff_to_double(r2) - zl;
  double ya[3] = {0.0, 0.0, 0.0}, xa[3] = {0.0, 0.0, 0.0};
  EdgeD out;
  out.flags = 0u;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double sk = (k == 0) ? GL3_S0 : ((k == 1) ? 0.5 : GL3_S2);
    const double w = (k == 1) ? GL3_W1 : GL3_W0;
    double y[3], x[3];
    node_f64<LAW>(Ld, hl + sk * dh, ql + sk * dq, dh, dq, dz, y, x, out.flags);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      ya[r] += w * y[r];
      xa[r] += w * x[r];
    }
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    out.dm[r] = (float)(0.5 * (ya[r] - xa[r]));
    out.dp[r] = (float)(0.5 * (ya[r] + xa[r]));
  }
  return out;
}

// D-/+ of one float32 edge (float-float states wl, wr) from float32 nodes: s0
// and s2 paired, the midpoint node scalar. Returns whether any node has
// 1 - arg^2 < TAU_FP64_FALLBACK (or arg not finite), i.e. two roots nearly
// coalesce and the edge must be redone in float64 (dm, dp are then the
// float32 values, not to be used).
template <int LAW>
__device__ __forceinline__ bool edge_fluct_f32x2_core(const LawT<float>& L, const float2 wl[3],
                                                      const float2 wr[3], float dm[3], float dp[3]) {
  const float dh = ff_diff(wr[0], wl[0]);
  const float dq = ff_diff(wr[1], wl[1]);
  const float dz = ff_diff(wr[2], wl[2]);
  const float h0 = wl[0].x, q0 = wl[1].x;
  const float2 s = make_float2((float)GL3_S0, (float)GL3_S2);
  const float2 h = fma2(s, p2(dh), p2(h0));
  const float2 q = fma2(s, p2(dq), p2(q0));
  Eig2 e;
  node_eig_x2<LAW>(L, h, q, e);
  float2 y[3], x[3];
  A_times_x2(e, dh, dq, dz, y);
  abs_A_times_proj_x2(e, dh, dq, dz, y, x);
  Eig<float> em;
  node_eig<float, LAW>(L, h0 + 0.5f * dh, q0 + 0.5f * dq, em);
  float ym[3], xm[3];
  A_times(em, dh, dq, dz, ym[0], ym[1], ym[2]);
  abs_A_times_proj(em, dh, dq, dz, ym, xm);
  const bool redo = !(fmaf(-e.arg.x, e.arg.x, 1.0f) >= TAU_FP64_FALLBACK) ||
                    !(fmaf(-e.arg.y, e.arg.y, 1.0f) >= TAU_FP64_FALLBACK) ||
                    !(fmaf(-em.arg, em.arg, 1.0f) >= TAU_FP64_FALLBACK);
  const float w0 = (float)GL3_W0, w1 = (float)GL3_W1;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float ya = fmaf(w0, y[r].x + y[r].y, w1 * ym[r]);
    const float xa = fmaf(w0, x[r].x + x[r].y, w1 * xm[r]);
    dm[r] = 0.5f * (ya - xa);
    dp[r] = 0.5f * (ya + xa);
  }
  return redo;
}

// The same with the float64 redo of a flagged edge done in place
// (edge_fluct_f64_redo).
template <int LAW>
__device__ __forceinline__ void edge_fluct_f32x2(const LawT<float>& L, const LawT<double>& Ld,
                                                 const float2 wl[3], const float2 wr[3], float dm[3],
                                                 float dp[3], unsigned& flags) {
  if (edge_fluct_f32x2_core<LAW>(L, wl, wr, dm, dp)) {
    const EdgeD d = edge_fluct_f64_redo<LAW>(Ld, wl[0], wl[1], wl[2], wr[0], wr[1], wr[2]);
    flags |= d.flags;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      dm[r] = d.dm[r];
      dp[r] = d.dp[r];
    }
  }
}

}  // namespace adot
