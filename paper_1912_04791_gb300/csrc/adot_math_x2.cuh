// Float32 edge fluctuations with paired instructions: the two outer
// Gauss-Legendre nodes s0 and s2 of Eq. DOTjumpN (equal weights) are evaluated
// together, one per half of a float2, through the paired float32 add, multiply
// and fused multiply-add of this architecture (__fadd2_rn, __fmul2_rn,
// __ffma2_rn: one issue slot for two lanes of work). The reciprocal, square
// root, arccos and sincos steps and the choice of the root taken from the
// product of the roots stay per lane. The midpoint node takes the scalar path.
// The arithmetic is that of node_f32 (Eq. charPol/lambda, Eq. RR, RR-1,
// Eq. asbA through one spectral projector), with the same identities and the
// same float64 redo of a node whose roots nearly coalesce.
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
  int ks0, ks1;
};

// The root of smallest magnitude of one lane from l1 l2 l3 = c^2 a (as in node_eig).
__device__ __forceinline__ int vieta_lane(float& l1, float& l2, float& l3, float ca) {
  const float m1 = fabsf(l1), m2 = fabsf(l2), m3 = fabsf(l3);
  if (m1 <= m2 && m1 <= m3) {
    const float pr = l2 * l3;
    if (pr != 0.0f) l1 = ca / pr;
    return 1;
  }
  if (m2 <= m3) {
    const float pr = l1 * l3;
    if (pr != 0.0f) l2 = ca / pr;
    return 2;
  }
  const float pr = l1 * l2;
  if (pr != 0.0f) l3 = ca / pr;
  return 3;
}

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
  __sincosf(acosf(ax) * (float)(1.0 / 3.0), &S.x, &C.x);
  __sincosf(acosf(ay) * (float)(1.0 / 3.0), &S.y, &C.y);
  const float2 k1rk = mul2(k1, rk);                               // sqrt(k1)
  const float2 m = mul2(p2((float)(2.0 / 3.0)), k1rk);            // (2/3) sqrt(k1)
  const float2 nm = mul2(p2((float)(-2.0 / 3.0)), k1rk);
  const float2 F = mul2(p2((float)(2.0 / 3.0)), Fr);
  const float2 hc = mul2(p2(0.5f), C);
  const float2 hs = mul2(p2(0.86602540378443864676f), S);  // (sqrt 3 / 2) S
  float2 l1 = mul2(c, fma2(nm, add2(hc, hs), F));  // cos(phi/3 - pi/3) = C/2 + (sqrt3/2) S
  float2 l2 = mul2(c, fma2(nm, sub2(hc, hs), F));  // cos(phi/3 + pi/3) = C/2 - (sqrt3/2) S
  float2 l3 = mul2(c, fma2(m, C, F));
  const float2 nca = mul2(c2, na);  // -c^2 a
  e.ks0 = vieta_lane(l1.x, l2.x, l3.x, -nca.x);
  e.ks1 = vieta_lane(l1.y, l2.y, l3.y, -nca.y);
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

// |A| dW for two states through one projector each, as abs_A_times_proj: the
// projector's root (l1 or l3) and the sign are chosen per lane.
__device__ __forceinline__ void abs_A_times_proj_x2(const Eig2& e, float dh, float dq, float dz,
                                                    const float2 y[3], float2 x[3]) {
  const bool lox = e.l2.x >= 0.0f, loy = e.l2.y >= 0.0f;
  const float2 lk = make_float2(lox ? e.l1.x : e.l3.x, loy ? e.l1.y : e.l3.y);
  const float2 lf = make_float2(lox ? e.l3.x : e.l1.x, loy ? e.l3.y : e.l1.y);
  const float2 m2 = make_float2(lox ? -2.0f * fminf(e.l1.x, 0.0f) : -2.0f * fmaxf(e.l3.x, 0.0f),
                                loy ? -2.0f * fminf(e.l1.y, 0.0f) : -2.0f * fmaxf(e.l3.y, 0.0f));
  const float2 sg = make_float2(lox ? 1.0f : -1.0f, loy ? 1.0f : -1.0f);
  const float2 dk = mul2(sub2(lk, e.l2), sub2(lk, lf));
  // (l_k . dW) d_k = (l_k (l_k - 2u) - c^2 b) dh + l_k dq + c^2 dz
  const float2 ntu = mul2(e.u, p2(-2.0f));
  const float2 czb = mul2(e.c2, fma2(e.b, p2(-dh), p2(dz)));
  const float2 pk = fma2(mul2(lk, add2(lk, ntu)), p2(dh), fma2(lk, p2(dq), czb));
  // third entry of r_k: b + a / l_k = b - na / l_k, or directly for the root of smallest magnitude
  float2 rk = fma2(e.na, nrcp2(lk), e.b);
  if (e.ks0 == (lox ? 1 : 3)) {
    const float v = e.u.x - lk.x;
    rk.x = v * v * e.inv_c2.x - 1.0f;
  }
  if (e.ks1 == (loy ? 1 : 3)) {
    const float v = e.u.y - lk.y;
    rk.y = v * v * e.inv_c2.y - 1.0f;
  }
  const float2 coef = mul2(m2, mul2(pk, rcp2(dk)));
  x[0] = mul2(sg, add2(y[0], coef));
  x[1] = mul2(sg, fma2(coef, lk, y[1]));
  x[2] = mul2(sg, fma2(coef, rk, y[2]));
}

// D-/+ of one float32 edge (float-float states wl, wr): nodes s0 and s2 paired,
// the midpoint node scalar, each node redone in float64 when 1 - arg^2 <
// TAU_FP64_FALLBACK (or arg is not finite).
template <int LAW>
__device__ __forceinline__ void edge_fluct_f32x2(const LawT<float>& L, const LawT<double>& Ld,
                                                 const float2 wl[3], const float2 wr[3], float dm[3],
                                                 float dp[3], unsigned& flags) {
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
  const float2 delta = make_float2(fmaf(-e.arg.x, e.arg.x, 1.0f), fmaf(-e.arg.y, e.arg.y, 1.0f));
  if (!(delta.x >= TAU_FP64_FALLBACK)) {
    float yy[3], xx[3];
    node_f64_fallback<LAW>(Ld, h.x, q.x, dh, dq, dz, yy, xx, &flags);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      y[r].x = yy[r];
      x[r].x = xx[r];
    }
  }
  if (!(delta.y >= TAU_FP64_FALLBACK)) {
    float yy[3], xx[3];
    node_f64_fallback<LAW>(Ld, h.y, q.y, dh, dq, dz, yy, xx, &flags);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      y[r].y = yy[r];
      x[r].y = xx[r];
    }
  }
  float ym[3], xm[3];
  node_f32<LAW>(L, Ld, h0 + 0.5f * dh, q0 + 0.5f * dq, dh, dq, dz, ym, xm, flags);
  const float w0 = (float)GL3_W0, w1 = (float)GL3_W1;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float ya = fmaf(w0, y[r].x + y[r].y, w1 * ym[r]);
    const float xa = fmaf(w0, x[r].x + x[r].y, w1 * xm[r]);
    dm[r] = 0.5f * (ya - xa);
    dp[r] = 0.5f * (ya + xa);
  }
}

}  // namespace adot
