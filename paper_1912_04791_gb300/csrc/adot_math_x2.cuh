// Float32 edge fluctuations with paired instructions: the two outer
// Gauss-Legendre nodes s0 and s2 of Eq. DOTjumpN (equal weights) are evaluated
// together, one per half of a float2, through the paired float32 add, multiply
// and fused multiply-add of this architecture (__fadd2_rn, __fmul2_rn,
// __ffma2_rn: one issue slot for two lanes of work). The reciprocal, square
// root, arccos and sincos steps and the choice of the root taken from the
// product of the roots stay per lane. The midpoint node takes the scalar path.
// The arithmetic is that of node_f32 (Eq. charPol/lambda, Eq. RR, RR-1,
// Eq. asbA), with the same identities and the same float64 redo of a node
// whose roots nearly coalesce.
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

// (u - l)^2 / c^2 - 1 for the root of smallest magnitude of one lane.
__device__ __forceinline__ void direct_r_lane(int ks, float u, float inv_c2, float l1, float l2, float l3,
                                              float& r1, float& r2, float& r3) {
  if (ks == 1) {
    const float v = u - l1;
    r1 = v * v * inv_c2 - 1.0f;
  } else if (ks == 2) {
    const float v = u - l2;
    r2 = v * v * inv_c2 - 1.0f;
  } else {
    const float v = u - l3;
    r3 = v * v * inv_c2 - 1.0f;
  }
}

// |A| dW for two states, as abs_A_times_eigvec.
__device__ __forceinline__ void abs_A_times_eigvec_x2(const Eig2& e, float dh, float dq, float dz,
                                                      float2 x[3]) {
  const float2 l1 = e.l1, l2 = e.l2, l3 = e.l3;
  const float2 e12 = sub2(l1, l2), e31 = sub2(l3, l1), e23 = sub2(l2, l3);
  const float2 invP = nrcp2(mul2(mul2(e12, e31), e23));  // 1 / ((l1-l2)(l1-l3)(l2-l3))
  const float2 ntu = mul2(e.u, p2(-2.0f));
  // p_i = l_i . dW times (l_i - l_j)(l_i - l_k):
  // (l_i (l_i - 2u) - c^2 b) dh + l_i dq + c^2 dz
  const float2 czb = mul2(e.c2, fma2(e.b, p2(-dh), p2(dz)));
  const float2 p1 = fma2(mul2(l1, add2(l1, ntu)), p2(dh), fma2(l1, p2(dq), czb));
  const float2 p2_ = fma2(mul2(l2, add2(l2, ntu)), p2(dh), fma2(l2, p2(dq), czb));
  const float2 p3 = fma2(mul2(l3, add2(l3, ntu)), p2(dh), fma2(l3, p2(dq), czb));
  // 1/d1 = e23/P, 1/d2 = -e13/P = e31/P, 1/d3 = e12/P
  const float2 al1 = mul2(mul2(abs2(l1), p1), mul2(e23, invP));
  const float2 al2 = mul2(mul2(abs2(l2), p2_), mul2(e31, invP));
  const float2 al3 = mul2(mul2(abs2(l3), p3), mul2(e12, invP));
  // third entries of r_i: b + a / l_i = b - na / l_i; the root of smallest magnitude directly
  float2 r1 = fma2(e.na, nrcp2(l1), e.b);
  float2 r2 = fma2(e.na, nrcp2(l2), e.b);
  float2 r3 = fma2(e.na, nrcp2(l3), e.b);
  direct_r_lane(e.ks0, e.u.x, e.inv_c2.x, l1.x, l2.x, l3.x, r1.x, r2.x, r3.x);
  direct_r_lane(e.ks1, e.u.y, e.inv_c2.y, l1.y, l2.y, l3.y, r1.y, r2.y, r3.y);
  x[0] = add2(add2(al1, al2), al3);
  x[1] = fma2(al3, l3, fma2(al2, l2, mul2(al1, l1)));
  x[2] = fma2(al3, r3, fma2(al2, r2, mul2(al1, r1)));
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
  abs_A_times_eigvec_x2(e, dh, dq, dz, x);
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
