// Device math of the A-DOT scheme (arXiv 1912.04791), templated on the working
// precision (float or double).
//
// One quadrature node of Eq. DOTjumpN needs, at the node state (h, q):
//   step 1  the sediment-flux derivatives a = xi dq_s/dh, b = xi dq_s/dq
//           (Eq. Grass / Eq. MPM with Eq. Shields);
//   step 2  k1, k2 and phi (Eq. parameters, Eq. parameters_bis);
//   step 3  the trigonometric roots of the characteristic polynomial
//           (Eq. charPol, Eq. lambda);
//   steps 4-5  |A| dW = R |Lambda| R^-1 dW (Eq. asbA, Eq. RR, Eq. RR-1).
// Steps 4-5 are evaluated matrix-free through one spectral projector (see
// abs_A_times_proj), which is the same product as the paper's three-matrix
// form applied to dW. The three cosines cos(phi/3 -+ pi/3), cos(phi/3) of
// Eq. lambda come from one sincos through cos(x -+ pi/3) = C/2 +- (sqrt3/2) S.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace adot {

// Transport laws. LAW_POWER (q_s = A sign(u) max(|u| - u_cr, 0)^beta) runs the
// LAW_GRASS_THR code with its own exponent (LawT::beta; 3 for Eq. GrassThr).
enum : int { LAW_GRASS = 0, LAW_MPM = 1, LAW_GRASS_THR = 2, LAW_POWER = 3 };

// Status bits recorded in the device control block.
enum : unsigned {
  ST_DEPTH = 1u,        // h <= 0
  ST_NONFINITE = 2u,    // NaN / Inf
  ST_NONHYPERBOLIC = 4u,
  ST_TIMEOUT = 8u
};

// Closure parameters in the working precision, with the porosity factor xi
// folded in where it multiplies.
template <typename T>
struct LawT {
  T g;
  T K3;         // Grass: 3 xi A_g, so b = K3 u^2 / h and a = -b u; power law: beta xi A
  T mpm_c;      // MPM: n^2 / ((s - 1) d50), theta = mpm_c u^2 h^(-1/3)
  T mpm_scale;  // MPM: xi sqrt(g (s - 1) d50^3)
  T ucr;        // Grass with threshold / power law: incipient transport velocity u_cr
  T beta;       // Grass with threshold / power law: exponent (3 for Eq. GrassThr)
  T xa;         // xi A_g (Grass, threshold and power laws): xi q_s = xa sign(u) v^beta
};

// Gap below which |A| dW switches to the Newton divided-difference form
// (relative to c), and the zero band of a coalesced pair's slope; the same
// reading the oracle uses for the coalescence case.
constexpr double TAU_GAP = 1e-6;
// Tolerance on |arg| - 1 before a node is declared non-hyperbolic.
constexpr double TAU_HYP = 1e-6;
// In float32 a node whose 1 - arg^2 is below this is redone in float64
// (two roots within ~0.7 sqrt(1e-4) c of each other).
constexpr float TAU_FP64_FALLBACK = 1e-4f;

// Gauss-Legendre 3-point rule on [0, 1] (Eq. DOTjumpN with G = 3).
constexpr double GL3_S0 = 0.1127016653792583115;  // 1/2 - sqrt(15)/10
constexpr double GL3_S2 = 0.8872983346207416885;  // 1/2 + sqrt(15)/10
constexpr double GL3_W0 = 5.0 / 18.0;
constexpr double GL3_W1 = 8.0 / 18.0;

__device__ __forceinline__ float d_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double d_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float d_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double d_rsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float d_acos(float x) { return acosf(x); }
__device__ __forceinline__ double d_acos(double x) { return acos(x); }

// phi / 3 = arccos(x) / 3 in float32 for x in [-1, 1], from
// arccos(x) = sqrt(1 - x) P(x) on [0, 1] and pi - arccos(-x) below 0 (the form
// of Abramowitz & Stegun 4.4.46), P of degree 7 with coefficients fitted for
// this library by reweighted least squares on 4000 Chebyshev points in float64
// (|arccos - sqrt(1 - x) P| < 1.3e-8 on [0, 1]) and divided by 3 here. Evaluated
// in float32 the arccos is within 3.5e-7 of the exact value over [-1, 1].
// Building with -DADOT_ACOS_LIBRARY takes acosf instead.
__host__ __device__ constexpr float acos3_coef(int i) {
  return i == 0 ? 0.5235987901687622f
       : i == 1 ? -0.07153329998254776f
       : i == 2 ? 0.029666420072317123f
       : i == 3 ? -0.016770916059613228f
       : i == 4 ? 0.010445117019116879f
       : i == 5 ? -0.005936262663453817f
       : i == 6 ? 0.0024150970857590437f
                : -0.0004804770287591964f;
}
constexpr float kPi3 = 1.0471975803375244f;  // pi / 3 in float32
__device__ __forceinline__ float acos_third(float x) {
#ifdef ADOT_ACOS_LIBRARY
  return acosf(x) * (float)(1.0 / 3.0);
#else
  const float ax = fabsf(x);
  float p = acos3_coef(7);
#pragma unroll
  for (int i = 6; i >= 0; --i) p = fmaf(p, ax, acos3_coef(i));
  const float r = sqrtf(1.0f - ax) * p;
  return x >= 0.0f ? r : kPi3 - r;
#endif
}
__device__ __forceinline__ double acos_third(double x) { return acos(x) * (1.0 / 3.0); }
// float32: the hardware sine/cosine; the argument is phi/3 in [0, pi/3], where
// their absolute error is below 2^-21.4.
__device__ __forceinline__ void d_sincos(float x, float* s, float* c) { __sincosf(x, s, c); }
__device__ __forceinline__ void d_sincos(double x, double* s, double* c) { sincos(x, s, c); }
__device__ __forceinline__ float d_rcbrt(float x) { return rcbrtf(x); }
__device__ __forceinline__ double d_rcbrt(double x) { return rcbrt(x); }
__device__ __forceinline__ float d_pow(float x, float y) { return powf(x, y); }
__device__ __forceinline__ double d_pow(double x, double y) { return pow(x, y); }
__device__ __forceinline__ float d_abs(float x) { return fabsf(x); }
__device__ __forceinline__ double d_abs(double x) { return fabs(x); }
__device__ __forceinline__ float d_min(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double d_min(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float d_max(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double d_max(double a, double b) { return fmax(a, b); }

// Step 1: a = xi dq_s/dh, b = xi dq_s/dq at (h, q), given 1/h and u = q/h.
// Grass (Eq. Grass, five-step procedure step 1): dq_s/dq = 3 A_g u^2/h and
// dq_s/dh = -3 A_g u^3/h, i.e. b = K3 u^2/h, a = -b u.
// MPM (Eq. MPM, Eq. Shields, Manning s_f = n^2 u^2 h^(-4/3)):
// theta = mpm_c u^2 h^(-1/3); q_s = sign(u) 8 (theta - 0.047)^1.5 scale;
// dtheta/dq = 2 mpm_c u h^(-4/3), dtheta/dh = -(7/3) theta / h.
template <typename T, int LAW>
__device__ __forceinline__ void sediment_derivs(const LawT<T>& L, T h, T q, T inv_h, T u, T& a,
                                                T& b) {
  if constexpr (LAW == LAW_GRASS) {
    (void)h;
    (void)q;
    b = L.K3 * u * u * inv_h;
    a = -b * u;
  } else if constexpr (LAW == LAW_GRASS_THR) {
    // Eq. GrassThr read as q_s = A_g sign(u) v^3, v = |u| - u_cr > 0, else 0:
    // b = K3 v^2 / h, a = -b u (d|u|/dq = sign(u)/h, d|u|/dh = -sign(u) u/h)
    (void)h;
    (void)q;
    // Power law (Eq. Soni_qs): the same with v^(beta-1) in place of v^2.
    const T v = d_abs(u) - L.ucr;
    if (v > T(0)) {
      const T vb1 = (L.beta == T(3)) ? v * v : d_pow(v, L.beta - T(1));
      b = L.K3 * vb1 * inv_h;
      a = -b * u;
    } else {
      a = T(0);
      b = T(0);
    }
  } else {
    T r3 = d_rcbrt(h);
    T theta = L.mpm_c * u * u * r3;
    T ex = theta - T(0.047);
    if (ex > T(0)) {
      T s = L.mpm_scale * T(12) * d_sqrt(ex);  // scale * dPhi/dtheta
      b = s * T(2) * L.mpm_c * d_abs(u) * r3 * inv_h;
      T sg = (q > T(0)) ? T(1) : ((q < T(0)) ? T(-1) : T(0));
      a = -s * sg * (T(7) / T(3)) * theta * inv_h;
    } else {
      a = T(0);
      b = T(0);
    }
  }
}

// xi q_s at (h, q): the bed discharge of a state, which a feeding end compares
// with the imposed one (Sec. 5.1).
template <typename T, int LAW>
__device__ __forceinline__ T sediment_xqs(const LawT<T>& L, T h, T q) {
  const T u = q / h;
  if constexpr (LAW == LAW_GRASS) {
    return L.xa * u * u * u;
  } else if constexpr (LAW == LAW_GRASS_THR) {
    const T v = d_abs(u) - L.ucr;
    if (!(v > T(0))) return T(0);
    const T vb = (L.beta == T(3)) ? v * v * v : d_pow(v, L.beta);
    return (u > T(0)) ? L.xa * vb : -(L.xa * vb);
  } else {
    const T theta = L.mpm_c * u * u * d_rcbrt(h);
    const T ex = theta - T(0.047);
    if (!(ex > T(0))) return T(0);
    const T qs = L.mpm_scale * T(8) * ex * d_sqrt(ex);
    return (q > T(0)) ? qs : ((q < T(0)) ? -qs : T(0));
  }
}

// Eigen-data of A at one state.
template <typename T>
struct Eig {
  T u, c, c2, inv_c2, a, b;
  T l1, l2, l3;  // l1 <= l2 <= l3
  T arg;         // k2 / sqrt(4 k1^3) before clamping
};

__device__ __forceinline__ float d_fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double d_fdiv(double a, double b) { return a / b; }

// Steps 1-3: derivatives, k1, k2, phi, and the three roots of Eq. lambda. A
// root of small magnitude comes out of Eq. lambda as a difference of two O(c)
// terms. In float64 the root of smallest magnitude is recomputed from the
// product of the roots, l1 l2 l3 = c^2 a (the constant term of Eq. charPol
// times c^3), unless the other two roots' product is zero (a double root at
// 0): a fixed bed (a = 0) then has its zero root exactly, so the projector's
// choice in abs_A_times_proj does not follow the sign of rounding noise. In
// float32 only the projector's own root is recomputed, where |A| dW needs it
// (abs_A_times_proj), which saves a division and a selection per node.
template <typename T, int LAW>
__device__ __forceinline__ void node_eig(const LawT<T>& L, T h, T q, Eig<T>& e) {
  const T inv_h = T(1) / h;
  const T u = q * inv_h;
  const T c2 = L.g * h;
  const T rc = d_rsqrt(c2);  // 1/c
  const T c = c2 * rc;
  const T Fr = u * rc;
  T a, b;
  sediment_derivs<T, LAW>(L, h, q, inv_h, u, a, b);
  const T k1 = T(3) + Fr * Fr + T(3) * b;
  const T k2 = Fr * (T(18) * (T(1) + b) - T(2) * Fr * Fr) + T(27) * a * rc;
  const T rk = d_rsqrt(k1);
  const T arg = T(0.5) * k2 * (rk * rk * rk);
  const T argc = d_min(d_max(arg, T(-1)), T(1));
  const T phi3 = acos_third(argc);
  T S, C;
  d_sincos(phi3, &S, &C);
  const T m = T(2.0 / 3.0) * (k1 * rk);  // (2/3) sqrt(k1)
  const T F = T(2.0 / 3.0) * Fr;
  const T hc = T(0.5) * C;
  const T hs = T(0.86602540378443864676) * S;  // (sqrt 3 / 2) S
  e.u = u;
  e.c = c;
  e.c2 = c2;
  e.inv_c2 = rc * rc;
  e.a = a;
  e.b = b;
  T l1 = c * (F - m * (hc + hs));  // cos(phi/3 - pi/3) = C/2 + (sqrt3/2) S
  T l2 = c * (F - m * (hc - hs));  // cos(phi/3 + pi/3) = C/2 - (sqrt3/2) S
  T l3 = c * (F + m * C);
  if constexpr (std::is_same<T, double>::value) {
    const T m1 = d_abs(l1), m2 = d_abs(l2), m3 = d_abs(l3);
    const T ca = c2 * a;
    if (m1 <= m2 && m1 <= m3) {
      const T pr = l2 * l3;
      if (pr != T(0)) l1 = ca / pr;
    } else if (m2 <= m3) {
      const T pr = l1 * l3;
      if (pr != T(0)) l2 = ca / pr;
    } else {
      const T pr = l1 * l2;
      if (pr != T(0)) l3 = ca / pr;
    }
  }
  e.l1 = l1;
  e.l2 = l2;
  e.l3 = l3;
  e.arg = arg;
}

// A(W) v with A from Eq. W&A_definition.
template <typename T>
__device__ __forceinline__ void A_times(const Eig<T>& e, T v0, T v1, T v2, T& y0, T& y1, T& y2) {
  y0 = v1;
  y1 = (e.c2 - e.u * e.u) * v0 + T(2) * e.u * v1 + e.c2 * v2;
  y2 = e.a * v0 + e.b * v1;
}

// Steps 4-5 applied to dW through one spectral projector. With the projectors
// P_i = r_i (l_i . ) / d_i of Eq. RR and RR-1 (r_i = [1, l_i, (u - l_i)^2/c^2 - 1],
// l_i = [c^2 - u^2 + l_j l_k, 2u - l_j - l_k, c^2], d_i = (l_i - l_j)(l_i - l_k)),
// A = sum_i l_i P_i and sum_i P_i = I, so Eq. asbA's |A| = sum_i |l_i| P_i equals
// A - 2 sum_{l_i < 0} l_i P_i and -A + 2 sum_{l_i > 0} l_i P_i. Of three ordered roots
// at most one lies on the minority side of zero: |A| dW = s (A dW - 2 m P_k dW)
// with k = 1, s = 1, m = min(l1, 0) when l2 >= 0, else k = 3, s = -1, m = max(l3, 0).
// The entries are evaluated through identities of the roots of Eq. charPol,
// l^3 - 2u l^2 - (c^2 - u^2 + c^2 b) l - c^2 a = 0, which avoid cancelling O(c)
// terms: c^2 - u^2 + l_j l_k = l_k (l_k - 2u) - c^2 b (pair products), 2u - l_j - l_k =
// l_k (sum of roots), and (u - l_k)^2/c^2 - 1 = b + a / l_k.
// The root of smallest magnitude is l_k or l2 (|l_f| >= |l2| for the far root
// l_f). When it is l_k (near critical flow), l_k is taken from the product of
// the roots, l1 l2 l3 = c^2 a, so that it keeps its relative precision (in
// float64 node_eig has done so already), and the third entry of r_k from its
// definition (b + a / l_k would divide by it); the product is skipped when
// l2 l_f = 0 (a double root at 0). When it is l2, its absolute error of a few
// ulp of c (float32) enters only d_k through l_k - l2 and the choice of k, and
// either choice gives the same |A| up to |l2| |P2 dW|.
// The other case takes one reciprocal for both quotients: m p_k / d_k and
// m p_k (b l_k + a) / (d_k l_k). y = A dW.
template <typename T>
__device__ __forceinline__ void abs_A_times_proj(const Eig<T>& e, T dh, T dq, T dz, const T y[3],
                                                 T x[3]) {
  const bool lo = e.l2 >= T(0);
  T lk = lo ? e.l1 : e.l3;
  const T lf = lo ? e.l3 : e.l1;  // the root on the far side
  const bool small = d_abs(lk) <= d_abs(e.l2);
  if (small) {
    const T pr = e.l2 * lf;
    if (pr != T(0)) lk = e.c2 * e.a / pr;
  }
  const T m2 = T(-2) * (lo ? d_min(lk, T(0)) : d_max(lk, T(0)));
  const T dk = (lk - e.l2) * (lk - lf);
  const T pk = (lk * (lk - T(2) * e.u) - e.c2 * e.b) * dh + lk * dq + e.c2 * dz;  // (l_k . dW) d_k
  const T mp = m2 * pk;
  T coef, c2nd;
  if (small) {
    coef = d_fdiv(mp, dk);
    const T v = e.u - lk;
    c2nd = coef * (v * v * e.inv_c2 - T(1));
  } else {
    const T inv = d_fdiv(T(1), dk * lk);
    coef = mp * lk * inv;
    c2nd = mp * (e.b * lk + e.a) * inv;
  }
  if (lo) {
    x[0] = y[0] + coef;
    x[1] = y[1] + coef * lk;
    x[2] = y[2] + c2nd;
  } else {
    x[0] = -(y[0] + coef);
    x[1] = -(y[1] + coef * lk);
    x[2] = -(y[2] + c2nd);
  }
}

// First divided difference of |x| with the coalescence reading: a pair closer
// than tau is one double root m = (a+b)/2 with slope sign(m), 0 if |m| < tau.
template <typename T>
__device__ __forceinline__ T dd1_abs(T a, T b, T tau) {
  if (d_abs(a - b) < tau) {
    T m = T(0.5) * (a + b);
    if (d_abs(m) < tau) return T(0);
    return m > T(0) ? T(1) : T(-1);
  }
  if (a >= T(0) && b >= T(0)) return T(1);
  if (a <= T(0) && b <= T(0)) return T(-1);
  return (d_abs(a) - d_abs(b)) / (a - b);
}

// |A| dW by Newton interpolation of |x| on the spectrum:
// |A| = f[l1] I + f[l1,l2](A - l1 I) + f[l1,l2,l3](A - l1 I)(A - l2 I).
template <typename T>
__device__ __forceinline__ void abs_A_times_newton(const Eig<T>& e, T dh, T dq, T dz, T& x0, T& x1,
                                                   T& x2) {
  const T tau = T(TAU_GAP) * e.c;
  const T f0 = d_abs(e.l1);
  const T f01 = dd1_abs(e.l1, e.l2, tau);
  const T f12 = dd1_abs(e.l2, e.l3, tau);
  const T span = e.l3 - e.l1;
  const T f012 = (span < tau) ? T(0) : (f12 - f01) / span;
  T y0, y1, y2;
  A_times(e, dh, dq, dz, y0, y1, y2);
  // v = (A - l2 I) dW; w = (A - l1 I) v
  const T v0 = y0 - e.l2 * dh, v1 = y1 - e.l2 * dq, v2 = y2 - e.l2 * dz;
  T w0, w1, w2;
  A_times(e, v0, v1, v2, w0, w1, w2);
  w0 -= e.l1 * v0;
  w1 -= e.l1 * v1;
  w2 -= e.l1 * v2;
  x0 = f0 * dh + f01 * (y0 - e.l1 * dh) + f012 * w0;
  x1 = f0 * dq + f01 * (y1 - e.l1 * dq) + f012 * w1;
  x2 = f0 * dz + f01 * (y2 - e.l1 * dz) + f012 * w2;
}

// Full float64 node: A dW and |A| dW, with the Newton form when two roots are
// closer than TAU_GAP * c. Sets ST_NONHYPERBOLIC when |arg| > 1 + TAU_HYP.
template <int LAW>
__device__ __forceinline__ void node_f64(const LawT<double>& L, double h, double q, double dh,
                                         double dq, double dz, double y[3], double x[3],
                                         unsigned& flags) {
  Eig<double> e;
  node_eig<double, LAW>(L, h, q, e);
  if (!(d_abs(e.arg) <= 1.0 + TAU_HYP)) flags |= ST_NONHYPERBOLIC;
  A_times(e, dh, dq, dz, y[0], y[1], y[2]);
  const double gap = d_min(e.l2 - e.l1, e.l3 - e.l2);
  if (gap < TAU_GAP * e.c)
    abs_A_times_newton(e, dh, dq, dz, x[0], x[1], x[2]);
  else
    abs_A_times_proj(e, dh, dq, dz, y, x);
}

// Spectral radius max(|l1|, |l3|) at a state (float64: from Eq. lambda; the
// extreme roots need no small-root correction).
template <typename T, int LAW>
__device__ __forceinline__ T spectral_radius(const LawT<T>& L, T h, T q) {
  Eig<T> e;
  node_eig<T, LAW>(L, h, q, e);
  return d_max(d_abs(e.l1), d_abs(e.l3));
}

// float32 spectral radius from Eq. lambda, kept out of line: the fallback of
// spectral_radius_f32.
template <int LAW>
__device__ __noinline__ float spectral_radius_f32_trig(const LawT<float>& L, float h, float q) {
  return spectral_radius<float, LAW>(L, h, q);
}

// float32 spectral radius. The root of largest magnitude is l3 when u >= 0 and
// l1 when u < 0 (the water waves u +- c carry the extreme speeds); by the
// mirror symmetry x -> -x (u -> -u, a -> -a, l -> -l) both cases reduce to the
// largest root of p(l) = l^3 - 2u l^2 - (c^2 - u^2 + c^2 b) l - c^2 a with
// u >= 0. p'' = 6l - 4u > 0 on [u + c, inf), so when p(u + c) <= 0 and
// p'(u + c) > 0 Newton's method from u + c (the root when a = b = 0) converges
// monotonically after its first step to the only root in [u + c, inf), the
// largest. At most four steps are taken (fewer once a correction falls below
// 1e-7 of the root); if the start does not meet those conditions
// (strong transport, b > ~2) or the last correction is not below 1e-5 of the
// root, the roots of Eq. lambda are used instead.
// SKIP: the caller wants only radii above floor (a running maximum). After the
// first step every Newton iterate lies above the root, so once it is below
// floor (1 - 1e-6) the radius cannot raise the maximum and 0 is returned (the
// margin covers the iterates' rounding, so the maximum is unchanged; 0.5 % on
// the 1e7-cell step).
template <int LAW, bool SKIP = false>
__device__ __forceinline__ float spectral_radius_f32(const LawT<float>& L, float h, float q,
                                                     float floor = 0.0f) {
  const float inv_h = __fdividef(1.0f, h);
  const float u = q * inv_h;
  const float c2 = L.g * h;
  const float c = c2 * rsqrtf(c2);
  float a, b;
  sediment_derivs<float, LAW>(L, h, q, inv_h, u, a, b);
  const float sg = (u >= 0.0f) ? 1.0f : -1.0f;
  const float us = sg * u;
  const float K = c2 - u * u + c2 * b;
  const float ca = c2 * (sg * a);
  const float tu = 2.0f * us, fu = 4.0f * us;
  float l = us + c;
  float pv = ((l - tu) * l - K) * l - ca;
  float dp = (3.0f * l - fu) * l - K;
  bool ok = (pv <= 1e-5f * c2 * c) && (dp > 0.0f);
  float d = 0.0f;
#pragma unroll
  for (int it = 0; it < 4; ++it) {
    d = __fdividef(pv, dp);
    l -= d;
    if constexpr (SKIP)
      if (it == 0 && ok && l <= floor * 0.999999f) return 0.0f;
    // quadratic convergence: once a correction is below 1e-7 of the root the
    // next one is below float rounding, so the iteration stops
    if (fabsf(d) <= 1e-7f * l) break;
    pv = ((l - tu) * l - K) * l - ca;
    dp = (3.0f * l - fu) * l - K;
  }
  ok = ok && (fabsf(d) <= 1e-5f * l);
  if (!ok) return spectral_radius_f32_trig<LAW>(L, h, q);
  return l;
}

// Full |A| (row-major 3x3) at a state in float64, column by column through the
// same evaluation as |A| dW (eigenvectors, or the Newton form near coalescence).
template <int LAW>
__device__ __forceinline__ void abs_A_matrix_f64(const LawT<double>& L, double h, double q,
                                                 double X[9], unsigned& flags) {
  Eig<double> e;
  node_eig<double, LAW>(L, h, q, e);
  if (!(d_abs(e.arg) <= 1.0 + TAU_HYP)) flags |= ST_NONHYPERBOLIC;
  const bool newton = d_min(e.l2 - e.l1, e.l3 - e.l2) < TAU_GAP * e.c;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const double v0 = (j == 0) ? 1.0 : 0.0, v1 = (j == 1) ? 1.0 : 0.0, v2 = (j == 2) ? 1.0 : 0.0;
    double x[3];
    if (newton) {
      abs_A_times_newton(e, v0, v1, v2, x[0], x[1], x[2]);
    } else {
      double y[3];
      A_times(e, v0, v1, v2, y[0], y[1], y[2]);
      abs_A_times_proj(e, v0, v1, v2, y, x);
    }
    X[0 * 3 + j] = x[0];
    X[1 * 3 + j] = x[1];
    X[2 * 3 + j] = x[2];
  }
}

// splitmix64 (Steele, Lea & Flood 2014): counter-based 64-bit mixer.
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// ---------------------------------------------------------------------------
// float-float helpers (value = hi + lo, |lo| <= ulp(hi)/2)
// ---------------------------------------------------------------------------

// (hi, lo) + b with Knuth's TwoSum on hi + b, the low parts folded in, and a
// Fast2Sum renormalisation. Uses only float32 adds (no contraction possible).
__device__ __forceinline__ float2 ff_add(float2 a, float b) {
  const float s = a.x + b;
  const float bb = s - a.x;
  const float err = (a.x - (s - bb)) + (b - bb);
  const float lo = a.y + err;
  const float hi = s + lo;
  return make_float2(hi, lo - (hi - s));
}

// (a - b) of two float-float values rounded to one float.
__device__ __forceinline__ float ff_diff(float2 a, float2 b) { return (a.x - b.x) + (a.y - b.y); }

__device__ __forceinline__ float2 ff_from_double(double d) {
  const float hi = (float)d;
  return make_float2(hi, (float)(d - (double)hi));
}

__device__ __forceinline__ double ff_to_double(float2 a) { return (double)a.x + (double)a.y; }

}  // namespace adot
