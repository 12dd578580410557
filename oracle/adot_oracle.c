/*
 * A-DOT oracle: a plain, slow, FP64 CPU implementation of the path-conservative
 * DOT scheme for the 1D de Saint Venant-Exner (dSVE) system, written from
 * Carraro, Valiani & Caleffi, "Efficient analytical implementation of the DOT
 * Riemann solver for the de Saint Venant-Exner morphodynamic model"
 * (arXiv 1912.04791).
 *
 * THIS IS TEST INFRASTRUCTURE. Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark call it. The CUDA library never links,
 * loads or calls it, and it shares no source with the CUDA library.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no FMA contraction,
 * so every product and sum rounds exactly as written).
 *
 * Contents (each function cites the passage it follows):
 *   sediment laws and their derivatives ............ Sec. 2, Eq. Grass, Eq. GrassThr,
 *                                                    Eq. MPM/Shields, Eq. Soni_qs
 *   flux matrix A(W) ............................... Sec. 2, Eq. W&A_definition
 *   analytical eigenstructure (A-DOT) .............. Sec. 3.3, Eq. charPol, lambda,
 *                                                    parameters, parameters_bis, RR, RR-1,
 *                                                    circPerm, five-step procedure
 *   numerical eigenstructure (original DOT) ........ Sec. 3.1/3.3: own shifted-QR
 *                                                    eigenvalues, null-vector eigenvectors,
 *                                                    pivoted Gauss-Jordan inverse
 *   |A| = R |Lambda| R^-1 .......................... Eq. asbA, Eq. ExAbsA
 *   Sylvester and Newton forms of |A| .............. standard matrix-function identities
 *                                                    (same matrix as Eq. asbA for distinct
 *                                                    eigenvalues; Newton form is the
 *                                                    coalescence reading)
 *   DOT fluctuations with G=3 Gauss-Legendre ....... Eq. path, Eq. DOTjumpN
 *   first-order update and time loop ............... Eq. scheme; S = 0 (frictionless,
 *                                                    Sec. 4 opening) or the Strickler
 *                                                    friction source of Sec. 2
 *   sediment feed through an end (Soni case) ....... Sec. 5.1 boundary data
 *   second-order MUSCL-Hancock variant ............. Sec. 6 (no restriction on the order);
 *                                                    Castro, Gallardo & Pares (2006), path-
 *                                                    conservative reconstruction of states
 *   PRICE-C jump function (comparison scheme) ...... Sec. 3.2, Eq. PRICEjump, AiPRICE, Apsi,
 *                                                    Im; A^Psi with the same 3-point rule
 *
 * Parity status: every function here is pinned by tests (library eigensolver,
 * closed forms, invariants, textbook special cases); none is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

enum {
  ORC_OK = 0,
  ORC_E_INVALID = 1,
  ORC_E_DEPTH = 2,
  ORC_E_NONFINITE = 3,
  ORC_E_NONHYPERBOLIC = 4,
  ORC_E_NOCONVERGE = 5
};

enum { ORC_LAW_GRASS = 0, ORC_LAW_MPM = 1, ORC_LAW_GRASS_THR = 2, ORC_LAW_POWER = 3 };

/* How |A| is evaluated at a quadrature node. */
enum {
  ORC_ABS_ANALYTIC = 0,  /* A-DOT: Eq. lambda + Eq. RR + Eq. RR-1, three-matrix product */
  ORC_ABS_NUMERIC = 1,   /* original DOT: numerical eigenstructure, then R|L|R^-1 */
  ORC_ABS_SYLVESTER = 2, /* sum_i |l_i| prod_{j!=i} (A - l_j I)/(l_i - l_j), analytic l_i */
  ORC_ABS_NEWTON = 3     /* Newton divided-difference interpolation of |.| on the spectrum */
};

enum {
  ORC_BC_TRANSMISSIVE = 0,
  ORC_BC_PERIODIC = 1,
  ORC_BC_INFLOW_Q = 2,  /* ghost q = v0, h and z copied from the adjacent cell */
  ORC_BC_OUTFLOW_H = 3, /* ghost h = v0, q and z copied */
  ORC_BC_INFLOW_QZ = 4, /* ghost q = v0, z = v1 - v2 * t, h copied (Test 2 inflow) */
  ORC_BC_INFLOW_QS = 5, /* ghost q = v0, h copied, z extrapolated linearly from the two
                           cells next to the end; the sediment discharge v1 (signed,
                           along +x) is imposed through the end edge */
  ORC_BC_OUTFLOW_HS = 6 /* ghost h = v0, q copied, z extrapolated linearly */
};

typedef struct {
  int kind;         /* ORC_LAW_* */
  double g;         /* gravitational acceleration */
  double xi;        /* 1/(1-p), p = bed porosity */
  double Ag;        /* Grass coefficient [s^2/m] */
  double s_rel;     /* MPM: relative grain density S_g */
  double d50;       /* MPM: median grain size [m] */
  double manning_n; /* MPM: Manning coefficient (= 1/K_s) */
  double u_cr;      /* Grass with threshold / power law: incipient velocity [m/s] */
  double beta;      /* power law: exponent (>= 1) */
} orc_law;

typedef struct {
  int64_t n;        /* number of cells */
  double x_min, x_max;
  double cfl;
  orc_law law;
  int abs_method;   /* ORC_ABS_* used for every node */
  int bc_left, bc_right;
  double bcl[3], bcr[3];
  double ks;        /* Strickler coefficient of the friction source [m^(1/3)/s]; 0 = none */
  int order;        /* 0 or 1: first-order scheme (Eq. scheme); 2: MUSCL-Hancock */
  int limiter;      /* order 2: 0 = minmod slopes, 1 = zero slopes (the first-order scheme
                       reached through the second-order code) */
  int scheme;       /* ORC_SCHEME_DOT (jump function of Eq. DOTjumpN) or ORC_SCHEME_PRICE_C
                       (Eq. PRICEjump) */
  double price_eps; /* PRICE-C: the small parameter epsilon of I_eps (Eq. Im) */
} orc_cfg;

enum { ORC_SCHEME_DOT = 0, ORC_SCHEME_PRICE_C = 1 };

/* Threshold on the eigenvalue gap, relative to c, below which |A| is taken
 * from the Newton divided-difference form instead of R|L|R^-1, whose R^-1
 * divides by the gaps (reading of the coalescence case, which the paper
 * declares impossible for a movable bed in Sec. 3.3). */
static const double ORC_TAU_GAP = 1e-6;
/* Tolerance on |k2 / sqrt(4 k1^3)| above 1 before a state is declared
 * non-hyperbolic (Sec. 3.3: the arccos argument must lie in [-1, 1]). */
static const double ORC_TAU_HYP = 1e-6;

/* ---------------------------------------------------------------------- */
/* Sediment discharge and its derivatives (Sec. 2).                         */
/* ---------------------------------------------------------------------- */

/* Grass law q_s = A_g u^3 (Eq. Grass). The five-step procedure (step 1) writes
 * dq_s/dh = -3 q_s/h and dq_s/dq = 3 q_s/q; with u = q/h these equal
 * -3 A_g u^3/h and 3 A_g u^2/h, which stay finite at q = 0.
 * MPM law (Eq. MPM, Eq. Shields) with the Strickler/Manning friction slope
 * s_f = n^2 u^2 / h^(4/3) (Sec. 2), theta = s_f h / ((S_g-1) d50), transport
 * directed along u. Derivatives by the chain rule through theta(h, q). */
int orc_sediment(const orc_law* L, double h, double q, double* qs, double* dqs_dh,
                 double* dqs_dq) {
  if (!(h > 0.0)) return ORC_E_DEPTH;
  double u = q / h;
  if (L->kind == ORC_LAW_GRASS) {
    *qs = L->Ag * u * u * u;
    *dqs_dh = -3.0 * L->Ag * u * u * u / h;
    *dqs_dq = 3.0 * L->Ag * u * u / h;
    return ORC_OK;
  }
  if (L->kind == ORC_LAW_GRASS_THR || L->kind == ORC_LAW_POWER) {
    /* Eq. GrassThr, q_s = A_g (u - u_cr)^3, read as transport along u that
     * starts at |u| = u_cr: q_s = A_g sign(u) v^3 with v = |u| - u_cr > 0, and
     * q_s = 0 for |u| <= u_cr. With d|u|/dq = sign(u)/h and d|u|/dh =
     * -sign(u) u/h: dq_s/dq = 3 A_g v^2/h, dq_s/dh = -3 A_g v^2 u/h.
     * Power law (Eq. Soni_qs, q_s = alpha u^beta, alpha in Ag, u_cr = 0 there):
     * the same with the exponent beta, dq_s/dq = beta A_g v^(beta-1)/h. */
    double v = fabs(u) - L->u_cr;
    if (v <= 0.0) {
      *qs = 0.0;
      *dqs_dh = 0.0;
      *dqs_dq = 0.0;
      return ORC_OK;
    }
    double sgn = (u > 0.0) ? 1.0 : -1.0;
    if (L->kind == ORC_LAW_GRASS_THR) {
      *qs = L->Ag * sgn * v * v * v;
      *dqs_dq = 3.0 * L->Ag * v * v / h;
      *dqs_dh = -3.0 * L->Ag * v * v * u / h;
      return ORC_OK;
    }
    if (!(L->beta >= 1.0)) return ORC_E_INVALID;
    double vb1 = pow(v, L->beta - 1.0);
    *qs = L->Ag * sgn * vb1 * v;
    *dqs_dq = L->beta * L->Ag * vb1 / h;
    *dqs_dh = -L->beta * L->Ag * vb1 * u / h;
    return ORC_OK;
  }
  if (L->kind == ORC_LAW_MPM) {
    double sm1 = L->s_rel - 1.0;
    double scale = sqrt(L->g * sm1 * L->d50 * L->d50 * L->d50);
    double n2 = L->manning_n * L->manning_n;
    /* theta = n^2 q^2 h^(-7/3) / ((S_g-1) d50) */
    double theta = n2 * q * q * pow(h, -7.0 / 3.0) / (sm1 * L->d50);
    double ex = theta - 0.047;
    if (ex <= 0.0) {
      *qs = 0.0;
      *dqs_dh = 0.0;
      *dqs_dq = 0.0;
      return ORC_OK;
    }
    double sgn = (q > 0.0) ? 1.0 : ((q < 0.0) ? -1.0 : 0.0);
    double Phi = 8.0 * ex * sqrt(ex);
    double dPhi = 12.0 * sqrt(ex); /* dPhi/dtheta */
    /* dtheta/dq = 2 n^2 q h^(-7/3) / ((S_g-1) d50); dtheta/dh = -(7/3) theta / h */
    double dth_dq = 2.0 * n2 * q * pow(h, -7.0 / 3.0) / (sm1 * L->d50);
    double dth_dh = -(7.0 / 3.0) * theta / h;
    *qs = sgn * Phi * scale;
    *dqs_dq = sgn * dPhi * dth_dq * scale;
    *dqs_dh = sgn * dPhi * dth_dh * scale;
    return ORC_OK;
  }
  return ORC_E_INVALID;
}

/* Flux matrix A(W) of the quasi-linear form (Eq. quasiLinNC, Eq. W&A_definition),
 * row-major. z does not enter A. */
int orc_flux_matrix(const orc_law* L, double h, double q, double A[9]) {
  double qs, dh, dq;
  int st = orc_sediment(L, h, q, &qs, &dh, &dq);
  if (st) return st;
  double u = q / h;
  double c2 = L->g * h;
  A[0] = 0.0;
  A[1] = 1.0;
  A[2] = 0.0;
  A[3] = c2 - u * u;
  A[4] = 2.0 * u;
  A[5] = c2;
  A[6] = L->xi * dh;
  A[7] = L->xi * dq;
  A[8] = 0.0;
  return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* Analytical eigenstructure (Sec. 3.3, A-DOT).                             */
/* ---------------------------------------------------------------------- */

/* Steps 1-3 of the five-step procedure: derivatives, then k1, k2, phi
 * (Eq. parameters, Eq. parameters_bis), then the trigonometric roots
 * (Eq. lambda). lam[0] <= lam[1] <= lam[2]. arg_out receives k2/sqrt(4 k1^3)
 * before clamping. */
int orc_eigvals_analytic(const orc_law* L, double h, double q, double lam[3],
                         double* arg_out) {
  double qs, dh, dq;
  int st = orc_sediment(L, h, q, &qs, &dh, &dq);
  if (st) return st;
  double u = q / h;
  double c = sqrt(L->g * h);
  double Fr = u / c;
  double xdh = L->xi * dh; /* xi dq_s/dh */
  double xdq = L->xi * dq; /* xi dq_s/dq */
  double k1 = 3.0 + Fr * Fr + 3.0 * xdq;
  double k2 = -2.0 * Fr * Fr * Fr + 18.0 * Fr * (1.0 + xdq) + 27.0 * xdh / c;
  double arg = k2 / sqrt(4.0 * k1 * k1 * k1);
  if (arg_out) *arg_out = arg;
  if (!(fabs(arg) <= 1.0 + ORC_TAU_HYP)) return ORC_E_NONHYPERBOLIC;
  if (arg > 1.0) arg = 1.0;
  if (arg < -1.0) arg = -1.0;
  double phi = acos(arg);
  const double pi = 3.14159265358979323846;
  double sk = sqrt(k1);
  lam[0] = c * (2.0 / 3.0 * Fr - 2.0 / 3.0 * sk * cos(phi / 3.0 - pi / 3.0));
  lam[1] = c * (2.0 / 3.0 * Fr - 2.0 / 3.0 * sk * cos(phi / 3.0 + pi / 3.0));
  lam[2] = c * (2.0 / 3.0 * Fr + 2.0 / 3.0 * sk * cos(phi / 3.0));
  return ORC_OK;
}

/* Step 4: right eigenvectors as columns of R (Eq. RR) and left eigenvectors as
 * rows of R^-1 (Eq. RR-1 with the circular permutation Eq. circPerm). The
 * paper's wording says the rows are composed "column-wise"; the matrix that
 * inverts R has the l_i as its rows, which is what is built here. */
int orc_eigvecs_analytic(const orc_law* L, double h, double q, const double lam[3],
                         double R[9], double Rinv[9]) {
  if (!(h > 0.0)) return ORC_E_DEPTH;
  double u = q / h;
  double c2 = L->g * h;
  for (int i = 0; i < 3; ++i) {
    double d = u - lam[i];
    R[0 * 3 + i] = 1.0;
    R[1 * 3 + i] = lam[i];
    R[2 * 3 + i] = d * d / c2 - 1.0;
  }
  for (int i = 0; i < 3; ++i) {
    int j = (i < 2) ? i + 1 : i - 2; /* Eq. circPerm, 0-based */
    int k = (i < 1) ? i + 2 : i - 1;
    double den = (lam[i] - lam[j]) * (lam[i] - lam[k]);
    Rinv[i * 3 + 0] = (c2 - u * u + lam[j] * lam[k]) / den;
    Rinv[i * 3 + 1] = (2.0 * u - lam[j] - lam[k]) / den;
    Rinv[i * 3 + 2] = c2 / den;
  }
  return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* Numerical eigenstructure (original DOT, Sec. 3.1: computed by "external  */
/* numerical libraries" in the paper; here by the oracle's own routines).  */
/* ---------------------------------------------------------------------- */

/* Eigenvalues of a real 3x3 matrix with real spectrum: Householder reduction
 * to upper Hessenberg form, then single-shift QR iterations with the Wilkinson
 * shift and deflation from the bottom. Sorted ascending on return. */
int orc_qr_eigenvalues(const double A[9], double lam[3]) {
  double H[3][3];
  for (int r = 0; r < 3; ++r)
    for (int s = 0; s < 3; ++s) H[r][s] = A[r * 3 + s];
  /* Householder on rows/cols 1..2 to zero H[2][0]. */
  double x0 = H[1][0], x1 = H[2][0];
  double nx = sqrt(x0 * x0 + x1 * x1);
  if (x1 != 0.0 && nx > 0.0) {
    double v0 = x0 + (x0 >= 0.0 ? nx : -nx);
    double v1 = x1;
    double vv = v0 * v0 + v1 * v1;
    /* H <- P H P with P = I - 2 v v^T / (v^T v) on indices 1, 2 */
    for (int s = 0; s < 3; ++s) { /* left: rows 1,2 */
      double t = 2.0 * (v0 * H[1][s] + v1 * H[2][s]) / vv;
      H[1][s] -= t * v0;
      H[2][s] -= t * v1;
    }
    for (int r = 0; r < 3; ++r) { /* right: cols 1,2 */
      double t = 2.0 * (H[r][1] * v0 + H[r][2] * v1) / vv;
      H[r][1] -= t * v0;
      H[r][2] -= t * v1;
    }
    H[2][0] = 0.0;
  }
  int m = 3; /* active leading block size */
  int iters = 0;
  while (m > 1) {
    double sub = fabs(H[m - 1][m - 2]);
    double scl = fabs(H[m - 1][m - 1]) + fabs(H[m - 2][m - 2]);
    if (scl == 0.0) scl = 1.0;
    if (sub <= 1e-17 * scl) {
      lam[m - 1] = H[m - 1][m - 1];
      H[m - 1][m - 2] = 0.0;
      --m;
      iters = 0;
      continue;
    }
    if (++iters > 200) return ORC_E_NOCONVERGE;
    /* Wilkinson shift from the trailing 2x2 of the active block. */
    double a = H[m - 2][m - 2], b = H[m - 2][m - 1];
    double c = H[m - 1][m - 2], d = H[m - 1][m - 1];
    double half = 0.5 * (a - d);
    double disc = half * half + b * c;
    double mu;
    if (disc >= 0.0) {
      double sq = sqrt(disc);
      double e1 = 0.5 * (a + d) + sq, e2 = 0.5 * (a + d) - sq;
      mu = (fabs(e1 - d) < fabs(e2 - d)) ? e1 : e2;
    } else {
      mu = d;
    }
    if (iters % 11 == 10) mu = d + sub; /* exceptional shift */
    for (int r = 0; r < m; ++r) H[r][r] -= mu;
    /* QR of the Hessenberg active block by Givens rotations G_r on rows (r, r+1). */
    double cs[2], sn[2];
    for (int r = 0; r < m - 1; ++r) {
      double p = H[r][r], q2 = H[r + 1][r];
      double rr = hypot(p, q2);
      double cc = (rr == 0.0) ? 1.0 : p / rr;
      double ss = (rr == 0.0) ? 0.0 : q2 / rr;
      cs[r] = cc;
      sn[r] = ss;
      for (int s = 0; s < m; ++s) {
        double t1 = H[r][s], t2 = H[r + 1][s];
        H[r][s] = cc * t1 + ss * t2;
        H[r + 1][s] = -ss * t1 + cc * t2;
      }
    }
    /* R Q: apply G_r^T on columns (r, r+1). */
    for (int r = 0; r < m - 1; ++r) {
      double cc = cs[r], ss = sn[r];
      for (int s = 0; s < m; ++s) {
        double t1 = H[s][r], t2 = H[s][r + 1];
        H[s][r] = cc * t1 + ss * t2;
        H[s][r + 1] = -ss * t1 + cc * t2;
      }
    }
    for (int r = 0; r < m; ++r) H[r][r] += mu;
  }
  lam[0] = H[0][0];
  /* sort ascending */
  for (int i = 0; i < 3; ++i)
    for (int j = i + 1; j < 3; ++j)
      if (lam[j] < lam[i]) {
        double t = lam[i];
        lam[i] = lam[j];
        lam[j] = t;
      }
  return ORC_OK;
}

/* Right eigenvector for eigenvalue l: a null vector of (A - l I), taken as the
 * largest of the three cross products of its row pairs, scaled so that its
 * first entry is 1 when that entry is not negligible (the scaling of Eq. RR). */
static void orc_null_vector(const double A[9], double l, double v[3]) {
  double M[3][3];
  for (int r = 0; r < 3; ++r)
    for (int s = 0; s < 3; ++s) M[r][s] = A[r * 3 + s] - (r == s ? l : 0.0);
  double best[3] = {0, 0, 0}, bn = -1.0;
  for (int p = 0; p < 3; ++p) {
    int a = p, b = (p + 1) % 3;
    double cx[3] = {M[a][1] * M[b][2] - M[a][2] * M[b][1],
                    M[a][2] * M[b][0] - M[a][0] * M[b][2],
                    M[a][0] * M[b][1] - M[a][1] * M[b][0]};
    double nn = cx[0] * cx[0] + cx[1] * cx[1] + cx[2] * cx[2];
    if (nn > bn) {
      bn = nn;
      best[0] = cx[0];
      best[1] = cx[1];
      best[2] = cx[2];
    }
  }
  double nrm = sqrt(bn);
  double sc = (fabs(best[0]) > 1e-8 * nrm) ? 1.0 / best[0] : 1.0 / nrm;
  for (int i = 0; i < 3; ++i) v[i] = best[i] * sc;
}

/* Inverse of a 3x3 matrix by Gauss-Jordan elimination with partial pivoting. */
int orc_inverse3(const double M[9], double Inv[9]) {
  double a[3][6];
  for (int r = 0; r < 3; ++r) {
    for (int s = 0; s < 3; ++s) a[r][s] = M[r * 3 + s];
    for (int s = 0; s < 3; ++s) a[r][3 + s] = (r == s) ? 1.0 : 0.0;
  }
  for (int col = 0; col < 3; ++col) {
    int piv = col;
    for (int r = col + 1; r < 3; ++r)
      if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
    if (a[piv][col] == 0.0) return ORC_E_INVALID;
    if (piv != col)
      for (int s = 0; s < 6; ++s) {
        double t = a[col][s];
        a[col][s] = a[piv][s];
        a[piv][s] = t;
      }
    double p = a[col][col];
    for (int s = 0; s < 6; ++s) a[col][s] /= p;
    for (int r = 0; r < 3; ++r) {
      if (r == col) continue;
      double f = a[r][col];
      for (int s = 0; s < 6; ++s) a[r][s] -= f * a[col][s];
    }
  }
  for (int r = 0; r < 3; ++r)
    for (int s = 0; s < 3; ++s) Inv[r * 3 + s] = a[r][3 + s];
  return ORC_OK;
}

/* Numerical eigenstructure of A: eigenvalues by QR, R by null vectors,
 * R^-1 by pivoted elimination. */
int orc_eig_numeric(const double A[9], double lam[3], double R[9], double Rinv[9]) {
  int st = orc_qr_eigenvalues(A, lam);
  if (st) return st;
  for (int i = 0; i < 3; ++i) {
    double v[3];
    orc_null_vector(A, lam[i], v);
    for (int r = 0; r < 3; ++r) R[r * 3 + i] = v[r];
  }
  return orc_inverse3(R, Rinv);
}

/* ---------------------------------------------------------------------- */
/* |A| (Eq. asbA).                                                          */
/* ---------------------------------------------------------------------- */

static void orc_matmul3(const double X[9], const double Y[9], double Z[9]) {
  for (int r = 0; r < 3; ++r)
    for (int s = 0; s < 3; ++s) {
      double acc = 0.0;
      for (int t = 0; t < 3; ++t) acc += X[r * 3 + t] * Y[t * 3 + s];
      Z[r * 3 + s] = acc;
    }
}

/* Step 5 (Eq. ExAbsA): |A| = R diag(|lam|) R^-1 as two full matrix products. */
static void orc_three_product(const double R[9], const double lam[3], const double Rinv[9],
                              double out[9]) {
  double RL[9];
  for (int r = 0; r < 3; ++r)
    for (int s = 0; s < 3; ++s) RL[r * 3 + s] = R[r * 3 + s] * fabs(lam[s]);
  orc_matmul3(RL, Rinv, out);
}

/* First divided difference of f(x) = |x| on a and b, with tau = ORC_TAU_GAP * c.
 * A pair closer than tau is read as one double eigenvalue m = (a+b)/2, whose
 * slope f'(m) is sign(m), taken as 0 when |m| < tau (|x| has no derivative at
 * 0; this is the coalescence reading). Otherwise, on one side of zero f is
 * linear and the slope is exactly +-1; across zero it is (|a|-|b|)/(a-b). */
static double orc_dd1(double a, double b, double tau) {
  if (fabs(a - b) < tau) {
    double m = 0.5 * (a + b);
    if (fabs(m) < tau) return 0.0;
    return m > 0.0 ? 1.0 : -1.0;
  }
  if (a >= 0.0 && b >= 0.0) return 1.0;
  if (a <= 0.0 && b <= 0.0) return -1.0;
  return (fabs(a) - fabs(b)) / (a - b);
}

/* Newton divided-difference form of |A| on the sorted spectrum l0<=l1<=l2:
 * |A| = f[l0] I + f[l0,l1](A - l0 I) + f[l0,l1,l2](A - l0 I)(A - l1 I).
 * Equal to R|L|R^-1 when the eigenvalues are distinct (interpolation of f on
 * the spectrum), and defined without dividing by eigenvalue gaps. */
static void orc_abs_newton(const double A[9], const double lam[3], double tau, double out[9]) {
  double f0 = fabs(lam[0]);
  double f01 = orc_dd1(lam[0], lam[1], tau);
  double f12 = orc_dd1(lam[1], lam[2], tau);
  double span = lam[2] - lam[0];
  double f012 = (span < tau) ? 0.0 : (f12 - f01) / span;
  double M0[9], M1[9], P[9];
  for (int i = 0; i < 9; ++i) {
    M0[i] = A[i];
    M1[i] = A[i];
  }
  for (int i = 0; i < 3; ++i) {
    M0[i * 4] -= lam[0];
    M1[i * 4] -= lam[1];
  }
  orc_matmul3(M0, M1, P);
  for (int i = 0; i < 9; ++i) out[i] = f01 * M0[i] + f012 * P[i];
  for (int i = 0; i < 3; ++i) out[i * 4] += f0;
}

/* Sylvester's formula |A| = sum_i |l_i| prod_{j != i} (A - l_j I) / (l_i - l_j). */
static void orc_abs_sylvester(const double A[9], const double lam[3], double out[9]) {
  for (int i = 0; i < 9; ++i) out[i] = 0.0;
  for (int i = 0; i < 3; ++i) {
    int j = (i + 1) % 3, k = (i + 2) % 3;
    double Mj[9], Mk[9], P[9];
    for (int t = 0; t < 9; ++t) {
      Mj[t] = A[t];
      Mk[t] = A[t];
    }
    for (int t = 0; t < 3; ++t) {
      Mj[t * 4] -= lam[j];
      Mk[t * 4] -= lam[k];
    }
    orc_matmul3(Mj, Mk, P);
    double w = fabs(lam[i]) / ((lam[i] - lam[j]) * (lam[i] - lam[k]));
    for (int t = 0; t < 9; ++t) out[t] += w * P[t];
  }
}

static double orc_min_gap(const double lam[3]) {
  double g01 = lam[1] - lam[0], g12 = lam[2] - lam[1];
  return g01 < g12 ? g01 : g12;
}

/* |A(W)| at state (h, q) by the chosen method. With distinct eigenvalues every
 * method returns the same matrix up to rounding. When the smallest gap is below
 * ORC_TAU_GAP * c the Newton form is used, whatever the method. */
int orc_abs_matrix(const orc_law* L, int method, double h, double q, double out[9],
                   double lam_out[3]) {
  double A[9], lam[3], R[9], Rinv[9];
  int st = orc_flux_matrix(L, h, q, A);
  if (st) return st;
  double c = sqrt(L->g * h);
  if (method == ORC_ABS_NUMERIC) {
    st = orc_qr_eigenvalues(A, lam);
    if (st) return st;
  } else {
    st = orc_eigvals_analytic(L, h, q, lam, 0);
    if (st) return st;
  }
  if (lam_out) memcpy(lam_out, lam, sizeof(lam));
  if (method == ORC_ABS_NEWTON || orc_min_gap(lam) < ORC_TAU_GAP * c) {
    orc_abs_newton(A, lam, ORC_TAU_GAP * c, out);
    return ORC_OK;
  }
  switch (method) {
    case ORC_ABS_ANALYTIC:
      orc_eigvecs_analytic(L, h, q, lam, R, Rinv);
      orc_three_product(R, lam, Rinv, out);
      return ORC_OK;
    case ORC_ABS_NUMERIC:
      for (int i = 0; i < 3; ++i) {
        double v[3];
        orc_null_vector(A, lam[i], v);
        for (int r = 0; r < 3; ++r) R[r * 3 + i] = v[r];
      }
      st = orc_inverse3(R, Rinv);
      if (st) return st;
      orc_three_product(R, lam, Rinv, out);
      return ORC_OK;
    case ORC_ABS_SYLVESTER:
      orc_abs_sylvester(A, lam, out);
      return ORC_OK;
    default:
      return ORC_E_INVALID;
  }
}

/* ---------------------------------------------------------------------- */
/* DOT fluctuations (Eq. path, Eq. DOTjumpN) with G = 3 Gauss-Legendre.    */
/* ---------------------------------------------------------------------- */

/* Gauss-Legendre nodes and weights on [0, 1] for G = 3: s = 1/2 -+ sqrt(15)/10,
 * 1/2; w = 5/18, 8/18, 5/18 (the G-point rule of Eq. DOTjumpN with G = 3). */
static void orc_gl3(double s[3], double w[3]) {
  double r = sqrt(15.0) / 10.0;
  s[0] = 0.5 - r;
  s[1] = 0.5;
  s[2] = 0.5 + r;
  w[0] = 5.0 / 18.0;
  w[1] = 8.0 / 18.0;
  w[2] = 5.0 / 18.0;
}

/* One edge: D-/+ = 1/2 sum_k w_k (A(Psi_k) -/+ |A(Psi_k)|) (W+ - W-), with the
 * segment path Psi(s) = W- + s (W+ - W-) (Eq. path). */
int orc_fluct_edge(const orc_law* L, int method, const double WL[3], const double WR[3],
                   double Dm[3], double Dp[3]) {
  double s[3], w[3];
  orc_gl3(s, w);
  double dW[3] = {WR[0] - WL[0], WR[1] - WL[1], WR[2] - WL[2]};
  double Mm[9] = {0}, Mp[9] = {0};
  for (int k = 0; k < 3; ++k) {
    double ph = WL[0] + s[k] * dW[0];
    double pq = WL[1] + s[k] * dW[1];
    double A[9], Aabs[9];
    int st = orc_flux_matrix(L, ph, pq, A);
    if (st) return st;
    st = orc_abs_matrix(L, method, ph, pq, Aabs, 0);
    if (st) return st;
    for (int i = 0; i < 9; ++i) {
      Mm[i] += 0.5 * w[k] * (A[i] - Aabs[i]);
      Mp[i] += 0.5 * w[k] * (A[i] + Aabs[i]);
    }
  }
  for (int r = 0; r < 3; ++r) {
    Dm[r] = Mm[r * 3 + 0] * dW[0] + Mm[r * 3 + 1] * dW[1] + Mm[r * 3 + 2] * dW[2];
    Dp[r] = Mp[r * 3 + 0] * dW[0] + Mp[r * 3 + 1] * dW[1] + Mp[r * 3 + 2] * dW[2];
  }
  return ORC_OK;
}

/* Batch of n edges; arrays are [3][n] (row 0 = h, row 1 = q, row 2 = z).
 * Returns the first non-OK status (edges are still all attempted). */
int orc_fluct(const orc_law* L, int method, int64_t n, const double* WL, const double* WR,
              double* Dm, double* Dp) {
  int status = ORC_OK;
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < n; ++e) {
    double wl[3] = {WL[e], WL[n + e], WL[2 * n + e]};
    double wr[3] = {WR[e], WR[n + e], WR[2 * n + e]};
    double dm[3], dp[3];
    int st = orc_fluct_edge(L, method, wl, wr, dm, dp);
    if (st) {
#pragma omp critical
      if (!status) status = st;
      dm[0] = dm[1] = dm[2] = dp[0] = dp[1] = dp[2] = NAN;
    }
    for (int r = 0; r < 3; ++r) {
      Dm[r * n + e] = dm[r];
      Dp[r * n + e] = dp[r];
    }
  }
  return status;
}

/* ---------------------------------------------------------------------- */
/* PRICE-C jump function (Sec. 3.2), the paper's centred comparison scheme. */
/* ---------------------------------------------------------------------- */

/* A^Psi = integral over [0, 1] of A(Psi(W-, W+, s)) ds along the segment path
 * (Eq. Apsi, Eq. path), row-major, with the 3-point Gauss-Legendre rule that
 * Eq. DOTjumpN uses for the DOT integral. */
int orc_a_psi(const orc_law* L, const double WL[3], const double WR[3], double out[9]) {
  double s[3], w[3];
  orc_gl3(s, w);
  for (int i = 0; i < 9; ++i) out[i] = 0.0;
  for (int k = 0; k < 3; ++k) {
    double ph = WL[0] + s[k] * (WR[0] - WL[0]);
    double pq = WL[1] + s[k] * (WR[1] - WL[1]);
    double A[9];
    int st = orc_flux_matrix(L, ph, pq, A);
    if (st) return st;
    for (int i = 0; i < 9; ++i) out[i] += w[k] * A[i];
  }
  return ORC_OK;
}

/* PRICE-C fluctuations of one edge (Eq. PRICEjump, Eq. AiPRICE, Eq. Im):
 *   A-/+ = 1/4 [ 2 A^Psi -/+ (dx/dt) I_eps -/+ (dt/dx) (A^Psi)^2 ],
 *   D-/+ = A-/+ (W+ - W-),   I_eps = diag(1, 1, eps),
 * given nu = dt/dx > 0. Each matrix is formed in full, as printed. */
int orc_price_fluct_edge(const orc_law* L, const double WL[3], const double WR[3], double nu,
                         double eps, double Dm[3], double Dp[3]) {
  if (!(nu > 0.0)) return ORC_E_INVALID;
  double Ap[9], Ap2[9];
  int st = orc_a_psi(L, WL, WR, Ap);
  if (st) return st;
  orc_matmul3(Ap, Ap, Ap2);
  double Ie[9] = {1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, eps};
  double Mm[9], Mp[9];
  for (int i = 0; i < 9; ++i) {
    Mm[i] = 0.25 * (2.0 * Ap[i] - (1.0 / nu) * Ie[i] - nu * Ap2[i]);
    Mp[i] = 0.25 * (2.0 * Ap[i] + (1.0 / nu) * Ie[i] + nu * Ap2[i]);
  }
  double dW[3] = {WR[0] - WL[0], WR[1] - WL[1], WR[2] - WL[2]};
  for (int r = 0; r < 3; ++r) {
    Dm[r] = Mm[r * 3 + 0] * dW[0] + Mm[r * 3 + 1] * dW[1] + Mm[r * 3 + 2] * dW[2];
    Dp[r] = Mp[r * 3 + 0] * dW[0] + Mp[r * 3 + 1] * dW[1] + Mp[r * 3 + 2] * dW[2];
  }
  return ORC_OK;
}

/* Batch of n PRICE-C edges; arrays are [3][n]. */
int orc_price_fluct(const orc_law* L, int64_t n, const double* WL, const double* WR, double nu,
                    double eps, double* Dm, double* Dp) {
  int status = ORC_OK;
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < n; ++e) {
    double wl[3] = {WL[e], WL[n + e], WL[2 * n + e]};
    double wr[3] = {WR[e], WR[n + e], WR[2 * n + e]};
    double dm[3], dp[3];
    int st = orc_price_fluct_edge(L, wl, wr, nu, eps, dm, dp);
    if (st) {
#pragma omp critical
      if (!status) status = st;
      dm[0] = dm[1] = dm[2] = dp[0] = dp[1] = dp[2] = NAN;
    }
    for (int r = 0; r < 3; ++r) {
      Dm[r * n + e] = dm[r];
      Dp[r * n + e] = dp[r];
    }
  }
  return status;
}

/* ---------------------------------------------------------------------- */
/* Time loop (Eq. scheme).                                                 */
/* ---------------------------------------------------------------------- */

/* Largest characteristic speed max(|l1|, |l3|) at a state: the extreme
 * eigenvalues bound the spectrum since l1 <= l2 <= l3. */
int orc_spectral_radius(const orc_law* L, double h, double q, double* rho) {
  double lam[3];
  int st = orc_eigvals_analytic(L, h, q, lam, 0);
  if (st) return st;
  double a = fabs(lam[0]), b = fabs(lam[2]);
  *rho = a > b ? a : b;
  return ORC_OK;
}

/* Ghost state beyond one end: adj = the cell next to the end, nxt = the one
 * after it (equal to adj when the domain has one cell). The extrapolating
 * kinds continue the bed of a sloping flume, z_g = 2 z_adj - z_nxt, so that a
 * uniform flow on a constant slope meets the same bed step at the end edge as
 * at every inner edge. */
static void orc_ghost(int kind, const double v[3], double t, const double adj[3],
                      const double nxt[3], double out[3]) {
  out[0] = adj[0];
  out[1] = adj[1];
  out[2] = adj[2];
  switch (kind) {
    case ORC_BC_INFLOW_Q: out[1] = v[0]; break;
    case ORC_BC_OUTFLOW_H: out[0] = v[0]; break;
    case ORC_BC_INFLOW_QZ:
      out[1] = v[0];
      out[2] = v[1] - v[2] * t;
      break;
    case ORC_BC_INFLOW_QS:
      out[1] = v[0];
      out[2] = 2.0 * adj[2] - nxt[2];
      break;
    case ORC_BC_OUTFLOW_HS:
      out[0] = v[0];
      out[2] = 2.0 * adj[2] - nxt[2];
      break;
    default: break; /* transmissive: copy */
  }
}

/* Momentum source of Eq. SV-Ex2 at a cell state, -g h s_f with the Strickler
 * closure of Sec. 2, s_f = q|q| / (K_s^2 h^(10/3)) (the printed q^2 taken with
 * the sign of q, so that friction opposes the flow in both directions). */
static double orc_friction_source(double g, double ks, double h, double q) {
  double sf = q * fabs(q) / (ks * ks * pow(h, 10.0 / 3.0));
  return -g * h * sf;
}

/* ---------------------------------------------------------------------- */
/* Second-order variant: MUSCL-Hancock in path-conservative form.           */
/* ---------------------------------------------------------------------- */

/* The paper applies A-DOT to the first-order scheme and notes (Sec. 6) that
 * nothing restricts the order. This variant is the standard path-conservative
 * reconstruction of states (Castro, Gallardo & Pares, Math. Comp. 2006) with a
 * Hancock half-step predictor, built on the same DOT edge (Eq. DOTjumpN):
 *   1. per cell, slopes of (eta = h + z, q, z) limited by minmod against both
 *      neighbours; boundary values W-_i, W+_i at the cell's left and right
 *      ends (reconstructing eta keeps a lake at rest exactly at rest);
 *   2. predictor: both values advance half a step by the quasi-linear form
 *      with the cell's own matrix, W+-_i <- W+-_i - dt/(2 dx) A(W_i) (W+_i - W-_i);
 *   3. update: W_i <- W_i - dt/dx (D-(W+_i, W-_{i+1}) + D+(W+_{i-1}, W-_i)
 *      + sum_k w_k A(Psi_i(s_k)) (W+_i - W-_i)), the last term being the
 *      path integral of A along the segment inside the cell, on the same
 *      three Gauss-Legendre nodes.
 * A cell whose reconstructed or predicted depth is not positive keeps zero
 * slopes (then W-_i = W+_i = W_i and the cell term vanishes). Ghost cells are
 * those of the first-order scheme, with zero slopes. */
static double orc_minmod(double a, double b) {
  if (a > 0.0 && b > 0.0) return a < b ? a : b;
  if (a < 0.0 && b < 0.0) return a > b ? a : b;
  return 0.0;
}

/* State of cell j, -1 <= j <= n, with the ghost rules or the periodic wrap. */
static void orc_cell_or_ghost(const orc_cfg* cfg, int periodic, const double* h, const double* q,
                              const double* z, int64_t j, double t, double out[3]) {
  int64_t n = cfg->n;
  if (j >= 0 && j < n) {
    out[0] = h[j]; out[1] = q[j]; out[2] = z[j];
  } else if (periodic) {
    int64_t k = (j < 0) ? j + n : j - n;
    out[0] = h[k]; out[1] = q[k]; out[2] = z[k];
  } else if (j < 0) {
    int64_t k = (n > 1) ? 1 : 0;
    double adj[3] = {h[0], q[0], z[0]}, nxt[3] = {h[k], q[k], z[k]};
    orc_ghost(cfg->bc_left, cfg->bcl, t, adj, nxt, out);
  } else {
    int64_t k = (n > 1) ? n - 2 : 0;
    double adj[3] = {h[n - 1], q[n - 1], z[n - 1]}, nxt[3] = {h[k], q[k], z[k]};
    orc_ghost(cfg->bc_right, cfg->bcr, t, adj, nxt, out);
  }
}

/* Edge fluctuations Dm, Dp ([3][n+1]) and cell terms Ic ([3][n]) of one
 * MUSCL-Hancock step; Wb ([6][n]) receives the predicted W-_i (rows 0-2) and
 * W+_i (rows 3-5). */
static int orc_mh_terms(const orc_cfg* cfg, int periodic, const double* h, const double* q,
                        const double* z, double t, double dt, double dx, double* Dm, double* Dp,
                        double* Ic, double* Wb) {
  const orc_law* L = &cfg->law;
  int64_t n = cfg->n, ne = n + 1;
  double half = 0.5 * dt / dx;
  for (int64_t i = 0; i < n; ++i) {
    double Wm[3], W0[3], Wp[3];
    orc_cell_or_ghost(cfg, periodic, h, q, z, i - 1, t, Wm);
    orc_cell_or_ghost(cfg, periodic, h, q, z, i, t, W0);
    orc_cell_or_ghost(cfg, periodic, h, q, z, i + 1, t, Wp);
    double Vm[3] = {Wm[0] + Wm[2], Wm[1], Wm[2]};
    double V0[3] = {W0[0] + W0[2], W0[1], W0[2]};
    double Vp[3] = {Wp[0] + Wp[2], Wp[1], Wp[2]};
    double sv[3], WL[3], WR[3];
    for (int r = 0; r < 3; ++r)
      sv[r] = (cfg->limiter == 1) ? 0.0 : orc_minmod(V0[r] - Vm[r], Vp[r] - V0[r]);
    /* slopes of (h, q, z): the h slope is the eta slope minus the z slope */
    double sw[3] = {sv[0] - sv[2], sv[1], sv[2]};
    for (int r = 0; r < 3; ++r) {
      WL[r] = W0[r] - 0.5 * sw[r];
      WR[r] = W0[r] + 0.5 * sw[r];
    }
    int flat = !(WL[0] > 0.0) || !(WR[0] > 0.0);
    if (!flat) {
      double A[9];
      int st = orc_flux_matrix(L, W0[0], W0[1], A);
      if (st) return st;
      double d[3] = {WR[0] - WL[0], WR[1] - WL[1], WR[2] - WL[2]};
      for (int r = 0; r < 3; ++r) {
        double Ad = A[3 * r] * d[0] + A[3 * r + 1] * d[1] + A[3 * r + 2] * d[2];
        WL[r] -= half * Ad;
        WR[r] -= half * Ad;
      }
      flat = !(WL[0] > 0.0) || !(WR[0] > 0.0);
    }
    if (flat) {
      for (int r = 0; r < 3; ++r) WL[r] = WR[r] = W0[r];
    }
    for (int r = 0; r < 3; ++r) {
      Wb[r * n + i] = WL[r];
      Wb[(3 + r) * n + i] = WR[r];
    }
  }
  int status = ORC_OK;
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < ne; ++e) {
    double wl[3], wr[3];
    if (e == 0 && !periodic) {
      orc_cell_or_ghost(cfg, periodic, h, q, z, -1, t, wl);
    } else {
      int64_t il = (e == 0) ? n - 1 : e - 1;
      for (int r = 0; r < 3; ++r) wl[r] = Wb[(3 + r) * n + il];
    }
    if (e == n && !periodic) {
      orc_cell_or_ghost(cfg, periodic, h, q, z, n, t, wr);
    } else {
      int64_t ir = (e == n) ? 0 : e;
      for (int r = 0; r < 3; ++r) wr[r] = Wb[r * n + ir];
    }
    double dm[3], dp[3];
    int st = orc_fluct_edge(L, cfg->abs_method, wl, wr, dm, dp);
    if (st) {
#pragma omp critical
      if (!status) status = st;
    }
    for (int r = 0; r < 3; ++r) {
      Dm[r * ne + e] = dm[r];
      Dp[r * ne + e] = dp[r];
    }
  }
  if (status) return status;
  double s[3], w[3];
  orc_gl3(s, w);
  for (int64_t i = 0; i < n; ++i) {
    double WL[3], d[3], acc[3] = {0.0, 0.0, 0.0};
    for (int r = 0; r < 3; ++r) {
      WL[r] = Wb[r * n + i];
      d[r] = Wb[(3 + r) * n + i] - WL[r];
    }
    for (int k = 0; k < 3; ++k) {
      double A[9];
      int st = orc_flux_matrix(L, WL[0] + s[k] * d[0], WL[1] + s[k] * d[1], A);
      if (st) return st;
      for (int r = 0; r < 3; ++r)
        acc[r] += w[k] * (A[3 * r] * d[0] + A[3 * r + 1] * d[1] + A[3 * r + 2] * d[2]);
    }
    for (int r = 0; r < 3; ++r) Ic[r * n + i] = acc[r];
  }
  return ORC_OK;
}

/* Advances the state (h, q, z arrays of n cells, in place) by at most
 * max_steps steps of Eq. scheme, stopping when the time reaches t_end.
 * Per step: dt = cfl * dx / max_i max(|l1|, |l3|)(W_i) over the cells; the last
 * step is shortened so that t lands on t_end. Edge e (0..n) joins cells e-1
 * and e; ghost cells follow the boundary kinds (evaluated at the step's start
 * time). Cell i takes D+ of edge i and D- of edge i+1.
 * *t_io: start time in, end time out. */
int orc_run(const orc_cfg* cfg, double* h, double* q, double* z, int64_t max_steps,
            double t_end, double* t_io, int64_t* steps_out, double* dt_last,
            double* work /* 6*(n+1) doubles */) {
  int64_t n = cfg->n;
  if (n < 1 || !(cfg->cfl > 0.0) || !(cfg->x_max > cfg->x_min)) return ORC_E_INVALID;
  int periodic = (cfg->bc_left == ORC_BC_PERIODIC);
  if (periodic != (cfg->bc_right == ORC_BC_PERIODIC)) return ORC_E_INVALID;
  if (!(cfg->ks >= 0.0)) return ORC_E_INVALID;
  int order2 = (cfg->order == 2);
  if (cfg->order < 0 || cfg->order > 2) return ORC_E_INVALID;
  int price = (cfg->scheme == ORC_SCHEME_PRICE_C);
  if (cfg->scheme != ORC_SCHEME_DOT && !price) return ORC_E_INVALID;
  /* PRICE-C enters the first-order scheme only */
  if (price && (order2 || !(cfg->price_eps >= 0.0) || !isfinite(cfg->price_eps)))
    return ORC_E_INVALID;
  /* the second-order variant covers the frictionless scheme without a feed */
  if (order2 && (cfg->ks > 0.0 || cfg->bc_left == ORC_BC_INFLOW_QS ||
                 cfg->bc_right == ORC_BC_INFLOW_QS))
    return ORC_E_INVALID;
  double dx = (cfg->x_max - cfg->x_min) / (double)n;
  int64_t ne = n + 1;
  double* Dm = work;
  double* Dp = work + 3 * ne;
  double t = *t_io;
  int64_t steps = 0;
  int status = ORC_OK;
  double *Ic = NULL, *Wb = NULL;
  if (order2) {
    Ic = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    Wb = (double*)malloc(sizeof(double) * 6 * (size_t)n);
    if (!Ic || !Wb) {
      free(Ic);
      free(Wb);
      return ORC_E_INVALID;
    }
  }
  if (steps_out) *steps_out = 0;
  while (steps < max_steps && t < t_end) {
    /* CFL */
    double rho = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      double r;
      int st = orc_spectral_radius(&cfg->law, h[i], q[i], &r);
      if (st) {
        status = st;
        break;
      }
      if (r > rho) rho = r;
    }
    if (status) break;
    if (!(rho > 0.0) || !isfinite(rho)) {
      status = ORC_E_NONFINITE;
      break;
    }
    double dt = cfg->cfl * dx / rho;
    if (t + dt >= t_end) dt = t_end - t;
    if (order2) {
      /* second-order variant: MUSCL-Hancock terms, then the update */
      status = orc_mh_terms(cfg, periodic, h, q, z, t, dt, dx, Dm, Dp, Ic, Wb);
      if (status) break;
      double nu2 = dt / dx;
      for (int64_t i = 0; i < n; ++i) {
        h[i] = h[i] - nu2 * (Dm[0 * ne + i + 1] + Dp[0 * ne + i] + Ic[0 * n + i]);
        q[i] = q[i] - nu2 * (Dm[1 * ne + i + 1] + Dp[1 * ne + i] + Ic[1 * n + i]);
        z[i] = z[i] - nu2 * (Dm[2 * ne + i + 1] + Dp[2 * ne + i] + Ic[2 * n + i]);
        if (!(h[i] > 0.0)) status = ORC_E_DEPTH;
        if (!isfinite(h[i]) || !isfinite(q[i]) || !isfinite(z[i])) status = ORC_E_NONFINITE;
      }
      t += dt;
      ++steps;
      if (dt_last) *dt_last = dt;
      if (steps_out) *steps_out = steps;
      if (status) break;
      continue;
    }
    /* fluctuations on every edge */
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < ne; ++e) {
      double wl[3], wr[3];
      if (periodic) {
        int64_t il = (e == 0) ? n - 1 : e - 1;
        int64_t ir = (e == n) ? 0 : e;
        wl[0] = h[il]; wl[1] = q[il]; wl[2] = z[il];
        wr[0] = h[ir]; wr[1] = q[ir]; wr[2] = z[ir];
      } else if (e == 0) {
        int64_t j = (n > 1) ? 1 : 0;
        double adj[3] = {h[0], q[0], z[0]};
        double nxt[3] = {h[j], q[j], z[j]};
        orc_ghost(cfg->bc_left, cfg->bcl, t, adj, nxt, wl);
        wr[0] = h[0]; wr[1] = q[0]; wr[2] = z[0];
      } else if (e == n) {
        int64_t j = (n > 1) ? n - 2 : 0;
        double adj[3] = {h[n - 1], q[n - 1], z[n - 1]};
        double nxt[3] = {h[j], q[j], z[j]};
        wl[0] = h[n - 1]; wl[1] = q[n - 1]; wl[2] = z[n - 1];
        orc_ghost(cfg->bc_right, cfg->bcr, t, adj, nxt, wr);
      } else {
        wl[0] = h[e - 1]; wl[1] = q[e - 1]; wl[2] = z[e - 1];
        wr[0] = h[e]; wr[1] = q[e]; wr[2] = z[e];
      }
      double dm[3], dp[3];
      int st = price ? orc_price_fluct_edge(&cfg->law, wl, wr, dt / dx, cfg->price_eps, dm, dp)
                     : orc_fluct_edge(&cfg->law, cfg->abs_method, wl, wr, dm, dp);
      if (st) {
#pragma omp critical
        if (!status) status = st;
      }
      for (int r = 0; r < 3; ++r) {
        Dm[r * ne + e] = dm[r];
        Dp[r * ne + e] = dp[r];
      }
    }
    if (status) return status;
    /* Sediment feed (Sec. 5.1: the solid discharge is set at the upstream
     * end). The bed row of Eq. scheme for cell i reads
     * z_i -= dt/dx (F_{i+1/2} - F_{i-1/2}) with the edge discharge
     * F_{i+1/2} = xi q_s(W_i) + D-_{i+1/2} = xi q_s(W_{i+1}) - D+_{i+1/2}. A
     * feeding end's edge discharge is the imposed xi q_s,in, so the bed gains
     * exactly what is fed: the bed row of D+ of edge 0 (cell 0's only left term)
     * becomes xi (q_s(W_0) - q_s,in), that of D- of edge n
     * xi (q_s,in - q_s(W_{n-1})). The h and q rows keep the DOT edge against the
     * ghost. (On a bed slope s the inner edges also carry the dissipative bed
     * flux of |A| dW, about |A|_zz s dx / 2, which the imposed discharge does
     * not; a uniform flow fed its own q_s therefore adjusts over the first cell
     * by that first-order amount.) */
    if (!periodic && (cfg->bc_left == ORC_BC_INFLOW_QS || cfg->bc_right == ORC_BC_INFLOW_QS)) {
      double xi = cfg->law.xi;
      if (cfg->bc_left == ORC_BC_INFLOW_QS) {
        double qs, a, b;
        int st = orc_sediment(&cfg->law, h[0], q[0], &qs, &a, &b);
        if (st) return st;
        Dp[2 * ne + 0] = xi * qs - xi * cfg->bcl[1];
      }
      if (cfg->bc_right == ORC_BC_INFLOW_QS) {
        double qs, a, b;
        int st = orc_sediment(&cfg->law, h[n - 1], q[n - 1], &qs, &a, &b);
        if (st) return st;
        Dm[2 * ne + n] = xi * cfg->bcr[1] - xi * qs;
      }
    }
    /* update (Eq. scheme): W_i -= dt/dx (D-_{i+1/2} + D+_{i-1/2}) - dt S(W_i),
     * S = (0, -g h s_f, 0) taken at the step's starting state */
    double nu = dt / dx;
    int friction = cfg->ks > 0.0;
    for (int64_t i = 0; i < n; ++i) {
      double h0 = h[i], q0 = q[i];
      h[i] = h0 - nu * (Dm[0 * ne + i + 1] + Dp[0 * ne + i]);
      q[i] = q0 - nu * (Dm[1 * ne + i + 1] + Dp[1 * ne + i]);
      if (friction) q[i] = q[i] + dt * orc_friction_source(cfg->law.g, cfg->ks, h0, q0);
      z[i] = z[i] - nu * (Dm[2 * ne + i + 1] + Dp[2 * ne + i]);
      if (!(h[i] > 0.0)) status = ORC_E_DEPTH;
      if (!isfinite(h[i]) || !isfinite(q[i]) || !isfinite(z[i])) status = ORC_E_NONFINITE;
    }
    t += dt;
    ++steps;
    if (dt_last) *dt_last = dt;
    if (steps_out) *steps_out = steps;
    if (status) break;
  }
  free(Ic);
  free(Wb);
  *t_io = t;
  return status;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* Quadrature average of |A| along the segment path,
 * |A|_Psi = sum_k w_k |A(Psi(s_k))| (the matrix that multiplies dW in the
 * dissipative part of Eq. DOTjumpN), row-major; the label of the learned
 * surrogate. */
int orc_abs_psi(const orc_law* L, int method, const double WL[3], const double WR[3],
                double out[9]) {
  double s[3], w[3];
  orc_gl3(s, w);
  for (int i = 0; i < 9; ++i) out[i] = 0.0;
  for (int k = 0; k < 3; ++k) {
    double ph = WL[0] + s[k] * (WR[0] - WL[0]);
    double pq = WL[1] + s[k] * (WR[1] - WL[1]);
    double X[9];
    int st = orc_abs_matrix(L, method, ph, pq, X, 0);
    if (st) return st;
    for (int i = 0; i < 9; ++i) out[i] += w[k] * X[i];
  }
  return ORC_OK;
}

/* Batch of n edges: WL, WR [3][n]; out [n][9]. */
int orc_abs_psi_batch(const orc_law* L, int method, int64_t n, const double* WL,
                      const double* WR, double* out) {
  int status = ORC_OK;
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < n; ++e) {
    double wl[3] = {WL[e], WL[n + e], WL[2 * n + e]};
    double wr[3] = {WR[e], WR[n + e], WR[2 * n + e]};
    int st = orc_abs_psi(L, method, wl, wr, out + 9 * e);
    if (st) {
#pragma omp critical
      if (!status) status = st;
    }
  }
  return status;
}
