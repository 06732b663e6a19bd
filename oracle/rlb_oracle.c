/*
 * rlb_oracle.c -- plain FP64 CPU oracle for one time step of the relativistic
 * lattice Boltzmann scheme with a quasiparticle equation of state
 * (Romatschke, "Relativistic (Lattice) Boltzmann Equation with Non-Ideal
 * Equation of State", arXiv:1108.5561).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this file.  The product (CUDA) path
 * never links, imports or calls it, and it shares no code with that path.
 *
 * It is written to be read against the paper, not to be fast:
 *   - modified Bessel functions from their integral representation,
 *   - the quasiparticle mass M(T) by safeguarded root finding (Sec. 3.1),
 *   - the bag function B(T) from thermodynamic consistency (Eq. cdef and the
 *     ODE dB/dT = -Z M^2 T K_1 dM/dT / (2 pi^2) of Sec. 3.1, integrated from
 *     B(0) = 0; equivalently B = p_kin - \int_0^T s dT'),
 *   - the momentum lattice of Sec. 4.3 (radial Gauss rule for the weight
 *     exp(-z0 cosh xi) sinh^2 xi, Gauss-Legendre in cos(theta), equispaced phi),
 *   - the Galerkin momentum-derivative operators S1, S2 of Sec. 4.4
 *     (coefficients s_1^{ml}, s_2^{ml}), built modally and then turned into
 *     nodal matrices,
 *   - Landau matching (Eq. sanity) by power iteration on T^mu_nu,
 *   - the predictor-corrector of Sec. 4.4 (Heun / trapezoid).
 * Every site is independent apart from the streaming stencil, and each is
 * evaluated with sequential sums in the node order (k fastest, then j, then l).
 *
 * The 2+1D extension (transverse streaming, flow, transverse mass-gradient
 * force) is not written out in the paper (Sec. 4.4 drops space dependence);
 * the readings used here are listed in the repository's design notes and in
 * the comments at each step below.
 *
 * Parity status: every function here is pinned by the -m "not gpu" tests
 * (closed forms, library routines, exact discrete identities, the paper's
 * 0+1D algorithm in modal form, conservation and equilibrium invariants).
 * The transverse nonlinear flow (2+1D with gradients of M) has no
 * independent pin beyond its ingredients: parity unpinned for that regime.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846
#define OR_HBARC 0.1973269804 /* GeV fm */

/* Scalar of everything that depends on the state or on eta/s (the lattice,
 * its weights and operators are plain doubles).  The default build uses
 * double.  Built with -DOR_COMPLEX_STEP the same code runs in C99 double
 * complex: an input with an imaginary part h * d (h tiny) returns outputs
 * whose imaginary parts are h times their derivatives along d, exact to
 * rounding (complex-step differentiation; every operation on the path is
 * analytic, and comparisons, brackets and convergence tests look at real
 * parts only).  That build serves as the forward-mode (tangent) oracle for
 * the adjoint's gradients. */
#ifdef OR_COMPLEX_STEP
#include <complex.h>
#undef I /* the imaginary unit is spelled _Complex_I; I is a variable name here */
typedef double _Complex real_t;
#define RE(v) creal(v)
#define R_EXP cexp
#define R_SQRT csqrt
#define R_LOG clog
#define R_COSH ccosh
#define R_TANH ctanh
#define R_POW cpow
#else
typedef double real_t;
#define RE(v) (v)
#define R_EXP exp
#define R_SQRT sqrt
#define R_LOG log
#define R_COSH cosh
#define R_TANH tanh
#define R_POW pow
#endif

/* ------------------------------------------------------------------------ */
/* parameters (mirrored by oracle/oracle.py)                                  */
/* ------------------------------------------------------------------------ */
typedef struct {
  int eos_kind;      /* 0: crossover s/T^3 = a(1+tanh((T-Tc)/w))/2 + b,
                        1: constant mass m0 (ideal massive Boltzmann gas),
                        2: conformal (M = 0)                               */
  int family;        /* radial rule: 0 = paper's R_k family, 1 = Laguerre */
  int metric;        /* 1 = Milne (tau, x, y, eta_s), 0 = Minkowski        */
  int nx, ny;        /* transverse grid                                   */
  int n_xi, n_theta, n_phi_half;
  int pad_;
  double eos_a, eos_b, eos_Tc, eos_w, eos_m0, Z;
  double z0;         /* reference M0/T0 of the radial rule (Eq. fansatz)    */
  double T0;         /* conformal momentum scale [GeV] (family 1)          */
  double dx;         /* lattice spacing [fm]                               */
  double eta_over_s; /* INFINITY switches collisions off                   */
  double eta_over_s_im; /* imaginary part of eta/s (complex-step build only) */
} or_params;

enum { OR_OK = 0, OR_ERR_ARG = -1, OR_ERR_NUMERIC = -3, OR_ERR_NOMEM = -6 };

/* ------------------------------------------------------------------------ */
/* modified Bessel functions K_0..K_3                                         */
/* K_nu(x) = \int_0^inf exp(-x cosh t) cosh(nu t) dt; the trapezoid rule on   */
/* this analytic, doubly-exponentially decaying integrand converges           */
/* geometrically in 1/h (error ~ exp(-pi^2/h)); h = 1/16 is far below 1e-16. */
/* ------------------------------------------------------------------------ */
static void bessel_k0123(real_t x, real_t K[4]) {
  const double h = 1.0 / 16.0;
  real_t e0 = R_EXP(-x);
  real_t s0 = 0.5 * e0, s1 = 0.5 * e0, s2 = 0.5 * e0, s3 = 0.5 * e0;
  for (int i = 1; i < 100000; ++i) {
    double t = i * h;
    real_t e = R_EXP(-x * cosh(t));
    double a1 = cosh(t), a2 = cosh(2 * t), a3 = cosh(3 * t);
    s0 += e;
    s1 += e * a1;
    s2 += e * a2;
    s3 += e * a3;
    if (RE(e) == 0.0 || RE(e) * a3 < 1e-22 * RE(s3)) break;
  }
  K[0] = h * s0; K[1] = h * s1; K[2] = h * s2; K[3] = h * s3;
}

/* J(x) = \int_0^inf sinh^6 t / cosh t exp(-x cosh t) dt, the shear-viscosity
 * integral of Sec. 4.1 after p = M sinh t (same trapezoid argument). */
static real_t visc_integral(real_t x) {
  const double h = 1.0 / 16.0;
  real_t s = 0.0;
  for (int i = 1; i < 100000; ++i) {
    double t = i * h;
    double sh = sinh(t), ch = cosh(t);
    real_t e = R_EXP(-x * ch);
    real_t term = e * sh * sh * sh * sh * sh * sh / ch;
    s += term;
    if (RE(e) == 0.0 || (t > 1.0 && RE(term) < 1e-22 * RE(s))) break;
  }
  return h * s;
}

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre rule on [-1,1] (Sec. 4.3: theta nodes are roots of L_N)    */
/* Newton iteration on the three-term recurrence; weights 2/((1-x^2)L_N'^2). */
/* ------------------------------------------------------------------------ */
static void legendre_eval(int n, long double x, long double* p, long double* dp) {
  long double p0 = 1.0L, p1 = x;
  if (n == 0) { *p = 1.0L; *dp = 0.0L; return; }
  for (int k = 2; k <= n; ++k) {
    long double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
    p0 = p1; p1 = p2;
  }
  *p = p1;
  *dp = n * (x * p1 - p0) / (x * x - 1.0L);
}

static void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    /* root i counted from +1 downwards, then stored ascending */
    long double z = cosl(OR_PI * (i + 0.75L) / (n + 0.5L));
    long double p, dp;
    for (int it = 0; it < 100; ++it) {
      legendre_eval(n, z, &p, &dp);
      long double dz = p / dp;
      z -= dz;
      if (fabsl(dz) < 1e-19L) break;
    }
    legendre_eval(n, z, &p, &dp);
    x[n - 1 - i] = (double)z;
    w[n - 1 - i] = (double)(2.0L / ((1.0L - z * z) * dp * dp));
  }
}

/* ------------------------------------------------------------------------ */
/* equation of state (Sec. 2.1, Eq. epsp, Sec. 3.1)                           */
/* ------------------------------------------------------------------------ */
typedef struct {
  real_t T;     /* GeV                                   */
  real_t x;     /* M/T                                   */
  real_t M;     /* equilibrium quasiparticle mass M(T)   */
  real_t s;     /* entropy density s(T)  [GeV^3]         */
  real_t sp;    /* ds/dT                                 */
  real_t pkin;  /* Z M^2 T^2 K_2(M/T)/(2 pi^2)           */
  real_t e;     /* kinetic equilibrium energy eps - B    */
  real_t ep;    /* de/dT                                 */
  real_t Bp;    /* dB/dT                                 */
  real_t D;     /* dB/deps = B'(T) / (T s'(T))           */
  real_t J;     /* \int d^3p/(2pi)^3 p^4/E^2 e^{-E/T}    */
  real_t tauR;  /* relaxation time [fm] (Sec. 4.1)       */
} eos_pt;

static real_t sigma_of(const or_params* P, real_t T) {
  return P->eos_a * 0.5 * (1.0 + R_TANH((T - P->eos_Tc) / P->eos_w)) + P->eos_b;
}
static real_t sigmap_of(const or_params* P, real_t T) {
  real_t c = R_COSH((T - P->eos_Tc) / P->eos_w);
  return P->eos_a * 0.5 / (P->eos_w * c * c);
}

/* x^3 K_3(x) decreases monotonically from 8 (x -> 0) to 0; solve
 * x^3 K_3(x) = tgt by Newton (derivative -x^3 K_2) inside a bisection bracket. */
static real_t solve_x(real_t tgt, double guess) {
  double lo = 1e-9, hi = 200.0;
  real_t x = guess;
  if (!(RE(x) > lo && RE(x) < hi)) x = 2.0;
  for (int it = 0; it < 300; ++it) {
    real_t K[4];
    bessel_k0123(x, K);
    real_t F = x * x * x * K[3] - tgt;
    if (RE(F) > 0) lo = RE(x); else hi = RE(x);
    real_t dF = -x * x * x * K[2];
    real_t xn = x - F / dF;
    if (!(RE(xn) > lo && RE(xn) < hi)) xn = 0.5 * (lo + hi);
    if (fabs(RE(xn) - RE(x)) <= 1e-16 * RE(x)) { x = xn; break; }
    x = xn;
    if (hi - lo <= 2e-16 * hi) break;
  }
#ifdef OR_COMPLEX_STEP
  {  /* one Newton step at the converged point sets the imaginary part exactly
        (a bisection step would have dropped it) */
    real_t K[4];
    bessel_k0123(x, K);
    x = x - (x * x * x * K[3] - tgt) / (-x * x * x * K[2]);
  }
#endif
  return x;
}

/* All local EOS quantities at temperature T (everything except B and p,
 * which need the integral of s). */
static void eos_eval(const or_params* P, real_t T, double x_guess, eos_pt* o) {
  const double Z = P->Z, c2 = 2.0 * OR_PI * OR_PI;
  memset(o, 0, sizeof(*o));
  o->T = T;
  if (P->eos_kind == 2) { /* conformal: M = B = 0, s = 4 Z T^3 / pi^2 */
    o->x = 0.0; o->M = 0.0;
    o->s = 4.0 * Z * T * T * T / (OR_PI * OR_PI);
    o->sp = 3.0 * o->s / T;
    o->pkin = Z * T * T * T * T / (OR_PI * OR_PI);
    o->e = 3.0 * o->pkin;
    o->ep = 4.0 * o->e / T;
    o->Bp = 0.0; o->D = 0.0;
    o->J = 24.0 * R_POW(T, 5) / c2;
  } else {
    real_t x, K[4];
    if (P->eos_kind == 1) {
      x = P->eos_m0 / T;
      bessel_k0123(x, K);
      o->s = Z * pow(P->eos_m0, 3) * K[3] / c2;
      o->sp = Z * pow(P->eos_m0, 3) * (x * K[2] + 3.0 * K[3]) / (c2 * T);
      o->Bp = 0.0;
    } else {
      real_t sg = sigma_of(P, T);
      x = solve_x(c2 * sg / Z, x_guess);
      bessel_k0123(x, K);
      o->s = T * T * T * sg;
      o->sp = 3.0 * T * T * sg + T * T * T * sigmap_of(P, T);
      /* implicit derivative of x^3 K_3(x) = 2 pi^2 sigma(T)/Z */
      real_t xp = -(c2 * sigmap_of(P, T) / Z) / (x * x * x * K[2]);
      real_t Mp = x + T * xp;
      real_t M = x * T;
      o->Bp = -Z * M * M * T * K[1] * Mp / c2; /* Sec. 3.1 consistency ODE */
    }
    o->x = x;
    o->M = x * T;
    o->pkin = Z * o->M * o->M * T * T * K[2] / c2;
    o->e = T * o->s - o->pkin;     /* = Z M^2 T^2 [3 K_2 + x K_1]/(2 pi^2) */
    o->ep = T * o->sp - o->Bp;
    o->D = o->Bp / (T * o->sp);
    o->J = R_POW(o->M, 5) * visc_integral(x) / c2;
  }
  /* eta = tau_R Z J / (15 T), eta = (eta/s) s  (Sec. 4.1) */
#ifdef OR_COMPLEX_STEP
  const real_t eta_s = P->eta_over_s + _Complex_I * P->eta_over_s_im;
#else
  const real_t eta_s = P->eta_over_s;
#endif
  real_t tauR_GeV = 15.0 * T * eta_s * o->s / (Z * o->J);
  o->tauR = tauR_GeV * OR_HBARC;
}


/* ------------------------------------------------------------------------ */
/* oracle context: parameters, momentum lattice, nodal operator matrices      */
/* ------------------------------------------------------------------------ */
#define OR_MAXN 32
typedef struct or_ctx {
  or_params P;
  int nxi, nth, nph, nn;        /* nph = 2 N_phi                          */
  double zexp;                  /* exponent scale of the radial weight    */
  /* radial nodes: c = cosh xi (family 0) or x (family 1), s = sinh xi or x */
  double c[OR_MAXN], s[OR_MAXN], wxi[OR_MAXN], ecw[OR_MAXN];
  double mu[OR_MAXN], sth[OR_MAXN], wth[OR_MAXN];
  double phi[OR_MAXN], cph[OR_MAXN], sph[OR_MAXN];
  double Dr[OR_MAXN * OR_MAXN], Dth[OR_MAXN * OR_MAXN];
  double g16x[16], g16w[16];
} or_ctx;

/* p(T) = \int_0^T s(T') dT' (composite 16-point Gauss-Legendre panels of width
 * <= 0.005 GeV; s(T) = T^3 sigma(T) is analytic within pi w/2 of the real axis,
 * so every panel is exact to rounding).  B = p_kin - p is then the solution of
 * the consistency ODE of Sec. 3.1 with B(0) = 0, because dp_kin/dT = s + dB/dT. */
static real_t p_of_T(const or_ctx* C, real_t T, const eos_pt* e) {
  const or_params* P = &C->P;
  if (P->eos_kind == 2) return P->Z * T * T * T * T / (OR_PI * OR_PI);
  if (P->eos_kind == 1) return e->pkin;
  int npan = (int)ceil(RE(T) / 0.005);
  if (npan < 1) npan = 1;
  real_t h = T / npan, sum = 0.0;
  for (int q = 0; q < npan; ++q) {
    real_t a = q * h, part = 0.0;
    for (int i = 0; i < 16; ++i) {
      real_t t = a + 0.5 * h * (C->g16x[i] + 1.0);
      part += C->g16w[i] * t * t * t * sigma_of(P, t);
    }
    sum += 0.5 * h * part;
  }
  return sum;
}

static real_t B_of_T(const or_ctx* C, real_t T, const eos_pt* e) {
  if (C->P.eos_kind != 0) return 0.0;
  return e->pkin - p_of_T(C, T, e);
}

/* Solve ln e(T) = ln target for T by Newton in ln T, inside a bisection
 * bracket.  which = 0: e = eps - B (kinetic matching, Eq. sanity with B at its
 * equilibrium value); which = 1: e = eps_EOS(T) = T s - p (initial condition). */
static int solve_T(const or_ctx* C, real_t target, int which, double T_guess, real_t* T_out,
                   eos_pt* e_out) {
  double ylo = log(1e-3), yhi = log(50.0);
  real_t y = (T_guess > 1e-3 && T_guess < 50.0) ? log(T_guess) : log(0.3);
  real_t lt = R_LOG(target);
  double xg = 2.0;
  eos_pt e;
  for (int it = 0; it < 400; ++it) {
    real_t T = R_EXP(y);
    eos_eval(&C->P, T, xg, &e);
    xg = RE(e.x);
    real_t val, dval;
    if (which == 0) { val = e.e; dval = e.ep; }
    else { val = T * e.s - p_of_T(C, T, &e); dval = T * e.sp; }
    real_t F = R_LOG(val) - lt;
    if (RE(F) < 0) ylo = RE(y); else yhi = RE(y);
    real_t yn = y - F / (T * dval / val);
    if (!(RE(yn) > ylo && RE(yn) < yhi)) yn = 0.5 * (ylo + yhi);
    if (fabs(RE(yn) - RE(y)) < 1e-15) {
      y = yn;
      T = R_EXP(y);
      eos_eval(&C->P, T, xg, &e);
#ifdef OR_COMPLEX_STEP
      {  /* one more Newton step: the imaginary part of y is then exact */
        real_t v2 = which == 0 ? e.e : T * e.s - p_of_T(C, T, &e), d2 = which == 0 ? e.ep : T * e.sp;
        y = y - (R_LOG(v2) - lt) / (T * d2 / v2);
        T = R_EXP(y);
        eos_eval(&C->P, T, xg, &e);
      }
#endif
      *T_out = T;
      if (e_out) *e_out = e;
      return OR_OK;
    }
    y = yn;
    if (yhi - ylo < 1e-15) break;
  }
  *T_out = R_EXP(y);
  eos_eval(&C->P, *T_out, xg, &e);
  if (e_out) *e_out = e;
  return (yhi - ylo < 1e-13) ? OR_OK : OR_ERR_NUMERIC;
}

/* ------------------------------------------------------------------------ */
/* radial quadrature (Sec. 4.3)                                               */
/* Family 0: polynomials R_k(cosh xi) orthogonal for \int dxi e^{-z0 cosh xi} */
/* sinh^2 xi; nodes are the roots of R_{N_xi}, weights satisfy                 */
/* sum w R_0 = K_1(z0)/z0.  The monic recurrence is found by the Stieltjes     */
/* procedure on a fine composite Gauss-Legendre discretisation in xi.          */
/* Family 1: the z0 -> 0 limit in the variable x = |p|/T0: weight x e^{-x}     */
/* (generalised Laguerre, alpha = 1), recurrence in closed form.               */
/* ------------------------------------------------------------------------ */
static void gauss_legendre_l(int n, long double* x, long double* w) {
  for (int i = 0; i < n; ++i) {
    long double z = cosl(OR_PI * (i + 0.75L) / (n + 0.5L));
    long double p, dp;
    for (int it = 0; it < 100; ++it) {
      legendre_eval(n, z, &p, &dp);
      long double dz = p / dp;
      z -= dz;
      if (fabsl(dz) < 1e-21L) break;
    }
    legendre_eval(n, z, &p, &dp);
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0L / ((1.0L - z * z) * dp * dp);
  }
}

static int radial_recurrence(const or_params* P, int N, long double* al, long double* be) {
  if (P->family == 1) {
    for (int k = 0; k <= N; ++k) {
      al[k] = 2.0L * k + 2.0L;
      be[k] = (k == 0) ? 1.0L : (long double)k * (k + 1.0L);
    }
    return OR_OK;
  }
  const long double z0 = P->z0;
  const int q = 24;
  long double gx[24], gw[24];
  gauss_legendre_l(q, gx, gw);
  long double xmax = acoshl(1.0L + 1000.0L / z0);
  const long double hp = 0.05L;
  int npan = (int)ceill(xmax / hp);
  int M = npan * q;
  long double* cc = (long double*)malloc(sizeof(long double) * M * 4);
  if (!cc) return OR_ERR_NOMEM;
  long double* W = cc + M;
  long double* p0 = cc + 2 * M;
  long double* p1 = cc + 3 * M;
  for (int a = 0; a < npan; ++a)
    for (int i = 0; i < q; ++i) {
      long double xi = (a + 0.5L * (gx[i] + 1.0L)) * hp;
      long double sh = sinhl(xi);
      cc[a * q + i] = coshl(xi);
      W[a * q + i] = 0.5L * hp * gw[i] * expl(-z0 * coshl(xi)) * sh * sh;
    }
  for (int i = 0; i < M; ++i) { p0[i] = 0.0L; p1[i] = 1.0L; }
  long double nprev = 1.0L;
  for (int k = 0; k <= N; ++k) {
    long double n2 = 0.0L, xn = 0.0L;
    for (int i = 0; i < M; ++i) {
      n2 += W[i] * p1[i] * p1[i];
      xn += W[i] * cc[i] * p1[i] * p1[i];
    }
    al[k] = xn / n2;
    be[k] = (k == 0) ? n2 : n2 / nprev;
    nprev = n2;
    for (int i = 0; i < M; ++i) {
      long double pn = (cc[i] - al[k]) * p1[i] - ((k == 0) ? 0.0L : be[k]) * p0[i];
      p0[i] = p1[i];
      p1[i] = pn;
    }
  }
  free(cc);
  return OR_OK;
}

/* monic p_0..p_{N} and derivatives at x */
static void radial_polys(int N, const long double* al, const long double* be, long double x,
                         long double* p, long double* dp) {
  p[0] = 1.0L; dp[0] = 0.0L;
  if (N == 0) return;
  p[1] = x - al[0]; dp[1] = 1.0L;
  for (int k = 1; k < N; ++k) {
    p[k + 1] = (x - al[k]) * p[k] - be[k] * p[k - 1];
    dp[k + 1] = p[k] + (x - al[k]) * dp[k] - be[k] * dp[k - 1];
  }
}

static int radial_rule(const or_params* P, int N, double* nodes, double* weights) {
  long double al[OR_MAXN + 2], be[OR_MAXN + 2], p[OR_MAXN + 2], dp[OR_MAXN + 2];
  int rc = radial_recurrence(P, N, al, be);
  if (rc) return rc;
  /* bracket: support lower end, Gershgorin bound of the Jacobi matrix above */
  long double lo = (P->family == 1) ? 0.0L : 1.0L, hi = 0.0L;
  for (int k = 0; k < N; ++k) {
    long double r = al[k] + (k > 0 ? sqrtl(be[k]) : 0.0L) + (k + 1 < N ? sqrtl(be[k + 1]) : 0.0L);
    if (r > hi) hi = r;
  }
  hi += 1.0L;
  const int nscan = 400000;
  int found = 0;
  long double xa = lo, fa;
  radial_polys(N, al, be, xa, p, dp);
  fa = p[N];
  for (int i = 1; i <= nscan && found < N; ++i) {
    long double xb = lo + (hi - lo) * i / nscan, fb;
    radial_polys(N, al, be, xb, p, dp);
    fb = p[N];
    if ((fa < 0) != (fb < 0)) {
      long double a = xa, b = xb, fl = fa;
      for (int it = 0; it < 200; ++it) {
        long double m = 0.5L * (a + b);
        if (m <= a || m >= b) break;
        radial_polys(N, al, be, m, p, dp);
        if ((p[N] < 0) == (fl < 0)) { a = m; fl = p[N]; } else b = m;
      }
      long double r = 0.5L * (a + b);
      /* Christoffel weight 1 / sum_l p_l(r)^2 / ||p_l||^2 */
      radial_polys(N, al, be, r, p, dp);
      long double nrm = 1.0L, acc = 0.0L;
      for (int l = 0; l < N; ++l) {
        nrm *= be[l];
        acc += p[l] * p[l] / nrm;
      }
      nodes[found] = (double)r;
      weights[found] = (double)(1.0L / acc);
      ++found;
    }
    xa = xb; fa = fb;
  }
  return found == N ? OR_OK : OR_ERR_NUMERIC;
}

/* ------------------------------------------------------------------------ */
/* nodal operator matrices (Sec. 4.4)                                         */
/* Dr : Galerkin representation of tanh(xi) d/dxi (= v.d/dv, the radial part   */
/*      of S2 and of S1), from the s_2^{ml} bracket                            */
/*      (2 + 1/cosh^2) R_l + R_l' cosh tanh^2 (family 1: 2 R_l + x R_l').      */
/* Dth: Galerkin representation of (mu - mu^3) d/dmu, from the angular part of */
/*      s_1^{ml}: (1 - 3 mu^2) L_m + (mu - mu^3) L_m'.                          */
/*      S1 = diag(mu^2) (x) Dr + Dth (x) 1 on each phi slice, S2 = 1 (x) Dr.     */
/* Each is built as (reconstruction) x (modal Galerkin/derivative map).         */
/* ------------------------------------------------------------------------ */
static int build_operators(or_ctx* C) {
  const or_params* P = &C->P;
  const int N = C->nxi, Nt = C->nth;
  long double al[OR_MAXN + 2], be[OR_MAXN + 2];
  int rc = radial_recurrence(P, N, al, be);
  if (rc) return rc;
  /* radial: Dr[k'][k] = sum_l e^{-z c_k'} p_l(c_k') * (-1/I_l) w_k e^{z c_k} G_l(c_k) */
  long double pk[OR_MAXN][OR_MAXN + 2], dpk[OR_MAXN][OR_MAXN + 2], I[OR_MAXN];
  for (int k = 0; k < N; ++k) radial_polys(N, al, be, (long double)C->c[k], pk[k], dpk[k]);
  long double nrm = 1.0L;
  for (int l = 0; l < N; ++l) { nrm *= be[l]; I[l] = nrm; }
  for (int kp = 0; kp < N; ++kp)
    for (int k = 0; k < N; ++k) {
      long double ck = C->c[k], acc = 0.0L;
      for (int l = 0; l < N; ++l) {
        long double G;
        if (P->family == 1)
          G = 2.0L * pk[k][l] + ck * dpk[k][l];
        else
          G = (2.0L + 1.0L / (ck * ck)) * pk[k][l] + dpk[k][l] * (ck * ck - 1.0L) / ck;
        long double recon = expl(-(long double)C->zexp * C->c[kp]) * pk[kp][l];
        long double gal = -(long double)C->wxi[k] * expl((long double)C->zexp * ck) * G / I[l];
        acc += recon * gal;
      }
      C->Dr[kp * N + k] = (double)acc;
    }
  /* polar Galerkin: Dth[j'][j] = sum_m L_m(mu_j') * (-(2m+1)/2) w_j H_m(mu_j) */
  for (int jp = 0; jp < Nt; ++jp)
    for (int j = 0; j < Nt; ++j) {
      long double acc = 0.0L;
      for (int m = 0; m < Nt; ++m) {
        long double Ljp, dLjp, Lj, dLj, u = C->mu[j];
        legendre_eval(m, C->mu[jp], &Ljp, &dLjp);
        legendre_eval(m, u, &Lj, &dLj);
        if (m == 0) { dLj = 0.0L; }
        long double H = (1.0L - 3.0L * u * u) * Lj + (u - u * u * u) * dLj;
        acc += Ljp * (-(2.0L * m + 1.0L) / 2.0L) * C->wth[j] * H;
      }
      C->Dth[jp * Nt + j] = (double)acc;
    }
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Landau matching (Eq. sanity): the timelike eigenvector of T^mu_nu.          */
/* Power iteration on A = T^{mu lambda} g_{lambda nu} (g = diag(1,-1,-1,-1));  */
/* the eigenvalue of largest modulus is eps (the others are -p_i, |p_i| < eps).*/
/* Orthonormal Milne frame (tau, x, y, tau*eta_s).                             */
/* ------------------------------------------------------------------------ */
static int landau(const real_t Tk[16], real_t u[4], real_t* eps) {
  static const double g[4] = {1.0, -1.0, -1.0, -1.0};
  real_t v[4] = {1.0, 0.0, 0.0, 0.0};
  int tail = -1;
  for (int it = 0; it < 20000; ++it) {
    real_t w[4], n2 = 0.0;
    for (int m = 0; m < 4; ++m) {
      w[m] = 0.0;
      for (int nu = 0; nu < 4; ++nu) w[m] += Tk[m * 4 + nu] * g[nu] * v[nu];
      n2 += w[m] * w[m];
    }
    real_t nrm = R_SQRT(n2);
    double d = 0.0;
    if (!(RE(nrm) > 0.0)) return OR_ERR_NUMERIC;
    if (RE(w[0]) < 0) nrm = -nrm;
    for (int m = 0; m < 4; ++m) {
      w[m] /= nrm;
      d = fmax(d, fabs(RE(w[m]) - RE(v[m])));
      v[m] = w[m];
    }
    if (tail < 0 && d < 1e-15) tail = 60;
    if (tail >= 0 && tail-- == 0) break;
  }
  real_t nn = v[0] * v[0] - v[1] * v[1] - v[2] * v[2] - v[3] * v[3];
  if (!(RE(nn) > 0.0)) return OR_ERR_NUMERIC;
  real_t r = 1.0 / R_SQRT(nn);
  for (int m = 0; m < 4; ++m) u[m] = v[m] * r;
  real_t e = 0.0;
  for (int m = 0; m < 4; ++m)
    for (int nu = 0; nu < 4; ++nu) e += g[m] * u[m] * g[nu] * u[nu] * Tk[m * 4 + nu];
  *eps = e;
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* context creation                                                           */
/* ------------------------------------------------------------------------ */
int or_create(const or_params* P, or_ctx** out) {
  if (!P || !out) return OR_ERR_ARG;
  if (P->n_xi < 1 || P->n_xi > OR_MAXN || P->n_theta < 1 || P->n_theta > OR_MAXN ||
      P->n_phi_half < 1 || 2 * P->n_phi_half > OR_MAXN || P->nx < 1 || P->ny < 1)
    return OR_ERR_ARG;
  if (P->family == 1 && P->eos_kind != 2) return OR_ERR_ARG;
  or_ctx* C = (or_ctx*)calloc(1, sizeof(or_ctx));
  if (!C) return OR_ERR_NOMEM;
  C->P = *P;
  C->nxi = P->n_xi; C->nth = P->n_theta; C->nph = 2 * P->n_phi_half;
  C->nn = C->nxi * C->nth * C->nph;
  C->zexp = (P->family == 1) ? 1.0 : P->z0;
  gauss_legendre(16, C->g16x, C->g16w);
  int rc = radial_rule(P, C->nxi, C->c, C->wxi);
  if (rc) { free(C); return rc; }
  for (int k = 0; k < C->nxi; ++k) {
    double ck = C->c[k];
    C->s[k] = (P->family == 1) ? ck : sqrt((ck - 1.0) * (ck + 1.0));
    C->ecw[k] = exp(C->zexp * ck) * C->wxi[k];
  }
  gauss_legendre(C->nth, C->mu, C->wth);
  for (int j = 0; j < C->nth; ++j) C->sth[j] = sqrt((1.0 - C->mu[j]) * (1.0 + C->mu[j]));
  for (int l = 0; l < C->nph; ++l) {
    /* phi_l = l pi / N_phi (zeros of sin(N_phi phi), Sec. 4.3) */
    C->phi[l] = l * OR_PI / P->n_phi_half;
    double cp = cos(C->phi[l]), sp = sin(C->phi[l]);
    C->cph[l] = (fabs(cp) < 1e-12) ? 0.0 : cp;
    C->sph[l] = (fabs(sp) < 1e-12) ? 0.0 : sp;
  }
  rc = build_operators(C);
  if (rc) { free(C); return rc; }
  *out = C;
  return OR_OK;
}

void or_destroy(or_ctx* C) { free(C); }

int or_num_nodes(const or_ctx* C) { return C->nn; }

int or_nodes(const or_ctx* C, double* c, double* s, double* wxi, double* ecw, double* mu,
             double* sth, double* wth, double* cph, double* sph) {
  for (int k = 0; k < C->nxi; ++k) { c[k] = C->c[k]; s[k] = C->s[k]; wxi[k] = C->wxi[k]; ecw[k] = C->ecw[k]; }
  for (int j = 0; j < C->nth; ++j) { mu[j] = C->mu[j]; sth[j] = C->sth[j]; wth[j] = C->wth[j]; }
  for (int l = 0; l < C->nph; ++l) { cph[l] = C->cph[l]; sph[l] = C->sph[l]; }
  return OR_OK;
}

int or_operators(const or_ctx* C, double* Dr, double* Dth) {
  memcpy(Dr, C->Dr, sizeof(double) * C->nxi * C->nxi);
  memcpy(Dth, C->Dth, sizeof(double) * C->nth * C->nth);
  return OR_OK;
}

/* out: x, M, s, s', p_kin, e(=eps-B), e', B', D, J, tauR[fm], p, B, eps, K1, K2 */
int or_eos(const or_ctx* C, real_t T, real_t* out) {
  eos_pt e;
  eos_eval(&C->P, T, 2.0, &e);
  real_t p = p_of_T(C, T, &e);
  real_t K[4] = {0, 0, 0, 0};
  if (C->P.eos_kind != 2) bessel_k0123(e.x, K);
  real_t v[16] = {e.x, e.M, e.s, e.sp, e.pkin, e.e, e.ep, e.Bp, e.D, e.J, e.tauR, p,
                  B_of_T(C, T, &e), T * e.s - p, K[1], K[2]};
  memcpy(out, v, sizeof(v));
  return OR_OK;
}

int or_solve_T(const or_ctx* C, real_t target, int which, real_t* T) {
  return solve_T(C, target, which, 0.3, T, NULL);
}

int or_landau(const real_t* Tk, real_t* u, real_t* eps) { return landau(Tk, u, eps); }

int or_bessel(real_t x, real_t* K) { bessel_k0123(x, K); return OR_OK; }

/* ------------------------------------------------------------------------ */
/* one stage of the right-hand side at one site                               */
/* ------------------------------------------------------------------------ */
typedef const real_t* (*or_getf)(void* ud, int site);
typedef real_t (*or_getm)(void* ud, int site);

typedef struct {
  real_t T, u[4], eps_kin, M, Meq, D, tauR, K, B;
} or_site;

static int site_index(const or_params* P, int x, int y) {
  x %= P->nx; if (x < 0) x += P->nx;
  y %= P->ny; if (y < 0) y += P->ny;
  return y * P->nx + x;
}

/* matching of one site's populations: T^{mu nu}_kin = M^4/(2 pi^2) sum_n w_n
 * f_n P^_n P^_n (Eq. emtnew, P^ = (cosh xi, v)), Landau u and eps_kin, then T
 * from e(T) = eps_kin and the EOS at T. */
static int match_site(const or_ctx* C, const real_t* f, real_t lnM, double T_guess, or_site* o) {
  const int Nx = C->nxi, Nt = C->nth, Np = C->nph;
  real_t Tk[16] = {0};
  real_t K = 0.0;
  for (int l = 0; l < Np; ++l)
    for (int j = 0; j < Nt; ++j)
      for (int k = 0; k < Nx; ++k) {
        int n = (l * Nt + j) * Nx + k;
        double w = C->ecw[k] * C->wth[j] / (2.0 * Np);
        double Ph[4] = {C->c[k], C->s[k] * C->sth[j] * C->cph[l], C->s[k] * C->sth[j] * C->sph[l],
                        C->s[k] * C->mu[j]};
        for (int a = 0; a < 4; ++a)
          for (int b = 0; b < 4; ++b) Tk[a * 4 + b] += w * f[n] * Ph[a] * Ph[b];
        K += w * f[n];
      }
  real_t M = R_EXP(lnM);
  real_t pref = M * M * M * M / (2.0 * OR_PI * OR_PI);
  for (int a = 0; a < 16; ++a) Tk[a] *= pref;
  o->K = K * pref;
  o->M = M;
  int rc = landau(Tk, o->u, &o->eps_kin);
  if (rc) return rc;
  if (!(RE(o->eps_kin) > 0.0)) return OR_ERR_NUMERIC;
  eos_pt e;
  rc = solve_T(C, o->eps_kin, 0, T_guess, &o->T, &e);
  if (rc) return rc;
  o->Meq = e.M;
  o->D = e.D;
  o->tauR = e.tauR;
  o->B = B_of_T(C, o->T, &e);
  return OR_OK;
}

/* RHS of the kinetic equation at fixed v = p~/M for every node of one site:
 *   rhs = -V.grad f + (1/tau) S1 f + g S2 f + T_M f_eq - (P.U/E)(f - f_eq)/tau_R
 * with S1 = mu^2 Dr + Dth (Milne term of Eq. newBeq; absent in Minkowski),
 * S2 = Dr, g = d ln M / d tau from the consistency condition (Eq. masschange).
 * T_M collects the transverse mass-gradient terms at fixed v, a = grad ln M:
 *   (a.v/cosh xi) v.d_v      nodes move with the local mass,
 *   (a/cosh xi).d_v          the force 1/2 d_i M^2 d^i_(p) of Eq. Bmilne,
 * applied to the local equilibrium f_eq, whose v-derivative is known in closed
 * form (a spectral v-derivative of f itself gives a discrete operator with
 * eigenvalues of positive real part ~ 9 |a|).  Streaming is second-order upwind
 * per axis, periodic.  `o` is the site's matching.  work: 3 nn doubles. */
static int stage_site(const or_ctx* C, or_getf gf, or_getm gm, void* ud, int site,
                      double tau, const or_site* os, real_t* rhs, real_t* g_out, real_t* work) {
  const or_params* P = &C->P;
  const int Nx = C->nxi, Nt = C->nth, Np = C->nph, nn = C->nn;
  const int x = site % P->nx, y = site / P->nx;
  const real_t* f = gf(ud, site);
  const or_site o = *os;
  const real_t M = o.M, T = o.T, invT = 1.0 / T;
  const real_t inv_tauR = isinf(RE(o.tauR)) ? 0.0 : 1.0 / o.tauR;
  const real_t ut = o.u[0], ux = o.u[1], uy = o.u[2], uz = o.u[3];
  const real_t* fxm1 = gf(ud, site_index(P, x - 1, y));
  const real_t* fxm2 = gf(ud, site_index(P, x - 2, y));
  const real_t* fxp1 = gf(ud, site_index(P, x + 1, y));
  const real_t* fxp2 = gf(ud, site_index(P, x + 2, y));
  const real_t* fym1 = gf(ud, site_index(P, x, y - 1));
  const real_t* fym2 = gf(ud, site_index(P, x, y - 2));
  const real_t* fyp1 = gf(ud, site_index(P, x, y + 1));
  const real_t* fyp2 = gf(ud, site_index(P, x, y + 2));
  const real_t ax = (gm(ud, site_index(P, x + 1, y)) - gm(ud, site_index(P, x - 1, y))) / (2.0 * P->dx);
  const real_t ay = (gm(ud, site_index(P, x, y + 1)) - gm(ud, site_index(P, x, y - 1))) / (2.0 * P->dx);
  real_t* Drf = work;
  real_t* Dthf = work + nn;
  real_t* R = work + 2 * nn;
  for (int l = 0; l < Np; ++l)
    for (int j = 0; j < Nt; ++j)
      for (int k = 0; k < Nx; ++k) {
        int n = (l * Nt + j) * Nx + k;
        real_t a = 0.0, b = 0.0;
        for (int q = 0; q < Nx; ++q) a += C->Dr[k * Nx + q] * f[(l * Nt + j) * Nx + q];
        for (int q = 0; q < Nt; ++q) b += C->Dth[j * Nt + q] * f[(l * Nt + q) * Nx + k];
        Drf[n] = a; Dthf[n] = b;
      }
  real_t K = 0.0, E = 0.0, Q = 0.0, A = 0.0;
  for (int l = 0; l < Np; ++l)
    for (int j = 0; j < Nt; ++j)
      for (int k = 0; k < Nx; ++k) {
        int n = (l * Nt + j) * Nx + k;
        const double c = C->c[k], s = C->s[k], st = C->sth[j], mu = C->mu[j];
        const double vx = s * st * C->cph[l], vy = s * st * C->sph[l], vz = s * mu;
        const double Vx = vx / c, Vy = vy / c;
        real_t dfx = 0.0, dfy = 0.0;
        if (Vx > 0) dfx = (3.0 * f[n] - 4.0 * fxm1[n] + fxm2[n]) / (2.0 * P->dx);
        else if (Vx < 0) dfx = (-3.0 * f[n] + 4.0 * fxp1[n] - fxp2[n]) / (2.0 * P->dx);
        if (Vy > 0) dfy = (3.0 * f[n] - 4.0 * fym1[n] + fym2[n]) / (2.0 * P->dx);
        else if (Vy < 0) dfy = (-3.0 * f[n] + 4.0 * fyp1[n] - fyp2[n]) / (2.0 * P->dx);
        const real_t stream = -Vx * dfx - Vy * dfy;
        const real_t milne = P->metric ? (mu * mu * Drf[n] + Dthf[n]) / tau : 0.0;
        const real_t Eeq = R_SQRT(o.Meq * o.Meq + M * M * s * s);
        const real_t PeqU = ut * Eeq - M * (vx * ux + vy * uy + vz * uz);
        const real_t feq = P->Z * R_EXP(-PeqU * invT);
        /* d_v f_eq = -(f_eq/T) (u^tau M^2 v/E_eq - M u): node motion (a.v/c) v.d_v and
         * force (a/c).d_v applied to it */
        const real_t av = ax * vx + ay * vy;
        const real_t vu3 = vx * ux + vy * uy + vz * uz;
        const real_t TM = -feq * invT * ((av / c) * (ut * M * M * s * s / Eeq - M * vu3) +
                                         (ut * M * M * av / Eeq - M * (ax * ux + ay * uy)) / c);
        const real_t pu = c * ut - (vx * ux + vy * uy + vz * uz);
        const real_t coll = -(pu / c) * (f[n] - feq) * inv_tauR;
        R[n] = stream + milne + TM + coll;
        const double w = C->ecw[k] * C->wth[j] / (2.0 * Np);
        K += w * f[n];
        E += w * pu * pu * f[n];
        Q += w * pu * pu * Drf[n];
        A += w * pu * pu * R[n];
      }
  /* d ln M/d tau from d_tau B = -K d_tau ln M (Eq. masschange) with
   * d_tau B = (dB/deps) d_tau eps and d_tau eps = u_mu u_nu d_tau T^{mu nu}
   * (the M^4/(2 pi^2) prefactor cancels).  At u = (1,0) this is the paper's
   * predictor -(dB/deps) sum w cosh^2 R / sum w f, because the discrete
   * integration by parts gives 4 E + Q = K exactly there. */
  const real_t D = o.D;
  const real_t g = -D * A / (K + D * (4.0 * E + Q - K));
  for (int n = 0; n < nn; ++n) rhs[n] = R[n] + g * Drf[n];
  *g_out = g;
  if (!isfinite(RE(g))) return OR_ERR_NUMERIC;
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* full-grid accessors and the Heun step (Sec. 4.4 predictor / trapezoid)     */
/* ------------------------------------------------------------------------ */
typedef struct { const real_t* f; const real_t* lnM; int nn; } or_grid;
static const real_t* grid_f(void* ud, int site) {
  or_grid* G = (or_grid*)ud; return G->f + (size_t)site * G->nn;
}
static real_t grid_m(void* ud, int site) { return ((or_grid*)ud)->lnM[site]; }

/* One stage on the whole grid: match every site, then evaluate the RHS. */
static int stage_grid(const or_ctx* C, const real_t* fin, const real_t* lnMin, double tau,
                      real_t* rhs, real_t* g, double* Tcache, int nthreads) {
  const int ns = C->P.nx * C->P.ny, nn = C->nn;
  or_site* S = (or_site*)malloc(sizeof(or_site) * ns);
  if (!S) return OR_ERR_NOMEM;
  or_grid G = {fin, lnMin, nn};
  int err = OR_OK;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads > 0 ? nthreads : 1) schedule(static)
#endif
  for (int i = 0; i < ns; ++i) {
    int rc = match_site(C, fin + (size_t)i * nn, lnMin[i], Tcache[i], &S[i]);
    if (rc) {
#ifdef _OPENMP
#pragma omp critical(or_err)
#endif
      err = rc;
    } else {
      Tcache[i] = RE(S[i].T);
    }
  }
  if (err) { free(S); return err; }
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
#endif
  {
    real_t* work = (real_t*)malloc(sizeof(real_t) * 3 * nn);
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
    for (int i = 0; i < ns; ++i) {
      int rc = work ? stage_site(C, grid_f, grid_m, &G, i, tau, &S[i], rhs + (size_t)i * nn,
                                 g + i, work)
                    : OR_ERR_NOMEM;
      if (rc) {
#ifdef _OPENMP
#pragma omp critical(or_err)
#endif
        err = rc;
      }
    }
    free(work);
  }
  free(S);
  return err;
}

int or_step(const or_ctx* C, real_t* f, real_t* lnM, double tau, double dtau, int nsteps,
            int nthreads) {
  const int ns = C->P.nx * C->P.ny, nn = C->nn;
  const size_t tot = (size_t)ns * nn;
  real_t* fs = (real_t*)malloc(sizeof(real_t) * tot);
  real_t* rhs = (real_t*)malloc(sizeof(real_t) * tot);
  real_t* lnMs = (real_t*)malloc(sizeof(real_t) * ns);
  real_t* g = (real_t*)malloc(sizeof(real_t) * ns);
  double* Tc = (double*)malloc(sizeof(double) * ns);
  int rc = OR_OK;
  if (!fs || !rhs || !lnMs || !g || !Tc) rc = OR_ERR_NOMEM;
  for (int i = 0; i < ns && !rc; ++i) Tc[i] = 0.3;
  for (int st = 0; st < nsteps && !rc; ++st) {
    double t = tau + st * dtau;
    rc = stage_grid(C, f, lnM, t, rhs, g, Tc, nthreads);
    if (rc) break;
    for (size_t q = 0; q < tot; ++q) fs[q] = f[q] + dtau * rhs[q];
    for (int i = 0; i < ns; ++i) lnMs[i] = lnM[i] + dtau * g[i];
    rc = stage_grid(C, fs, lnMs, t + dtau, rhs, g, Tc, nthreads);
    if (rc) break;
    for (size_t q = 0; q < tot; ++q) f[q] = 0.5 * (f[q] + fs[q] + dtau * rhs[q]);
    for (int i = 0; i < ns; ++i) lnM[i] = 0.5 * (lnM[i] + lnMs[i] + dtau * g[i]);
  }
  free(fs); free(rhs); free(lnMs); free(g); free(Tc);
  return rc;
}

/* the stage right-hand side of the whole grid (for tests) */
int or_rhs(const or_ctx* C, const real_t* f, const real_t* lnM, double tau, real_t* rhs, real_t* g,
           int nthreads) {
  const int ns = C->P.nx * C->P.ny;
  double* Tc = (double*)malloc(sizeof(double) * ns);
  if (!Tc) return OR_ERR_NOMEM;
  for (int i = 0; i < ns; ++i) Tc[i] = 0.3;
  int rc = stage_grid(C, f, lnM, tau, rhs, g, Tc, nthreads);
  free(Tc);
  return rc;
}

/* per site: eps [GeV/fm^3], T [GeV], u^tau, u^x, u^y, M [GeV], P_L [GeV/fm^3], M(T) [GeV] */
int or_moments(const or_ctx* C, const real_t* f, const real_t* lnM, real_t* out, int nthreads) {
  const int ns = C->P.nx * C->P.ny, nn = C->nn;
  const double h3 = OR_HBARC * OR_HBARC * OR_HBARC;
  int err = OR_OK;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads > 0 ? nthreads : 1) schedule(static)
#endif
  for (int i = 0; i < ns; ++i) {
    or_site o;
    const real_t* fi = f + (size_t)i * nn;
    int rc = match_site(C, fi, lnM[i], 0.3, &o);
    if (rc) {
#ifdef _OPENMP
#pragma omp critical(or_err2)
#endif
      err = rc;
      continue;
    }
    /* kinetic zz component for the longitudinal pressure */
    real_t Tzz = 0.0;
    for (int l = 0; l < C->nph; ++l)
      for (int j = 0; j < C->nth; ++j)
        for (int k = 0; k < C->nxi; ++k) {
          double w = C->ecw[k] * C->wth[j] / (2.0 * C->nph);
          double vz = C->s[k] * C->mu[j];
          Tzz += w * fi[(l * C->nth + j) * C->nxi + k] * vz * vz;
        }
    Tzz *= R_POW(o.M, 4) / (2.0 * OR_PI * OR_PI);
    real_t* r = out + (size_t)i * 8;
    r[0] = (o.eps_kin + o.B) / h3;
    r[1] = o.T;
    r[2] = o.u[0]; r[3] = o.u[1]; r[4] = o.u[2];
    r[5] = o.M;
    r[6] = (Tzz - o.B) / h3;
    r[7] = o.Meq;
  }
  return err;
}

/* Observables of the whole grid.  The paper defines none; these are the
 * usual heavy-ion ones, built from the paper's moments (Eq. emtnew) and its
 * momentum weights (Sec. 4.3):
 *   eps_p = sum_x (T^xx - T^yy) / sum_x (T^xx + T^yy),
 *           T^{mu nu} = T_kin^{mu nu} + B(T) g^{mu nu}  (g^xx = g^yy = -1),
 *   v2    = sum_{x,n} W_n p_perp,n cos(2 phi_n) f_n / sum_{x,n} W_n p_perp,n f_n,
 *           W_n = M^2 w_n / (2 pi^2),  p_perp,n = M sinh xi_k sin theta_j.
 * B(T) comes from matching each site.  out[0] = eps_p, out[1] = v2.  The sums
 * over sites run in site order. */
int or_observables(const or_ctx* C, const real_t* f, const real_t* lnM, real_t* out, int nthreads) {
  const int ns = C->P.nx * C->P.ny, nn = C->nn;
  real_t* part = (real_t*)malloc(sizeof(real_t) * 4 * (size_t)ns);
  if (!part) return OR_ERR_NUMERIC;
  int err = OR_OK;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads > 0 ? nthreads : 1) schedule(static)
#endif
  for (int i = 0; i < ns; ++i) {
    or_site o;
    const real_t* fi = f + (size_t)i * nn;
    int rc = match_site(C, fi, lnM[i], 0.3, &o);
    if (rc) {
#ifdef _OPENMP
#pragma omp critical(or_err3)
#endif
      err = rc;
      continue;
    }
    real_t txx = 0.0, tyy = 0.0, num = 0.0, den = 0.0;
    for (int l = 0; l < C->nph; ++l)
      for (int j = 0; j < C->nth; ++j)
        for (int k = 0; k < C->nxi; ++k) {
          const double w = C->ecw[k] * C->wth[j] / (2.0 * C->nph);
          const real_t fn = fi[(l * C->nth + j) * C->nxi + k];
          const double vx = C->s[k] * C->sth[j] * C->cph[l], vy = C->s[k] * C->sth[j] * C->sph[l];
          const double vperp = C->s[k] * C->sth[j];
          const double cos2phi = C->cph[l] * C->cph[l] - C->sph[l] * C->sph[l];
          txx += w * fn * vx * vx;
          tyy += w * fn * vy * vy;
          num += w * fn * vperp * cos2phi;
          den += w * fn * vperp;
        }
    const real_t M = o.M, m4 = M * M * M * M / (2.0 * OR_PI * OR_PI), m3 = M * M * M / (2.0 * OR_PI * OR_PI);
    part[4 * (size_t)i + 0] = m4 * txx - o.B;
    part[4 * (size_t)i + 1] = m4 * tyy - o.B;
    part[4 * (size_t)i + 2] = m3 * num;
    part[4 * (size_t)i + 3] = m3 * den;
  }
  real_t sxx = 0.0, syy = 0.0, sn = 0.0, sd = 0.0;
  for (int i = 0; i < ns; ++i) {
    sxx += part[4 * (size_t)i + 0];
    syy += part[4 * (size_t)i + 1];
    sn += part[4 * (size_t)i + 2];
    sd += part[4 * (size_t)i + 3];
  }
  free(part);
  out[0] = (sxx - syy) / (sxx + syy);
  out[1] = sn / sd;
  return err;
}

/* initial state: T from eps_EOS(T) = eps0, M = M(T), u = 0, f = f_eq */
int or_init_state(const or_ctx* C, const real_t* eps0, real_t* f, real_t* lnM, int nthreads) {
  const int ns = C->P.nx * C->P.ny, nn = C->nn;
  const double h3 = OR_HBARC * OR_HBARC * OR_HBARC;
  int err = OR_OK;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads > 0 ? nthreads : 1) schedule(static)
#endif
  for (int i = 0; i < ns; ++i) {
    real_t T;
    eos_pt e;
    int rc = solve_T(C, eps0[i] * h3, 1, 0.3, &T, &e);
    if (rc) {
#ifdef _OPENMP
#pragma omp critical(or_err3)
#endif
      err = rc;
      continue;
    }
    real_t M = (C->P.family == 1) ? C->P.T0 : e.M;
    lnM[i] = R_LOG(M);
    for (int l = 0; l < C->nph; ++l)
      for (int j = 0; j < C->nth; ++j)
        for (int k = 0; k < C->nxi; ++k) {
          real_t Eeq = R_SQRT(e.M * e.M + M * M * C->s[k] * C->s[k]);
          f[(size_t)i * nn + (l * C->nth + j) * C->nxi + k] = C->P.Z * R_EXP(-Eeq / T);
        }
  }
  return err;
}

/* One Heun step evaluated only at selected sites (for sampled parity on large
 * grids).  The corrector at site s reads predictor populations and ln M at s,
 * s+-1, s+-2 along x and y; the predictor at those sites reads the input at
 * their own +-2 neighbours. */
typedef struct {
  const or_ctx* C; const real_t* f; const real_t* lnM;
  int np; const int* pid; const real_t* fs; const real_t* lnMs; /* predictor patch */
  int use_patch;
} or_patch;
static const real_t* patch_f(void* ud, int site) {
  or_patch* G = (or_patch*)ud;
  if (!G->use_patch) return G->f + (size_t)site * G->C->nn;
  for (int q = 0; q < G->np; ++q)
    if (G->pid[q] == site) return G->fs + (size_t)q * G->C->nn;
  return NULL;
}
static real_t patch_m(void* ud, int site) {
  or_patch* G = (or_patch*)ud;
  if (!G->use_patch) return G->lnM[site];
  for (int q = 0; q < G->np; ++q)
    if (G->pid[q] == site) return G->lnMs[q];
  return NAN;
}
int or_step_sites(const or_ctx* C, const real_t* f, const real_t* lnM, double tau, double dtau,
                  const int* sites, int nsel, real_t* f_out, real_t* lnM_out, int nthreads) {
  const or_params* P = &C->P;
  const int nn = C->nn;
  int err = OR_OK;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads > 0 ? nthreads : 1) schedule(dynamic)
#endif
  for (int q = 0; q < nsel; ++q) {
    int s0 = sites[q], x = s0 % P->nx, y = s0 / P->nx;
    int ids[9], np = 0;
    int offs[9][2] = {{0, 0}, {-1, 0}, {-2, 0}, {1, 0}, {2, 0}, {0, -1}, {0, -2}, {0, 1}, {0, 2}};
    for (int a = 0; a < 9; ++a) {
      int id = site_index(P, x + offs[a][0], y + offs[a][1]), dup = 0;
      for (int b = 0; b < np; ++b) dup |= (ids[b] == id);
      if (!dup) ids[np++] = id;
    }
    real_t* fs = (real_t*)malloc(sizeof(real_t) * (size_t)nn * (9 + 4));
    real_t lnMs[9], g;
    int rc = fs ? OR_OK : OR_ERR_NOMEM;
    real_t* rhs = fs + (size_t)9 * nn;
    real_t* work = rhs + nn;
    or_patch G;
    memset(&G, 0, sizeof G);
    G.C = C; G.f = f; G.lnM = lnM;
    for (int a = 0; a < np && !rc; ++a) {
      or_site o;
      rc = match_site(C, f + (size_t)ids[a] * nn, lnM[ids[a]], 0.3, &o);
      if (!rc) rc = stage_site(C, patch_f, patch_m, &G, ids[a], tau, &o, rhs, &g, work);
      for (int n = 0; n < nn && !rc; ++n) fs[(size_t)a * nn + n] = f[(size_t)ids[a] * nn + n] + dtau * rhs[n];
      lnMs[a] = lnM[ids[a]] + dtau * g;
    }
    if (!rc) {
      or_patch H;
      memset(&H, 0, sizeof H);
      H.C = C; H.f = f; H.lnM = lnM; H.np = np; H.pid = ids; H.fs = fs; H.lnMs = lnMs; H.use_patch = 1;
      or_site o;
      rc = match_site(C, fs, lnMs[0], 0.3, &o);
      if (!rc) rc = stage_site(C, patch_f, patch_m, &H, s0, tau + dtau, &o, rhs, &g, work);
      for (int n = 0; n < nn && !rc; ++n)
        f_out[(size_t)q * nn + n] = 0.5 * (f[(size_t)s0 * nn + n] + fs[n] + dtau * rhs[n]);
      lnM_out[q] = 0.5 * (lnM[s0] + lnMs[0] + dtau * g);
    }
    free(fs);
    if (rc) {
#ifdef _OPENMP
#pragma omp critical(or_err4)
#endif
      err = rc;
    }
  }
  return err;
}
