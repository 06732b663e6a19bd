// rlb_kernels.cuh -- GB300 (sm_103a) kernels of the relativistic lattice
// Boltzmann step with a quasiparticle equation of state (Romatschke,
// arXiv:1108.5561, Sec. 3-4).
//
// Thread mapping: one CTA per lattice site, one thread per "xi-line" (the
// n_xi radial nodes at fixed polar index j and azimuth l, contiguous in
// memory), so a warp's loads of a site are contiguous and vectorised.  The
// site's populations are staged in shared memory for the polar (theta-line)
// operator; the per-site FP64 Landau matching and EOS inversion run on lane 0
// of warp 0 while the other warps apply the polar operator.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include <type_traits>

namespace rlbk {

enum : int { ERR_LANDAU = 1, ERR_EOS = 2, ERR_NONFINITE = 4, ERR_INDEX = 8 };

// Debug builds (-DRLB_CHECKS, the library built with checks=True): every site
// index and grid coordinate a kernel derives is checked against its range; a
// failure sets ERR_INDEX in the error word and the value is replaced by 0 (a
// valid index), so that no access leaves its array and no thread leaves the
// CTA's barrier sequence.  Release builds return the value unchanged.
__device__ __forceinline__ int idx_checked(int v, int n, int* err) {
#ifdef RLB_CHECKS
  if (v < 0 || v >= n) {
    atomicOr(err, (int)ERR_INDEX);
    return 0;
  }
#else
  (void)n;
  (void)err;
#endif
  return v;
}
// ln M of f_in at `site` into dst[0] and, in the corrector (mode 1), ln M of
// f_base into dst[2] (dst in shared memory, 8-byte aligned), by cp.async: the
// thread that updates ln M after the site's reductions then reads shared
// memory instead of waiting there for a global load.  The reader calls
// lnm_wait() first.
__device__ __forceinline__ void lnm_fetch(double* dst, const double* lnM_in, const double* lnM_base, int site,
                                          int mode) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(lnM_in + site) : "memory");
  if (mode == 1) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d + 16), "l"(lnM_base + site) : "memory");
}
__device__ __forceinline__ void lnm_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Debug builds: ERR_NONFINITE when one of the n values is not finite.
template <class R>
__device__ __forceinline__ void finite_checked(const R* v, int n, int* err) {
#ifdef RLB_CHECKS
  bool ok = true;
  for (int i = 0; i < n; ++i) ok = ok && isfinite((double)v[i]);
  if (!ok) atomicOr(err, (int)ERR_NONFINITE);
#else
  (void)v;
  (void)n;
  (void)err;
#endif
}

// ---------------------------------------------------------------------------
// per-run constants, passed by value (kernel parameter space = constant bank)
// ---------------------------------------------------------------------------
template <class R, int NXI, int NTH, int NPH>
struct Ops {
  R Dr[NXI * NXI];    // Galerkin v.d/dv (radial part of S1, S2)
  R Dth[NTH * NTH];   // Galerkin (mu - mu^3) d/dmu (polar part of S1)
  // radial node constants
  R c[NXI], s[NXI], s2[NXI], inv_c[NXI], tv[NXI];  // cosh, sinh, sinh^2, 1/cosh, tanh
  R q1[NXI], q2[NXI];  // sinh (sinh^2 + 1)/cosh, sinh^2/cosh
  R w0[NXI], w1[NXI], w2[NXI], w3[NXI];  // ecw * {1, c s, c^2, s^2}
  R ecw[NXI];
  // polar
  R mu[NTH], mu2[NTH], sth[NTH], sth_mu[NTH], wj[NTH];  // wj = w^th_j / (2 NPH)
  // azimuth
  R cph[NPH], sph[NPH];
};

struct EosView {
  const double* tab;   // n x 8 doubles, uniform in y = ln T
  const float* tabf;   // the same table rounded to FP32
  double y0, inv_h;
  int n;
  // FP32 cell location: u = (y - y0)/h = y (ih_hi + ih_lo) - (c_hi + c_lo), with
  // c = y0/h split into an integer c_hi and a remainder, so that the offset in
  // the cell keeps FP32 relative precision (u itself reaches n ~ 6.5e4)
  float ih_hi, ih_lo, c_hi, c_lo;
  // the interior of the table in FP32: [y0 + 2h, y0 + (n - 4)h]
  float ylo_f, yhi_f;
  // double-FP32 form of the table for the FP64-accurate EOS step of the FP32
  // path: tabf + tabl = tab to 2^-48, y0 = y0_hi + y0_lo
  const float* tabl;
  float y0_hi, y0_lo;
};


// ---------------------------------------------------------------------------
// storage <-> compute conversions
// ---------------------------------------------------------------------------
template <class S, class R> __device__ __forceinline__ R ld1(const S& v) { return (R)v; }
template <> __device__ __forceinline__ float ld1<__nv_bfloat16, float>(const __nv_bfloat16& v) {
  return __bfloat162float(v);
}
template <class S, class R> __device__ __forceinline__ S st1(R v) { return (S)v; }
template <> __device__ __forceinline__ __nv_bfloat16 st1<__nv_bfloat16, float>(float v) {
  return __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ __nv_bfloat16 st1<__nv_bfloat16, double>(double v) {
  return __double2bfloat16(v);
}

// 8 FP32 values in one 256-bit access (p 32-byte aligned: a line of 8k FP32
// values at a multiple of 8 elements in a 256-byte aligned array; two 128-bit
// accesses make every request of the warp touch all 32 sectors of its 1 KB)
__device__ __forceinline__ void ldg8f(const float* p, float (&v)[8]) {
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
      : "l"(p));
}
__device__ __forceinline__ void stg8f(float* p, const float (&v)[8]) {
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(v[0]), "f"(v[1]),
               "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
               : "memory");
}

template <class S, class R, int N>
__device__ __forceinline__ void load_line(const S* __restrict__ p, R (&v)[N]) {
  if constexpr (std::is_same<S, float>::value && N % 8 == 0) {
#pragma unroll
    for (int i = 0; i < N / 8; ++i) {
      float a[8];
      ldg8f(p + 8 * i, a);
#pragma unroll
      for (int h = 0; h < 8; ++h) v[8 * i + h] = (R)a[h];
    }
  } else if constexpr (sizeof(S) == 4 && N % 4 == 0) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int i = 0; i < N / 4; ++i) {
      float4 a = __ldg(q + i);
      v[4 * i] = (R)a.x; v[4 * i + 1] = (R)a.y; v[4 * i + 2] = (R)a.z; v[4 * i + 3] = (R)a.w;
    }
  } else if constexpr (sizeof(S) == 8 && N % 2 == 0) {
    const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
      double2 a = __ldg(q + i);
      v[2 * i] = (R)a.x; v[2 * i + 1] = (R)a.y;
    }
  } else if constexpr (sizeof(S) == 2 && N % 8 == 0) {
    const uint4* q = reinterpret_cast<const uint4*>(p);
#pragma unroll
    for (int i = 0; i < N / 8; ++i) {
      uint4 a = __ldg(q + i);
      const __nv_bfloat162* b = reinterpret_cast<const __nv_bfloat162*>(&a);
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        float2 t = __bfloat1622float2(b[h]);
        v[8 * i + 2 * h] = (R)t.x; v[8 * i + 2 * h + 1] = (R)t.y;
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = ld1<S, R>(p[i]);
  }
}

template <class S, class R, int N>
__device__ __forceinline__ void store_line(S* __restrict__ p, const R (&v)[N]) {
  if constexpr (std::is_same<S, float>::value && N % 8 == 0) {
#pragma unroll
    for (int i = 0; i < N / 8; ++i) {
      float a[8];
#pragma unroll
      for (int h = 0; h < 8; ++h) a[h] = (float)v[8 * i + h];
      stg8f(p + 8 * i, a);
    }
  } else if constexpr (sizeof(S) == 4 && N % 4 == 0) {
    float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
    for (int i = 0; i < N / 4; ++i)
      q[i] = make_float4((float)v[4 * i], (float)v[4 * i + 1], (float)v[4 * i + 2], (float)v[4 * i + 3]);
  } else if constexpr (sizeof(S) == 8 && N % 2 == 0) {
    double2* q = reinterpret_cast<double2*>(p);
#pragma unroll
    for (int i = 0; i < N / 2; ++i) q[i] = make_double2((double)v[2 * i], (double)v[2 * i + 1]);
  } else if constexpr (sizeof(S) == 2 && N % 8 == 0) {
    uint4* q = reinterpret_cast<uint4*>(p);
#pragma unroll
    for (int i = 0; i < N / 8; ++i) {
      uint4 a;
      __nv_bfloat162* b = reinterpret_cast<__nv_bfloat162*>(&a);
#pragma unroll
      for (int h = 0; h < 4; ++h)
        b[h] = __floats2bfloat162_rn((float)v[8 * i + 2 * h], (float)v[8 * i + 2 * h + 1]);
      q[i] = a;
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) p[i] = st1<S, R>(v[i]);
  }
}

template <class R> __device__ __forceinline__ R fexp(R x);
template <> __device__ __forceinline__ float fexp<float>(float x) { return __expf(x); }
template <> __device__ __forceinline__ double fexp<double>(double x) { return exp(x); }
__device__ __forceinline__ float ex2_ftz(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
template <class R> __device__ __forceinline__ R fsqrt(R x);
template <> __device__ __forceinline__ float fsqrt<float>(float x) { return sqrtf(x); }
template <> __device__ __forceinline__ double fsqrt<double>(double x) { return sqrt(x); }

// ---------------------------------------------------------------------------
// EOS table: 6-point Lagrange interpolation in y = ln T (node offsets -2..3).
// Fields (8 doubles per node): 0 e(T) = eps - B [GeV^4], 1 M(T)/T, 2 dB/deps,
// 3 1/h with tau_R = (eta/s) h [1/fm], 4 B/T^4, 5 eps(T) [GeV^4].
// ---------------------------------------------------------------------------
enum : int { EOS_E = 0, EOS_X = 1, EOS_D = 2, EOS_INVH = 3, EOS_B = 4, EOS_EPS = 5 };

__device__ __forceinline__ void lagrange6(double t, double w[6]) {
  const double a = t + 2.0, b = t + 1.0, c = t, d = t - 1.0, e = t - 2.0, f = t - 3.0;
  const double ab = a * b, de = d * e, ef = e * f, cd = c * d;
  w[0] = b * cd * ef * (-1.0 / 120.0);
  w[1] = a * cd * ef * (1.0 / 24.0);
  w[2] = ab * de * f * (-1.0 / 12.0);
  w[3] = ab * c * ef * (1.0 / 12.0);
  w[4] = ab * cd * f * (-1.0 / 24.0);
  w[5] = ab * cd * e * (1.0 / 120.0);
}

// derivative of the six weights with respect to t
__device__ __forceinline__ void lagrange6_d(double t, double dw[6]) {
  const double fac[6] = {t + 2.0, t + 1.0, t, t - 1.0, t - 2.0, t - 3.0};
  const double inv[6] = {-1.0 / 120.0, 1.0 / 24.0, -1.0 / 12.0, 1.0 / 12.0, -1.0 / 24.0, 1.0 / 120.0};
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    double prod = 1.0, dprod = 0.0;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      if (q == m) continue;
      dprod = dprod * fac[q] + prod;
      prod *= fac[q];
    }
    dw[m] = dprod * inv[m];
  }
}

// Locate y; returns false when y lies outside the tabulated range.
__device__ __forceinline__ bool eos_cell(const EosView& E, double y, int* i0, double* t) {
  double u = (y - E.y0) * E.inv_h;
  if (!(u >= 2.0 && u <= (double)(E.n - 4))) return false;
  int i = (int)floor(u);
  if (i > E.n - 4) i = E.n - 4;
  *i0 = i;
  *t = u - i;
  return true;
}

__device__ __forceinline__ double eos_field(const EosView& E, int i0, const double w[6], int field) {
  double v = 0.0;
#pragma unroll
  for (int m = 0; m < 6; ++m) v += w[m] * __ldg(E.tab + (size_t)(i0 - 2 + m) * 8 + field);
  return v;
}

// Solve table field `field`(y) = target for y (the field increases with y) by
// Newton on the interpolant, safeguarded by a bisection bracket that starts as
// the whole tabulated range; a target outside the range is reported as failure.
__device__ bool eos_invert(const EosView& E, int field, double target, double y, double* y_out) {
  double lo = E.y0 + 2.0 / E.inv_h, hi = E.y0 + (E.n - 4) / E.inv_h;
  const double ymin = lo, ymax = hi;
  if (!(y > lo && y < hi)) y = 0.5 * (lo + hi);
  int settled = 0;
  for (int it = 0; it < 200; ++it) {
    int i0;
    double t, w[6], dw[6];
    if (!eos_cell(E, y, &i0, &t)) return false;
    lagrange6(t, w);
    lagrange6_d(t, dw);
    double F = 0.0, dF = 0.0;
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      double v = __ldg(E.tab + (size_t)(i0 - 2 + m) * 8 + field);
      F += w[m] * v;
      dF += dw[m] * v;
    }
    dF *= E.inv_h;
    if (F == target) { *y_out = y; return true; }
    if (F < target) lo = y; else hi = y;
    double yn = (dF > 0.0) ? y - (F - target) / dF : 0.5 * (lo + hi);
    if (!(yn >= lo && yn <= hi)) yn = 0.5 * (lo + hi);
    const double dy = yn - y;
    y = yn;
    if (fabs(dy) < 1e-13 || hi - lo < 1e-14) {
      if (++settled == 2) {
        // a target beyond the table drives the bracket onto one of its ends
        if (y - ymin < 1e-12 || ymax - y < 1e-12) return false;
        *y_out = y;
        return true;
      }
    } else {
      settled = 0;
    }
  }
  return false;
}

// FP32 versions for the FP32-arithmetic kernels (start values and the fields
// that feed FP32 arithmetic).
__device__ __forceinline__ void lagrange6f(float t, float w[6]) {
  const float a = t + 2.f, b = t + 1.f, c = t, d = t - 1.f, e = t - 2.f, f = t - 3.f;
  const float ab = a * b, de = d * e, ef = e * f, cd = c * d;
  w[0] = b * cd * ef * (-1.f / 120.f);
  w[1] = a * cd * ef * (1.f / 24.f);
  w[2] = ab * de * f * (-1.f / 12.f);
  w[3] = ab * c * ef * (1.f / 12.f);
  w[4] = ab * cd * f * (-1.f / 24.f);
  w[5] = ab * cd * e * (1.f / 120.f);
}
__device__ __forceinline__ void lagrange6f_d(float t, float dw[6]) {
  const float fac[6] = {t + 2.f, t + 1.f, t, t - 1.f, t - 2.f, t - 3.f};
  const float inv[6] = {-1.f / 120.f, 1.f / 24.f, -1.f / 12.f, 1.f / 12.f, -1.f / 24.f, 1.f / 120.f};
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    float prod = 1.f, dprod = 0.f;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      if (q == m) continue;
      dprod = dprod * fac[q] + prod;
      prod *= fac[q];
    }
    dw[m] = dprod * inv[m];
  }
}
__device__ __forceinline__ float eos_fieldf(const EosView& E, int i0, const float w[6], int field) {
  float v = 0.f;
#pragma unroll
  for (int m = 0; m < 6; ++m) v += w[m] * __ldg(E.tabf + (size_t)(i0 - 2 + m) * 8 + field);
  return v;
}

// FP32 cell location of y: i0 (clamped to the interior) and the offset t in the
// cell; false outside the tabulated range.
__device__ __forceinline__ bool eos_cellf(const EosView& E, float y, int* i0, float* t) {
  const float u = fmaf(y, E.ih_hi, -E.c_hi);
  if (!(u >= 2.f && u <= (float)(E.n - 4))) return false;
  const int i = min((int)floorf(u), E.n - 4);
  *i0 = i;
  *t = fmaf(y, E.ih_hi, -(E.c_hi + (float)i)) + fmaf(y, E.ih_lo, -E.c_lo);
  return true;
}

// Table inversion in FP32 (FP32 storage path): Newton on the interpolant of the
// FP32 table, safeguarded by a bisection bracket; same failure rules as
// eos_invert.  It stops once a step is below kEosStopF in y = ln T: the error
// left is about C dy^2 with C = e''/(2 e') (2 for e ~ T^4; at most 7.9 for the
// crossover EOS, at T = 0.145 GeV), at most 2e-6, which the one Newton step
// of eos_refine_df that follows takes to C (2e-6)^2 ~ 3e-11; stopping at 2e-6
// instead cost one more table iteration per site.
constexpr float kEosStopF = 5e-4f;
__device__ bool eos_invert_f(const EosView& E, int field, float target, float y, float* y_out) {
  const float ih = E.ih_hi + E.ih_lo;
  float lo = E.ylo_f, hi = E.yhi_f;
  const float ymin = lo, ymax = hi;
  float yf = (y > ymin && y < ymax) ? y : 0.5f * (lo + hi);
  bool ok = false;
  for (int it = 0; it < 100; ++it) {
    int i0;
    float t;
    if (!eos_cellf(E, yf, &i0, &t)) return false;
    float w[6], dw[6];
    lagrange6f(t, w);
    lagrange6f_d(t, dw);
    float F = 0.f, dF = 0.f;
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      const float v = __ldg(E.tabf + (size_t)(i0 - 2 + m) * 8 + field);
      F += w[m] * v;
      dF += dw[m] * v;
    }
    dF *= ih;
    if (F == target) { ok = true; break; }
    if (F < target) lo = yf; else hi = yf;
    float yn = (dF > 0.f) ? yf - (F - target) / dF : 0.5f * (lo + hi);
    if (!(yn >= lo && yn <= hi)) yn = 0.5f * (lo + hi);
    const float dy = yn - yf;
    yf = yn;
    if (fabsf(dy) < kEosStopF || hi - lo < 4e-6f) { ok = true; break; }
  }
  if (!ok || yf - ymin < 1e-5f || ymax - yf < 1e-5f) return false;
  *y_out = yf;
  return true;
}

// a + b = s + e exactly (Knuth's TwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Double-FP32 numbers: the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi) / 2 (about 48 significant bits).  Exact sums by TwoSum,
// exact products by the fused multiply-add (the error of a * b is
// fma(a, b, -a b)); every multiply-add below is written out, so that no
// contraction can change an error term.
struct f2x {
  float hi, lo;
};
__device__ __forceinline__ f2x two_sum_f2x(float a, float b) {
  f2x r;
  two_sum(a, b, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ f2x fast_two_sum(float a, float b) {  // |a| >= |b| or a = 0
  const float s = a + b;
  return f2x{s, b - (s - a)};
}
__device__ __forceinline__ f2x two_prod(float a, float b) {
  const float p = a * b;
  return f2x{p, fmaf(a, b, -p)};
}
__device__ __forceinline__ f2x df_add(f2x a, f2x b) {
  f2x s = two_sum_f2x(a.hi, b.hi);
  s.lo += a.lo + b.lo;
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ f2x df_mul(f2x a, f2x b) {
  f2x p = two_prod(a.hi, b.hi);
  p.lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
  return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ f2x df_div(f2x a, f2x b) {  // a / b, b != 0
  const float q1 = a.hi / b.hi;
  const f2x r = df_add(a, df_mul(b, f2x{-q1, 0.f}));
  const float q2 = r.hi / b.hi;
  return fast_two_sum(q1, q2);
}

// One Newton step of e(y) = target, FP64-accurate, from an FP32 root (slope
// from the FP32 table): the EOS inversion of the FP32 storage path.  Run on
// the FP32 pipes in double-FP32 arithmetic (GB300 issues one FP64 warp
// instruction per 16 cycles per SM):
//   the offset t in the cell of the FP32 location, from y - y0 and 1/h as
//   double-FP32 numbers (t to ~1e-9 cells; the FP32 location alone is good to
//   ~4e-3 cells at u ~ 6.5e4);
//   the residual sum_m w_m (tab_m - target): sum_m w_m = 1, so the FP32
//   weights multiply the differences tab_m - target, taken exactly (Sterbenz)
//   from the double-FP32 table and target, and the sum keeps ~1e-7 of terms of
//   the size of the step, about 1e-9 in y.
// The cell comes from the FP32 location (at a cell edge the two locations may
// differ by one cell; the offset is then just outside [0, 1), where the same
// interpolating polynomial still holds to the table's accuracy).
__device__ __forceinline__ float eos_refine_df(const EosView& E, int field, f2x target, float y) {
  int i0;
  float tf;
  if (!eos_cellf(E, y, &i0, &tf)) return y;
  f2x s = two_sum_f2x(y, -E.y0_hi);
  s.lo -= E.y0_lo;
  const f2x u = df_mul(fast_two_sum(s.hi, s.lo), f2x{E.ih_hi, E.ih_lo});
  const float t = (u.hi - (float)i0) + u.lo;
  float w[6], dw[6];
  lagrange6f(t, w);
  lagrange6f_d(t, dw);
  float r = 0.f, dF = 0.f;
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    const size_t k = (size_t)(i0 - 2 + m) * 8 + field;
    const float hi = __ldg(E.tabf + k), lo = __ldg(E.tabl + k);
    const float d = (hi - target.hi) + (lo - target.lo);
    r = fmaf(w[m], d, r);
    dF = fmaf(dw[m], hi, dF);
  }
  dF *= E.ih_hi + E.ih_lo;
  if (!(dF > 0.f)) return y;
  return y - r / dF;
}


// ---------------------------------------------------------------------------
// Landau matching on the (tau, x, y) block (Eq. sanity).  Boost invariance and
// the eta_s -> -eta_s reflection of the lattice make the Y row and column of
// T^{mu nu} vanish, so the timelike eigenvector lives in this block.
// tm = {T00, T01, T02, T11, T12, T22} (upper indices, orthonormal frame).
// Largest root of the characteristic cubic of A = T g by Newton from an
// upper bound (monotone for a real-rooted cubic), eigenvector from the null
// space of A - eps (largest cross product of two rows), normalised by the
// Minkowski norm; eps is then the Rayleigh quotient u_mu u_nu T^{mu nu}.
// ---------------------------------------------------------------------------
// Version for the FP32 storage path: tm the matrix in FP32, tmd the same in
// double-FP32 (the compensated moment sums times the prefactor).  Newton from
// the infinity-norm bound in FP32 on the scaled matrix gives lambda to FP32
// precision and the eigenvector u by the cross products; the eigenvalue is
// then the generalised Rayleigh quotient eps = (w^T T w) / (w^T g w), w = g u
// (T w = lambda g w for the covariant eigenvector), evaluated in double-FP32:
// stationary at the eigenvector, its error is second order in the FP32 error
// of u (~1e-14 relative), as accurate as an FP64 Newton step on the cubic but
// on the FP32 pipes.  u is recomputed by the cross products at the refined
// eigenvalue (it is consumed in FP32).
__device__ __forceinline__ bool null_vector3(float a00, float a01, float a02, float a10, float a11, float a12,
                                             float a20, float a21, float a22, float lam, float u[3]) {
  const float r00 = a00 - lam, r11 = a11 - lam, r22 = a22 - lam;
  const float p0 = a01 * a12 - a02 * r11, p1 = a02 * a10 - r00 * a12, p2 = r00 * r11 - a01 * a10;
  const float q0 = a01 * r22 - a02 * a21, q1 = a02 * a20 - r00 * r22, q2 = r00 * a21 - a01 * a20;
  const float s0 = r11 * r22 - a12 * a21, s1 = a12 * a20 - a10 * r22, s2 = a10 * a21 - r11 * a20;
  const float np = p0 * p0 + p1 * p1 + p2 * p2, nq = q0 * q0 + q1 * q1 + q2 * q2;
  const float nsq = s0 * s0 + s1 * s1 + s2 * s2;
  float v0 = s0, v1 = s1, v2 = s2;
  if (np >= nq && np >= nsq) { v0 = p0; v1 = p1; v2 = p2; }
  else if (nq >= nsq) { v0 = q0; v1 = q1; v2 = q2; }
  const float mn = v0 * v0 - v1 * v1 - v2 * v2;
  if (!(mn > 0.f)) return false;
  float r = rsqrtf(mn);
  if (v0 < 0.f) r = -r;
  u[0] = v0 * r; u[1] = v1 * r; u[2] = v2 * r;
  return true;
}

__device__ bool landau3_df(const f2x tmd[6], const float tm[6], float u[3], f2x* eps) {
  const float sc = fmaxf(fabsf(tm[0]) + fabsf(tm[1]) + fabsf(tm[2]),
                         fmaxf(fabsf(tm[1]) + fabsf(tm[3]) + fabsf(tm[4]),
                               fabsf(tm[2]) + fabsf(tm[4]) + fabsf(tm[5])));
  if (!(sc > 0.f) || !isfinite(sc)) return false;
  const float is = 1.f / sc;
  const float a00 = tm[0] * is, a01 = -tm[1] * is, a02 = -tm[2] * is;
  const float a10 = -a01, a11 = -tm[3] * is, a12 = -tm[4] * is;
  const float a20 = -a02, a21 = a12, a22 = -tm[5] * is;
  const float c2 = a00 + a11 + a22;
  const float c1 = a00 * a11 - a01 * a10 + a00 * a22 - a02 * a20 + a11 * a22 - a12 * a21;
  const float c0 = a00 * (a11 * a22 - a12 * a21) - a01 * (a10 * a22 - a12 * a20) + a02 * (a10 * a21 - a11 * a20);
  // Newton start: an upper bound on the largest root.  The infinity norm (1
  // here) bounds every eigenvalue; closer, where T^{mu nu} satisfies the
  // energy conditions eps is the minimum of u_mu u_nu T^{mu nu} over timelike
  // unit u, so the energy in the frame moving with beta = T^{0i} / T^{00}
  // bounds it from above, with an excess second order in the difference of
  // the two velocities (a few Newton steps instead of up to a dozen for a
  // fast-moving cell).  It is taken only where the cubic places it above its
  // largest root (p >= 0, p' > 0, p'' > 0), raised by 1e-6 against rounding.
  float lam = 1.f;
  {
    const float t0 = tm[0] * is, t1 = tm[1] * is, t2 = tm[2] * is;
    const float b1 = t1 / t0, b2 = t2 / t0, bb = b1 * b1 + b2 * b2;
    if (t0 > 0.f && bb < 1.f) {
      const float e = (t0 - 2.f * (b1 * t1 + b2 * t2) + is * (b1 * b1 * tm[3] + 2.f * b1 * b2 * tm[4] + b2 * b2 * tm[5])) /
                      (1.f - bb);
      const float l0 = e * (1.f + 1e-6f);
      const float p = ((l0 - c2) * l0 + c1) * l0 - c0, dp = (3.f * l0 - 2.f * c2) * l0 + c1;
      if (l0 < 1.f && p >= 0.f && dp > 0.f && 3.f * l0 > c2) lam = l0;
    }
  }
  for (int it = 0; it < 60; ++it) {
    const float p = ((lam - c2) * lam + c1) * lam - c0;
    const float dp = (3.f * lam - 2.f * c2) * lam + c1;
    if (!(dp > 0.f)) break;
    const float d = p / dp;
    if (!(d > 0.f)) break;
    lam -= d;
    if (d <= 1e-7f * lam) break;
  }
  float v[3];
  if (!null_vector3(a00, a01, a02, a10, a11, a12, a20, a21, a22, lam, v)) return false;
  // w^T T w and w^T g w with w = (v0, -v1, -v2): the products v_i v_j exact
  const f2x v00 = two_prod(v[0], v[0]), v01 = two_prod(v[0], v[1]), v02 = two_prod(v[0], v[2]);
  const f2x v11 = two_prod(v[1], v[1]), v12 = two_prod(v[1], v[2]), v22 = two_prod(v[2], v[2]);
  const f2x m2{-2.f, 0.f}, p2{2.f, 0.f};
  f2x num = df_mul(v00, tmd[0]);
  num = df_add(num, df_mul(df_mul(m2, v01), tmd[1]));
  num = df_add(num, df_mul(df_mul(m2, v02), tmd[2]));
  num = df_add(num, df_mul(v11, tmd[3]));
  num = df_add(num, df_mul(df_mul(p2, v12), tmd[4]));
  num = df_add(num, df_mul(v22, tmd[5]));
  f2x den = df_add(v00, f2x{-v11.hi, -v11.lo});
  den = df_add(den, f2x{-v22.hi, -v22.lo});
  if (!(den.hi > 0.f)) return false;
  *eps = df_div(num, den);
  if (!(eps->hi > 0.f)) return false;
  const float lam2 = fmaf(eps->hi, is, eps->lo * is);
  return null_vector3(a00, a01, a02, a10, a11, a12, a20, a21, a22, lam2, u);
}

__device__ bool landau3(const double tm[6], double u[3], double* eps) {
  const double a00 = tm[0], a01 = -tm[1], a02 = -tm[2];
  const double a10 = tm[1], a11 = -tm[3], a12 = -tm[4];
  const double a20 = tm[2], a21 = -tm[4], a22 = -tm[5];
  const double c2 = a00 + a11 + a22;
  const double c1 = a00 * a11 - a01 * a10 + a00 * a22 - a02 * a20 + a11 * a22 - a12 * a21;
  const double c0 = a00 * (a11 * a22 - a12 * a21) - a01 * (a10 * a22 - a12 * a20) +
                    a02 * (a10 * a21 - a11 * a20);
  double lam = fmax(fabs(a00) + fabs(a01) + fabs(a02),
                    fmax(fabs(a10) + fabs(a11) + fabs(a12), fabs(a20) + fabs(a21) + fabs(a22)));
  const int iters = 200;
  for (int it = 0; it < iters; ++it) {
    double p = ((lam - c2) * lam + c1) * lam - c0;
    double dp = (3.0 * lam - 2.0 * c2) * lam + c1;
    if (!(dp > 0.0)) break;
    double d = p / dp;
    if (!(d > 0.0)) break;  // no further decrease: converged from above
    lam -= d;
    if (d <= 1e-16 * fabs(lam)) break;
  }
  // null vector of A - lam: the largest of the three row cross products
  const double r00 = a00 - lam, r11 = a11 - lam, r22 = a22 - lam;
  const double p0 = a01 * a12 - a02 * r11, p1 = a02 * a10 - r00 * a12, p2 = r00 * r11 - a01 * a10;  // r0 x r1
  const double q0 = a01 * r22 - a02 * a21, q1 = a02 * a20 - r00 * r22, q2 = r00 * a21 - a01 * a20;  // r0 x r2
  const double s0 = r11 * r22 - a12 * a21, s1 = a12 * a20 - a10 * r22, s2 = a10 * a21 - r11 * a20;  // r1 x r2
  const double np = p0 * p0 + p1 * p1 + p2 * p2, nq = q0 * q0 + q1 * q1 + q2 * q2;
  const double nsq = s0 * s0 + s1 * s1 + s2 * s2;
  double v0 = s0, v1 = s1, v2 = s2;
  if (np >= nq && np >= nsq) { v0 = p0; v1 = p1; v2 = p2; }
  else if (nq >= nsq) { v0 = q0; v1 = q1; v2 = q2; }
  double mn = v0 * v0 - v1 * v1 - v2 * v2;
  if (!(mn > 0.0)) return false;
  double r = rsqrt(mn);
  if (v0 < 0) r = -r;
  u[0] = v0 * r; u[1] = v1 * r; u[2] = v2 * r;
  *eps = u[0] * u[0] * tm[0] - 2.0 * u[0] * u[1] * tm[1] - 2.0 * u[0] * u[2] * tm[2] +
         u[1] * u[1] * tm[3] + 2.0 * u[1] * u[2] * tm[4] + u[2] * u[2] * tm[5];
  return *eps > 0.0;
}

// per-site moments (without the M^4/(2 pi^2) prefactor), 8 doubles per site:
//   K^ = sum w f, T00, T01, T02, T11, T12, T22 (sum w f P^ P^), Tzz
// FP32 storage keeps kMomParts float partial sums per moment instead
// ([site][moment][part]); the moment is their sum.
constexpr int kMom = 8;
constexpr int kMomParts = 4;

// (hi, lo) pairs of a compensated block sum -> the kMomParts layout
__device__ __forceinline__ void store_mom_parts(float* dst, const float* pairs) {
  float4* d = reinterpret_cast<float4*>(dst);
#pragma unroll
  for (int q = 0; q < kMom; ++q) d[q] = make_float4(pairs[2 * q], pairs[2 * q + 1], 0.f, 0.f);
}
// per-site matching results consumed by the stage kernel: kScUsed values,
// stored kSc apart (64 bytes in FP32: four 16-byte loads per site; the two
// padding slots hold zeros)
constexpr int kScUsed = 15, kSc = 16;
enum : int {
  SC_UT = 0, SC_UX, SC_UY, SC_INVT, SC_MEQ, SC_M, SC_ITR, SC_D, SC_B, SC_K, SC_KH, SC_T,
  SC_AX, SC_AY,  // grad ln M (central differences, 1/fm)
  SC_L2T         // log2(e) / T, one rounding from the product (the exponent scale of f_eq)
};
static_assert(SC_L2T + 1 == kScUsed && kSc % 4 == 0, "site scalar layout");

// Grid of one or more independent events: periodic transverse grids of their
// own size and eta/s, stored event after event, row-major inside an event.
// 32 bytes, 16-byte aligned: the first four ints are read as one int4
struct alignas(16) EventInfo {
  int site_off, nx, ny, pad;
  double eta_over_s, pad2;
};
static_assert(sizeof(EventInfo) == 32 && alignof(EventInfo) == 16, "EventInfo layout");
struct GridMap {
  const EventInfo* ev;   // n_events entries (device)
  const int2* loc;       // per site (event, y << 16 | x) when n_events > 1 (device)
  int n_events;
  int nx0, ny0;          // the grid when n_events == 1 (no table reads)
  int n_sites;           // all events
};

// Launch grid of the per-site kernels: (ny, nx) CTAs for one grid (CTA (y, x)),
// one CTA per site for a batch.
struct SiteLoc {
  int site, x, y, nx, ny, base;
};
__device__ __forceinline__ void locate_site(const GridMap& G, int bx, int by, SiteLoc* L) {
  if (G.n_events == 1) {
    L->base = 0;
    L->nx = G.nx0;
    L->ny = G.ny0;
    L->x = by;
    L->y = bx;
    L->site = bx * G.nx0 + by;
    return;
  }
  const int2 c = __ldg(G.loc + bx);
  const int4 v = __ldg(reinterpret_cast<const int4*>(G.ev + c.x));  // site_off, nx, ny, pad
  L->base = v.x;
  L->nx = v.y;
  L->ny = v.z;
  L->x = c.y & 0xffff;
  L->y = c.y >> 16;
  L->site = bx;
}

// Event holding `site`.
__device__ __forceinline__ int event_of_site(const GridMap& G, int site) {
  return G.n_events == 1 ? 0 : __ldg(G.loc + site).x;
}

// Proper time of the state being advanced, in device memory: the matching
// launch of the corrector stage advances it, so every launch of a step has the
// same parameters from step to step (a step can be replayed as a CUDA graph).
struct Clock {
  double tau, inv_tau;
  float inv_tau_f, pad;
};

struct MatchArgs {
  const double* mom;    // kMom per site (FP64 storage)
  const float* momf;    // kMom x kMomParts partial sums per site (FP32 storage)
  const double* lnM;
  double* Tsite;        // Newton start in, T out
  double* sc;           // kSc per site
  float* scf;           // FP32 copy of sc (read by the FP32-arithmetic kernels)
  double* obs;          // 8 observables per site, or nullptr
  int* err;
  EosView eos;
  GridMap grid;         // events (eta/s per event) and their sizes
  double inv2dx;
  int ns;
  Clock* clock;         // advanced by dtau when non-null (corrector matching)
  double dtau;
};

// Position of a site inside its event (matching: one thread per site).
__device__ __forceinline__ void site_xy(const GridMap& G, int site, int* e, int* x, int* y) {
  if (G.n_events == 1) {
    *e = 0;
    *y = site / G.nx0;
    *x = site - *y * G.nx0;
    return;
  }
  const int2 c = __ldg(G.loc + site);
  *e = c.x;
  *y = c.y >> 16;
  *x = c.y & 0xffff;
}

// Matching of one site in FP64 (FP64 storage path): Landau (u, eps_kin), T from
// e(T) = eps_kin (B at its equilibrium value, Eq. sanity), then M(T), dB/deps,
// tau_R (Sec. 4.1) and B(T) from the table.  Writes the kSc site scalars to o,
// the temperature to Tsite (the next Newton start) and the observables when
// A.obs is set; returns the error bits.
__device__ __forceinline__ int match_site_d(const MatchArgs& A, int site, double (&o)[kSc]) {
  double m[kMom];
  const double* q = A.mom + (size_t)site * kMom;
#pragma unroll
  for (int i = 0; i < kMom; ++i) m[i] = q[i];
  const double lnM = A.lnM[site];
  const double M = exp(lnM);
  const double pref = M * M * M * M * (1.0 / (2.0 * 3.14159265358979323846 * 3.14159265358979323846));
  double tm[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) tm[i] = pref * m[1 + i];
  int err = 0;
  double u[3], eps;
  if (!landau3(tm, u, &eps)) {
    err |= ERR_LANDAU;
    u[0] = 1.0; u[1] = 0.0; u[2] = 0.0;
    eps = fmax(tm[0], 1e-300);
  }
  const double Tg = A.Tsite[site];
  double y, yg = (Tg > 0.0) ? log(Tg) : 0.0;
  if (!eos_invert(A.eos, EOS_E, eps, yg, &y)) {
    err |= ERR_EOS;
    y = fmin(fmax(yg, A.eos.y0 + 2.0 / A.eos.inv_h), A.eos.y0 + (A.eos.n - 4) / A.eos.inv_h);
  }
  int i0;
  double t, w[6];
  eos_cell(A.eos, y, &i0, &t);
  lagrange6(t, w);
  int ev, sxi, syi;
  site_xy(A.grid, site, &ev, &sxi, &syi);
  const EventInfo& evi = A.grid.ev[ev];
  const double T = exp(y);
  const double Meq = eos_field(A.eos, i0, w, EOS_X) * T;
  const double D = eos_field(A.eos, i0, w, EOS_D);
  const double itr = eos_field(A.eos, i0, w, EOS_INVH) / evi.eta_over_s;
  const double T2 = T * T;
  const double B = eos_field(A.eos, i0, w, EOS_B) * T2 * T2;
  if (!isfinite(T) || !isfinite(u[1]) || !isfinite(u[2]) || !isfinite(B)) err |= ERR_NONFINITE;
  A.Tsite[site] = T;
  o[SC_UT] = u[0]; o[SC_UX] = u[1]; o[SC_UY] = u[2];
  o[SC_INVT] = 1.0 / T; o[SC_MEQ] = Meq; o[SC_M] = M; o[SC_ITR] = itr; o[SC_D] = D;
  o[SC_L2T] = 1.4426950408889634 / T;
  o[SC_B] = B; o[SC_K] = pref * m[0]; o[SC_KH] = m[0]; o[SC_T] = T;
  {
    const int nx = evi.nx, ny = evi.ny, x = sxi, yy = syi;
    const double* lm = A.lnM + evi.site_off;
    const int xp = x + 1 == nx ? 0 : x + 1, xm = x == 0 ? nx - 1 : x - 1;
    const int yp = yy + 1 == ny ? 0 : yy + 1, ym = yy == 0 ? ny - 1 : yy - 1;
    const int ne = nx * ny;
    o[SC_AX] = (lm[idx_checked(yy * nx + xp, ne, A.err)] - lm[idx_checked(yy * nx + xm, ne, A.err)]) * A.inv2dx;
    o[SC_AY] = (lm[idx_checked(yp * nx + x, ne, A.err)] - lm[idx_checked(ym * nx + x, ne, A.err)]) * A.inv2dx;
  }
  if (A.obs) {
    const double hc = 0.1973269804, h3 = hc * hc * hc;
    double* r = A.obs + (size_t)site * 8;
    r[0] = (eps + B) / h3;
    r[1] = T;
    r[2] = u[0]; r[3] = u[1]; r[4] = u[2];
    r[5] = M;
    r[6] = (pref * m[7] - B) / h3;
    r[7] = Meq;
  }
  return err;
}

// The same matching in FP32 arithmetic (FP32 and BF16 storage paths, whose
// kernels consume the site scalars in FP32).  On GB300 an FP64 warp
// instruction occupies the pipe for 64 cycles, so the matching keeps FP64 only
// for the differences of ln M (central differences of nearly equal values).
__device__ __forceinline__ int match_site_f(const MatchArgs& A, int site, float (&o)[kSc]) {
  // moments: the kMomParts FP32 partial sums combined with TwoSum; T^{mu nu}
  // in double-FP32 for the FP64-accurate Landau eigenvalue and EOS step
  float m[kMom], mlo[kMom];
  const float4* q = reinterpret_cast<const float4*>(A.momf + (size_t)site * kMom * kMomParts);
#pragma unroll
  for (int i = 0; i < kMom; ++i) {
    const float4 v = __ldg(q + i);
    float s1, e1, s2, e2, s, e;
    two_sum(v.x, v.y, s1, e1);
    two_sum(v.z, v.w, s2, e2);
    two_sum(s1, s2, s, e);
    e += e1 + e2;
    two_sum(s, e, m[i], mlo[i]);  // m + mlo = the compensated sum
  }
  // M = exp(ln M) in FP32 (M is consumed in FP32; its rounding scales all of
  // T^{mu nu} alike, which moves eps by the same relative amount and leaves u)
  const double lnMd = A.lnM[site];
  const float lh = (float)lnMd, ll = (float)(lnMd - (double)lh);
  const float M = expf(lh) * (1.f + ll);
  const float M2 = M * M;
  const float pref = M2 * M2 * (float)(1.0 / (2.0 * 3.14159265358979323846 * 3.14159265358979323846));
  f2x tmd[6];
  float tmf[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    tmd[i] = df_mul(f2x{pref, 0.f}, f2x{m[1 + i], mlo[1 + i]});
    tmf[i] = pref * m[1 + i];
  }
  int err = 0;
  float u[3];
  f2x epsx;
  if (!landau3_df(tmd, tmf, u, &epsx)) {
    err |= ERR_LANDAU;
    u[0] = 1.f; u[1] = 0.f; u[2] = 0.f;
    epsx = tmd[0].hi > 0.f ? tmd[0] : f2x{1e-30f, 0.f};
  }
  const float eps = epsx.hi + epsx.lo;
  const float Tg = (float)A.Tsite[site];
  const float yg = (Tg > 0.f) ? logf(Tg) : 0.f;
  float y;
  if (!eos_invert_f(A.eos, EOS_E, eps, yg, &y)) {
    err |= ERR_EOS;
    y = fminf(fmaxf(yg, A.eos.ylo_f), A.eos.yhi_f);
  } else {
    y = eos_refine_df(A.eos, EOS_E, epsx, y);
  }
  int i0;
  float t, w[6];
  eos_cellf(A.eos, y, &i0, &t);
  lagrange6f(t, w);
  int ev, sxi, syi;
  site_xy(A.grid, site, &ev, &sxi, &syi);
  const EventInfo& evi = A.grid.ev[ev];
  const float T = expf(y);
  const float Meq = eos_fieldf(A.eos, i0, w, EOS_X) * T;
  const float D = eos_fieldf(A.eos, i0, w, EOS_D);
  const float itr = eos_fieldf(A.eos, i0, w, EOS_INVH) / (float)evi.eta_over_s;
  const float T2 = T * T;
  const float B = eos_fieldf(A.eos, i0, w, EOS_B) * T2 * T2;
  if (!isfinite(T) || !isfinite(u[1]) || !isfinite(u[2]) || !isfinite(B)) err |= ERR_NONFINITE;
  A.Tsite[site] = (double)T;
  o[SC_UT] = u[0]; o[SC_UX] = u[1]; o[SC_UY] = u[2];
  o[SC_INVT] = 1.f / T; o[SC_MEQ] = Meq; o[SC_M] = M; o[SC_ITR] = itr; o[SC_D] = D;
  {
    // log2(e) / T with log2(e) split into FP32 hi + lo: the product is within
    // an ulp of the exact one (an FP32 log2(e) alone is 1.3e-8 low, the same
    // sign at every site)
    constexpr float kL2eHi = 1.44269502162933349609375f, kL2eLo = 1.92596298909109e-8f;
    const float iT = o[SC_INVT];
    o[SC_L2T] = fmaf(kL2eHi, iT, kL2eLo * iT);
  }
  o[SC_B] = B; o[SC_K] = pref * m[0]; o[SC_KH] = m[0]; o[SC_T] = T;
  {
    const int nx = evi.nx, ny = evi.ny, x = sxi, yy = syi;
    const double* lm = A.lnM + evi.site_off;
    const int xp = x + 1 == nx ? 0 : x + 1, xm = x == 0 ? nx - 1 : x - 1;
    const int yp = yy + 1 == ny ? 0 : yy + 1, ym = yy == 0 ? ny - 1 : yy - 1;
    const float i2dx = (float)A.inv2dx;
    const int ne = nx * ny;
    o[SC_AX] = (float)(lm[idx_checked(yy * nx + xp, ne, A.err)] - lm[idx_checked(yy * nx + xm, ne, A.err)]) * i2dx;
    o[SC_AY] = (float)(lm[idx_checked(yp * nx + x, ne, A.err)] - lm[idx_checked(ym * nx + x, ne, A.err)]) * i2dx;
  }
  if (A.obs) {
    const double hc = 0.1973269804, h3 = hc * hc * hc;
    double* r = A.obs + (size_t)site * 8;
    r[0] = ((double)epsx.hi + (double)epsx.lo + (double)B) / h3;
    r[1] = T;
    r[2] = u[0]; r[3] = u[1]; r[4] = u[2];
    r[5] = M;
    r[6] = ((double)pref * ((double)m[7] + (double)mlo[7]) - (double)B) / h3;
    r[7] = Meq;
  }
  return err;
}

// Matching of every site, one thread per site.  FAST: FP32 arithmetic, results
// to scf only; otherwise FP64, results to sc (and scf when set).
template <bool FAST>
__global__ void __launch_bounds__(128) match_kernel(const MatchArgs A) {
  const int site = blockIdx.x * blockDim.x + threadIdx.x;
  if (A.clock && site == 0) {  // the state being matched is at tau + dtau
    const double tau = A.clock->tau + A.dtau, inv = 1.0 / tau;
    A.clock->tau = tau;
    A.clock->inv_tau = inv;
    A.clock->inv_tau_f = (float)inv;
  }
  if (site >= A.ns) return;
  if constexpr (FAST) {
    float o[kSc];
    o[kSc - 1] = 0.f;
    const int err = match_site_f(A, site, o);
    if (err) atomicOr(A.err, err);
    float4* of = reinterpret_cast<float4*>(A.scf + (size_t)site * kSc);  // 64 bytes per site
#pragma unroll
    for (int q = 0; q < kSc / 4; ++q) of[q] = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
  } else {
    double o[kSc];
    o[kSc - 1] = 0.0;
    const int err = match_site_d(A, site, o);
    if (err) atomicOr(A.err, err);
    double2* od = reinterpret_cast<double2*>(A.sc + (size_t)site * kSc);
#pragma unroll
    for (int q = 0; q < kSc / 2; ++q) od[q] = make_double2(o[2 * q], o[2 * q + 1]);
    if (A.scf) {
      float4* of = reinterpret_cast<float4*>(A.scf + (size_t)site * kSc);
#pragma unroll
      for (int q = 0; q < kSc / 4; ++q)
        of[q] = make_float4((float)o[4 * q], (float)o[4 * q + 1], (float)o[4 * q + 2], (float)o[4 * q + 3]);
    }
  }
}

// ---------------------------------------------------------------------------
// block reductions (FP64)
// ---------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ void warp_sum(double (&v)[NV]) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] += __shfl_down_sync(0xffffffffu, v[q], off);
}


// Warp sums of NV values (NV a power of two <= 32) by recursive halving: each
// exchange level hands half of the remaining values to the partner lane, so 8
// values take 9 shuffles instead of 40.  On return v[0] of lane l holds the
// warp sum of value (l >> (5 - log2 NV)).
template <int NV>
__device__ __forceinline__ void warp_reduce_halving(float (&v)[NV], int lane) {
  constexpr int L = NV >= 32 ? 5 : NV >= 16 ? 4 : NV >= 8 ? 3 : NV >= 4 ? 2 : NV >= 2 ? 1 : 0;
  static_assert((1 << L) == NV, "power of two");
#pragma unroll
  for (int lev = 0; lev < L; ++lev) {
    const int h = NV >> (lev + 1), off = 16 >> lev;
    const bool upper = (lane & off) != 0;
#pragma unroll
    for (int q = 0; q < h; ++q) {
      const float keep = upper ? v[q + h] : v[q];
      const float send = upper ? v[q] : v[q + h];
      v[q] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
#pragma unroll
  for (int off = 16 >> L; off > 0; off >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], off);
}

// Block sum of NV per-thread values on thread 0.  FP32: compensated FP32 warp
// trees, then the per-warp (s, c) pairs combined with TwoSum by thread 0; the
// result is left in redf[2q] + redf[2q+1].  FP64: plain warp trees, result in
// redd[q].  The caller synchronises before other threads read the result.
template <int NV, int NT, class R>
__device__ __forceinline__ void block_reduce(const R (&v)[NV], float* redf, double* redd) {
  constexpr int NW = (NT + 31) / 32;
  static_assert(NT < 32 || NT % 32 == 0, "one partial warp or whole warps");
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if constexpr (NT < 32) {
    // a block of one partial warp: no shuffles (lanes >= NT do not exist);
    // thread 0 sums the staged values in FP64
    __shared__ double buf[NT * NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) buf[threadIdx.x * NV + q] = (double)v[q];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        double acc = 0.0;
        for (int i = 0; i < NT; ++i) acc += buf[i * NV + q];
        if constexpr (sizeof(R) == 4) {
          const float hi = (float)acc;
          redf[2 * q] = hi;
          redf[2 * q + 1] = (float)(acc - (double)hi);
        } else {
          redd[q] = acc;
        }
      }
    }
  } else if constexpr (sizeof(R) == 4) {
    // pairwise sums inside each warp (recursive halving over the NV values,
    // padded to a power of two); the warp partials are combined with TwoSum so
    // the block total keeps a compensation term
    constexpr int NP = NV <= 1 ? 1 : NV <= 2 ? 2 : NV <= 4 ? 4 : NV <= 8 ? 8 : 16;
    constexpr int L = NP == 1 ? 0 : NP == 2 ? 1 : NP == 4 ? 2 : NP == 8 ? 3 : 4;
    float s[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) s[q] = q < NV ? (float)v[q] : 0.0f;
    warp_reduce_halving<NP>(s, lane);
    const int q = lane >> (5 - L);
    if ((lane & ((1 << (5 - L)) - 1)) == 0 && q < NV) {
      redf[(wid * NV + q) * 2] = s[0];
      redf[(wid * NV + q) * 2 + 1] = 0.0f;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        float a = redf[2 * q], ca = redf[2 * q + 1];
        for (int w = 1; w < NW; ++w) {
          const float b = redf[(w * NV + q) * 2], cb = redf[(w * NV + q) * 2 + 1];
          const float t = a + b, bp = t - a;
          ca += cb + ((a - (t - bp)) + (b - bp));
          a = t;
        }
        const float t = a + ca;  // renormalise the pair
        redf[2 * q + 1] = ca - (t - a);
        redf[2 * q] = t;
      }
    }
  } else {
    double d[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) d[q] = (double)v[q];
    warp_sum<NV>(d);
    if (lane == 0)
#pragma unroll
      for (int q = 0; q < NV; ++q) redd[wid * NV + q] = d[q];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        double acc = redd[q];
        for (int w = 1; w < NW; ++w) acc += redd[w * NV + q];
        redd[q] = acc;
      }
    }
  }
}

__device__ __forceinline__ int wrap(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// Per-thread partial moments of a xi-line (kMom values, no M^4/(2 pi^2)
// prefactor), in the compute precision R.
template <class R, int NXI, int NTH, int NPH>
__device__ __forceinline__ void line_moments(const Ops<R, NXI, NTH, NPH>& op, const R (&f)[NXI],
                                             int j, int l, R (&mom)[kMom]) {
  R r0 = 0, r1 = 0, r2 = 0, r3 = 0;
#pragma unroll
  for (int k = 0; k < NXI; ++k) {
    r0 += op.w0[k] * f[k];
    r1 += op.w1[k] * f[k];
    r2 += op.w2[k] * f[k];
    r3 += op.w3[k] * f[k];
  }
  const R wj = op.wj[j], st = op.sth[j], mu = op.mu[j];
  const R cp = op.cph[l], sp = op.sph[l];
  const R a1 = wj * r1 * st, a3 = wj * r3 * st * st;
  mom[0] = wj * r0;
  mom[1] = wj * r2;
  mom[2] = a1 * cp;
  mom[3] = a1 * sp;
  mom[4] = a3 * cp * cp;
  mom[5] = a3 * cp * sp;
  mom[6] = a3 * sp * sp;
  mom[7] = wj * r3 * mu * mu;
}

// ---------------------------------------------------------------------------
// fused stream-collide stage: evaluates the kinetic right-hand side of one
// site on f_in (with the site scalars of f_in's matching) and writes the
// predictor or the trapezoid corrector, then the moments of what it wrote.
//   rhs = -V.grad f + (1/tau) [mu^2 Dr f + Dth f] + g Dr f + T_M f_eq
//         - ((P.U)/E) (f - f_eq) / tau_R
//   T_M f_eq = -(f_eq/T) [ (a.v/c)(u^tau M^2 s^2/E_eq - M v.u)
//                          + (u^tau M^2 (a.v)/E_eq - M a.u)/c ],   a = grad ln M
//   (node motion with the local mass and the force 1/2 d_i M^2 d^i_(p) of
//   Eq. Bmilne, applied to the local equilibrium),
//   g   = -D sum w (P^.U)^2 R / (K + D (4 E + Q - K))   (d ln M / d tau)
// ---------------------------------------------------------------------------
template <class S, class R, int NXI, int NTH, int NPH>
struct StageArgs {
  const S* f_in;          // populations the right-hand side is evaluated on
  const double* lnM_in;
  const double* sc;       // matching of f_in, kSc per site
  const float* scf;       // FP32 copy of sc
  const S* f_base;        // corrector: populations at the start of the step
  const double* lnM_base;
  S* f_out;
  double* lnM_out;
  double* mom_out;        // moments of f_out, kMom per site (FP64 storage)
  float* momf_out;        // moments of f_out, kMomParts partial sums (FP32 storage)
  int* err;
  GridMap grid;
  const Clock* clock;     // proper time of f_in
  int milne_on;           // Milne metric (1/tau terms) or Minkowski
  int mode;               // 0 predictor, 1 corrector
  double dtau, inv2dx;    // FP64 copies for the per-site (thread 0) arithmetic
  R dtau_r, inv2dx_r, Z;  // the same constants in the compute precision
  Ops<R, NXI, NTH, NPH> op;
};

template <class S, class R, int NXI, int NTH, int NPH>
__global__ void __launch_bounds__(NTH* NPH)
    stage_kernel(const __grid_constant__ StageArgs<S, R, NXI, NTH, NPH> A) {
  constexpr int NL = NTH * NPH;
  constexpr int NN = NL * NXI;
  constexpr int NW = (NL + 31) / 32;
  const auto& op = A.op;
  SiteLoc L;
  locate_site(A.grid, blockIdx.x, blockIdx.y, &L);
  const int x = L.x, y = L.y, site = idx_checked(L.site, A.grid.n_sites, A.err), nx = L.nx, ny = L.ny;
  const int t = threadIdx.x;
  const int j = t % NTH, l = t / NTH;

  // populations staged k-major with a padded stride, so that both the xi-line
  // (consecutive threads) and the polar-line accesses are bank-conflict free
  constexpr int LD = NL + 1;
  __shared__ R fs[NXI * LD];
  __shared__ R pth[NXI * LD];
  __shared__ double redd[kMom * NW];
  __shared__ float redf[2 * kMom * NW];
  __shared__ R gsh;
  __shared__ __align__(16) R Etab[2 * NXI];  // (E_eq, 1/E_eq) per radial node
  __shared__ double lnm_s[4];                  // ln M of f_in, f_base (lnm_fetch)
  if (t == 0) lnm_fetch(lnm_s, A.lnM_in, A.lnM_base, site, A.mode);

  // 1. own xi-line and the upwind neighbours for streaming
  R f[NXI];
  load_line<S, R, NXI>(A.f_in + (size_t)site * NN + t * NXI, f);
  const R cp = op.cph[l], sp = op.sph[l];
  // upwind neighbours (periodic): x -/+ 1, 2 when cos(phi) >/<= 0, likewise y
  const int sx = (cp > (R)0) ? -1 : 1, sy = (sp > (R)0) ? -1 : 1;
  int x1 = x + sx, x2 = x + 2 * sx, y1 = y + sy, y2 = y + 2 * sy;
  x1 += (x1 < 0) ? nx : (x1 >= nx ? -nx : 0);
  x2 += (x2 < 0) ? nx : (x2 >= nx ? -nx : 0);
  x2 += (x2 < 0) ? nx : (x2 >= nx ? -nx : 0);  // grids of one site
  y1 += (y1 < 0) ? ny : (y1 >= ny ? -ny : 0);
  y2 += (y2 < 0) ? ny : (y2 >= ny ? -ny : 0);
  y2 += (y2 < 0) ? ny : (y2 >= ny ? -ny : 0);
  const int ns_all = A.grid.n_sites;
  const int sx1 = idx_checked(L.base + y * nx + idx_checked(x1, nx, A.err), ns_all, A.err);
  const int sx2 = idx_checked(L.base + y * nx + idx_checked(x2, nx, A.err), ns_all, A.err);
  const int sy1 = idx_checked(L.base + idx_checked(y1, ny, A.err) * nx + x, ns_all, A.err);
  const int sy2 = idx_checked(L.base + idx_checked(y2, ny, A.err) * nx + x, ns_all, A.err);
  R fx1[NXI], fx2[NXI], fy1[NXI], fy2[NXI];
  load_line<S, R, NXI>(A.f_in + (size_t)sx1 * NN + t * NXI, fx1);
  load_line<S, R, NXI>(A.f_in + (size_t)sx2 * NN + t * NXI, fx2);
  load_line<S, R, NXI>(A.f_in + (size_t)sy1 * NN + t * NXI, fy1);
  load_line<S, R, NXI>(A.f_in + (size_t)sy2 * NN + t * NXI, fy2);

  // 2. radial operator on the own line; stage the site for the polar operator;
  //    per-site radial tables E_eq(k) = sqrt(M_eq^2 + M^2 sinh^2 xi_k) and 1/E_eq
  R scl[kSc];
  if constexpr (sizeof(R) == 4) {
    const float* q = A.scf + (size_t)site * kSc;
#pragma unroll
    for (int i = 0; i < kScUsed; ++i) scl[i] = __ldg(q + i);
  } else {
    const double* q = A.sc + (size_t)site * kSc;
#pragma unroll
    for (int i = 0; i < kScUsed; ++i) scl[i] = __ldg(q + i);
  }
  const R ut = scl[SC_UT], ux = scl[SC_UX], uy = scl[SC_UY];
  const R invT = scl[SC_INVT], Meq = scl[SC_MEQ], M = scl[SC_M], itr = scl[SC_ITR];
  const R M2 = M * M;
  if (t < NXI) {
    const R e = fsqrt<R>(Meq * Meq + M2 * op.s2[t]);
    Etab[2 * t] = e;
    Etab[2 * t + 1] = (R)1 / e;
  }
#pragma unroll
  for (int k = 0; k < NXI; ++k) fs[k * LD + t] = f[k];
  R Drf[NXI];
#pragma unroll
  for (int kp = 0; kp < NXI; ++kp) {
    R acc = 0;
#pragma unroll
    for (int k = 0; k < NXI; ++k) acc += op.Dr[kp * NXI + k] * f[k];
    Drf[kp] = acc;
  }
  __syncthreads();
  R milne = 0;
  if (A.milne_on) {
    if constexpr (sizeof(R) == 8) milne = (R)A.clock->inv_tau;
    else milne = (R)A.clock->inv_tau_f;
  }
  if (milne != (R)0) {
    for (int it = t; it < NXI * NPH; it += NL) {  // polar lines (k', l'): (1/tau) Dth along j
      const int kq = it % NXI, lq = it / NXI;
      R g[NTH];
#pragma unroll
      for (int jj = 0; jj < NTH; ++jj) g[jj] = fs[kq * LD + lq * NTH + jj];
#pragma unroll
      for (int jp = 0; jp < NTH; ++jp) {
        R dth = 0;
#pragma unroll
        for (int jj = 0; jj < NTH; ++jj) dth += op.Dth[jp * NTH + jj] * g[jj];
        pth[kq * LD + lq * NTH + jp] = dth;
      }
    }
  }
  __syncthreads();

  // 3. right-hand side on the own xi-line.  With vu = (v.u)/sinh, A1 = (a.v)/sinh:
  //    f_eq  = Z exp((M vu sinh - u^tau E_eq)/T)
  //    force = -(f_eq/(T cosh)) [A1 u^tau M^2 sinh (sinh^2+1)/E_eq - A1 M vu sinh^2 - M a.u]
  //          = f_eq [Gp q1/E_eq + Hp q2 + Jp/cosh]
  //    coll  = -(f - f_eq) (u^tau - tanh vu)/tau_R,    pu = cosh u^tau - sinh vu
  const R ax = scl[SC_AX], ay = scl[SC_AY];
  const R st = op.sth[j], mu2 = op.mu2[j];
  const R vu = st * (cp * ux + sp * uy);
  const R A1 = st * (ax * cp + ay * sp);
  const R au = ax * ux + ay * uy;
  const R nsx = -st * (cp < 0 ? -cp : cp) * A.inv2dx_r;
  const R nsy = -st * (sp < 0 ? -sp : sp) * A.inv2dx_r;
  const R wj = op.wj[j];
  const R milne_mu2 = milne * mu2;
  constexpr bool kF = sizeof(R) == 4;
  const R lsc = kF ? (R)1.4426950408889634 : (R)1;  // exp2 in FP32, exp in FP64
  const R c1 = -lsc * invT * ut, c2 = lsc * invT * M * vu;
  const R lZ = kF ? (R)log2f((float)A.Z) : (R)0;
  const R Gp = -invT * A1 * ut * M2, Hp = invT * A1 * M * vu, Jp = invT * M * au;
  const R cc0 = ut * itr, cc1 = -vu * itr;
  const bool pol = milne != (R)0;
  R Rn[NXI];
  R sA = 0, sQ = 0, sE = 0;
#pragma unroll
  for (int k = 0; k < NXI; ++k) {
    const R E = Etab[2 * k], iE = Etab[2 * k + 1];
    const R Sx = (R)3 * f[k] - (R)4 * fx1[k] + fx2[k];
    const R Sy = (R)3 * f[k] - (R)4 * fy1[k] + fy2[k];
    R r = op.tv[k] * (nsx * Sx + nsy * Sy) + milne_mu2 * Drf[k];
    if (pol) r += milne * pth[k * LD + t];
    R feq;
    if constexpr (kF) feq = ex2_ftz(c1 * E + (c2 * op.s[k] + lZ));
    else feq = A.Z * exp(c1 * E + c2 * op.s[k]);
    const R fc = (Gp * op.q1[k]) * iE + (Hp * op.q2[k] + Jp * op.inv_c[k]);
    const R cc = cc0 + cc1 * op.tv[k];
    r += feq * (fc + cc) - f[k] * cc;
    Rn[k] = r;
    const R pu = op.c[k] * ut - op.s[k] * vu;
    const R wpu2 = (wj * op.ecw[k]) * (pu * pu);
    sA += wpu2 * r;
    sQ += wpu2 * Drf[k];
    sE += wpu2 * f[k];
  }
  const R v3[3] = {sA, sQ, sE};
  block_reduce<3, NL, R>(v3, redf, redd);
  if (t == 0) {
    // d ln M / d tau from the consistency condition, in the compute precision
    R g;
    const R D = scl[SC_D], Kh = scl[SC_KH];
    if constexpr (sizeof(R) == 4) {
      const float Af = redf[0] + redf[1], Qf = redf[2] + redf[3], Ef = redf[4] + redf[5];
      g = (D == 0.f) ? 0.f : -D * Af / (Kh + D * (4.f * Ef + Qf - Kh));
    } else {
      g = (D == 0.0) ? 0.0 : -D * redd[0] / (Kh + D * (4.0 * redd[2] + redd[1] - Kh));
    }
    if (!isfinite((double)g)) atomicOr(A.err, (int)ERR_NONFINITE);
    gsh = g;
    lnm_wait();
    const double lnM = lnm_s[0], gd = (double)g;
    A.lnM_out[site] = A.mode == 0 ? lnM + A.dtau * gd : 0.5 * (lnm_s[2] + lnM + A.dtau * gd);
  }
  __syncthreads();
  const R g = gsh;
  const R dt = A.dtau_r;
  R out[NXI];
  if (A.mode == 0) {
#pragma unroll
    for (int k = 0; k < NXI; ++k) out[k] = f[k] + dt * (Rn[k] + g * Drf[k]);
  } else {
    R fb[NXI];
    load_line<S, R, NXI>(A.f_base + (size_t)site * NN + t * NXI, fb);
#pragma unroll
    for (int k = 0; k < NXI; ++k) out[k] = (R)0.5 * (fb[k] + f[k] + dt * (Rn[k] + g * Drf[k]));
  }
  // the moments describe exactly what is stored (after rounding to S)
#pragma unroll
  for (int k = 0; k < NXI; ++k) out[k] = ld1<S, R>(st1<S, R>(out[k]));
  finite_checked(out, NXI, A.err);
  store_line<S, R, NXI>(A.f_out + (size_t)site * NN + t * NXI, out);
  R mom[kMom];
  line_moments<R, NXI, NTH, NPH>(op, out, j, l, mom);
  block_reduce<kMom, NL, R>(mom, redf, redd);
  if (t == 0) {
    if constexpr (sizeof(R) == 4) {
      store_mom_parts(A.momf_out + (size_t)site * kMom * kMomParts, redf);
    } else {
#pragma unroll
      for (int q = 0; q < kMom; ++q) A.mom_out[(size_t)site * kMom + q] = redd[q];
    }
  }
}

// ---------------------------------------------------------------------------
// initial condition: local equilibrium at rest with energy density eps0
// (eps_EOS(T) = eps0, M = M(T), f = Z exp(-E/T)), and its moments
// ---------------------------------------------------------------------------
template <class S, class R, int NXI, int NTH, int NPH>
struct InitArgs {
  const double* eps0;  // GeV/fm^3
  double eps_scale;    // (hbar c)^3: GeV/fm^3 -> GeV^4
  const double* tsm;   // per site (T, M_eq, M) from init_site_kernel
  S* f;
  double* lnM;
  double* Tsite;
  double* mom;
  float* momf;
  int* err;
  EosView eos;
  double Z;
  int family;
  double T0;
  double s2d[NXI];  // sinh^2 xi_k in FP64 (the exponent of f_eq is evaluated in FP64)
  Ops<R, NXI, NTH, NPH> op;
};

// Initial condition, per site (one thread each: the FP64 Newton inversion of
// the EOS is a serial chain, and a warp of sites keeps all 32 lanes of each
// FP64 instruction busy): T from eps_EOS(T) = eps0, M_eq = x(T) T, M = M_eq
// (or T0 for the conformal family); writes T, ln M and (T, M_eq, M) to tsm.
struct InitSiteArgs {
  const double* eps0;  // GeV/fm^3
  double eps_scale;    // (hbar c)^3: GeV/fm^3 -> GeV^4
  double* lnM;
  double* Tsite;
  double* tsm;         // 3 per site
  int* err;
  EosView eos;
  int family;
  double T0;
  int ns;
};

__global__ void __launch_bounds__(128) init_site_kernel(const InitSiteArgs A) {
  const int site = blockIdx.x * blockDim.x + threadIdx.x;
  if (site >= A.ns) return;
  double y = 0.0;
  if (!eos_invert(A.eos, EOS_EPS, __ldg(A.eps0 + site) * A.eps_scale, log(0.3), &y)) {
    atomicOr(A.err, (int)ERR_EOS);
    y = log(0.3);
  }
  int i0;
  double tt, w[6];
  eos_cell(A.eos, y, &i0, &tt);
  lagrange6(tt, w);
  const double T = exp(y);
  const double Meq = eos_field(A.eos, i0, w, EOS_X) * T;
  const double M = A.family == 1 ? A.T0 : Meq;
  A.Tsite[site] = T;
  A.lnM[site] = log(M);
  double* o = A.tsm + (size_t)site * 3;
  o[0] = T; o[1] = Meq; o[2] = M;
}

template <class S, class R, int NXI, int NTH, int NPH>
__global__ void __launch_bounds__(NTH* NPH)
    init_kernel(const __grid_constant__ InitArgs<S, R, NXI, NTH, NPH> A) {
  // At rest f_eq = Z exp(-E_eq/T) depends on the radial node only: the NXI
  // values of a site are evaluated once, in FP64 (the exponent reaches ~40 in
  // magnitude, where an FP32 evaluation would be off by ~1e-6), and rounded
  // once to the storage precision; the moments of what is stored are summed
  // in R.
  constexpr int NL = NTH * NPH;
  constexpr int NN = NL * NXI;
  constexpr int NW = (NL + 31) / 32;
  static_assert(NXI <= NL, "one thread per radial node");
  const int site = blockIdx.x, t = threadIdx.x;
  const int j = t % NTH, l = t / NTH;
  __shared__ double redd[kMom * NW];
  __shared__ float redf[2 * kMom * NW];
  __shared__ double fk[NXI];
  if (t < NXI) {
    const double* sc = A.tsm + (size_t)site * 3;  // (T, M_eq, M) of init_site_kernel
    const double T = __ldg(sc), Meq = __ldg(sc + 1), M = __ldg(sc + 2);
    fk[t] = A.Z * exp(-sqrt(Meq * Meq + M * M * A.s2d[t]) / T);
  }
  __syncthreads();
  R out[NXI];
#pragma unroll
  for (int k = 0; k < NXI; ++k) out[k] = ld1<S, R>(st1<S, double>(fk[k]));
  store_line<S, R, NXI>(A.f + (size_t)site * NN + t * NXI, out);
  R mom[kMom];
  line_moments<R, NXI, NTH, NPH>(A.op, out, j, l, mom);
  block_reduce<kMom, NL, R>(mom, redf, redd);
  if (t == 0) {
    if constexpr (sizeof(R) == 4) {
      store_mom_parts(A.momf + (size_t)site * kMom * kMomParts, redf);
    } else {
#pragma unroll
      for (int q = 0; q < kMom; ++q) A.mom[(size_t)site * kMom + q] = redd[q];
    }
  }
}

// ---------------------------------------------------------------------------
// moments of stored populations (kMom per site), used where no stage kernel
// has produced them (the step variant that works in static scratch)
// ---------------------------------------------------------------------------
template <class S, class R, int NXI, int NTH, int NPH>
struct MomentsArgs {
  const S* f;
  double* mom;
  float* momf;
  Ops<R, NXI, NTH, NPH> op;
};

template <class S, class R, int NXI, int NTH, int NPH>
__global__ void __launch_bounds__(NTH* NPH)
    moments_kernel(const __grid_constant__ MomentsArgs<S, R, NXI, NTH, NPH> A) {
  constexpr int NL = NTH * NPH;
  constexpr int NN = NL * NXI;
  constexpr int NW = (NL + 31) / 32;
  const int site = blockIdx.x, t = threadIdx.x;
  const int j = t % NTH, l = t / NTH;
  __shared__ double redd[kMom * NW];
  __shared__ float redf[2 * kMom * NW];
  R f[NXI];
  load_line<S, R, NXI>(A.f + (size_t)site * NN + t * NXI, f);
  R mom[kMom];
  line_moments<R, NXI, NTH, NPH>(A.op, f, j, l, mom);
  block_reduce<kMom, NL, R>(mom, redf, redd);
  if (t == 0) {
    if constexpr (sizeof(R) == 4) {
      store_mom_parts(A.momf + (size_t)site * kMom * kMomParts, redf);
    } else {
#pragma unroll
      for (int q = 0; q < kMom; ++q) A.mom[(size_t)site * kMom + q] = redd[q];
    }
  }
}

// ---------------------------------------------------------------------------
// grid observables (no counterpart in the paper; the usual heavy-ion forms on
// the paper's moments, Eq. emtnew, and momentum weights, Sec. 4.3):
//   eps_p = sum_x (T^xx - T^yy) / sum_x (T^xx + T^yy),  T = T_kin + B g
//   v2    = sum_{x,n} W_n p_perp,n cos 2phi_n f_n / sum_{x,n} W_n p_perp,n f_n,
//           W_n = M^2 w_n / (2 pi^2), p_perp = M sinh xi sin theta
// Pass 1 (one CTA per site) writes four FP64 partial sums per site; pass 2 (one
// CTA) adds them in a fixed order.
// ---------------------------------------------------------------------------
template <class S, class R, int NXI, int NTH, int NPH>
struct ObsArgs {
  const S* f;
  const double* lnM;
  const double* sc;   // site scalars (FP64 matching) or nullptr
  const float* scf;   // site scalars (FP32 matching) when sc is nullptr
  double* part;       // 4 per site: T^xx, T^yy (with B), num, den of v2
  Ops<R, NXI, NTH, NPH> op;
};

template <class S, class R, int NXI, int NTH, int NPH>
__global__ void __launch_bounds__(NTH* NPH)
    observables_kernel(const __grid_constant__ ObsArgs<S, R, NXI, NTH, NPH> A) {
  constexpr int NL = NTH * NPH;
  constexpr int NN = NL * NXI;
  constexpr int NW = (NL + 31) / 32;
  const int site = blockIdx.x, t = threadIdx.x;
  const int j = t % NTH, l = t / NTH;
  __shared__ double redd[4 * NW];
  __shared__ float redf[8 * NW];
  R f[NXI];
  load_line<S, R, NXI>(A.f + (size_t)site * NN + t * NXI, f);
  double r3 = 0.0, rs = 0.0;
#pragma unroll
  for (int k = 0; k < NXI; ++k) {
    r3 += (double)A.op.w3[k] * (double)f[k];
    rs += (double)A.op.ecw[k] * (double)A.op.s[k] * (double)f[k];
  }
  const double wj = A.op.wj[j], st = A.op.sth[j], cp = A.op.cph[l], sp = A.op.sph[l];
  const double den = wj * rs * st;
  const double v[4] = {wj * r3 * st * st * cp * cp, wj * r3 * st * st * sp * sp, den * (cp * cp - sp * sp), den};
  block_reduce<4, NL, double>(v, redf, redd);
  if (t == 0) {
    const double M = exp(__ldg(A.lnM + site));
    const double pi2 = 2.0 * 3.14159265358979323846 * 3.14159265358979323846;
    const double p3 = M * M * M / pi2, p4 = p3 * M;
    const double B = A.sc ? A.sc[(size_t)site * kSc + SC_B] : (double)A.scf[(size_t)site * kSc + SC_B];
    double* o = A.part + (size_t)site * 4;
    o[0] = p4 * redd[0] - B;
    o[1] = p4 * redd[1] - B;
    o[2] = p3 * redd[2];
    o[3] = p3 * redd[3];
  }
}

// out[0] = eps_p, out[1] = v2, out[2..5] the four grid sums; one block of 1024
// threads, fixed summation order
__global__ void __launch_bounds__(1024) observables_reduce_kernel(const double* part, int ns, double* out) {
  __shared__ double red[4 * 32];
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < ns; i += 1024)
#pragma unroll
    for (int q = 0; q < 4; ++q) a[q] += part[(size_t)i * 4 + q];
  warp_sum<4>(a);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < 4; ++q) red[wid * 4 + q] = a[q];
  __syncthreads();
  if (threadIdx.x == 0) {
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int w = 0; w < 32; ++w)
#pragma unroll
      for (int q = 0; q < 4; ++q) s[q] += red[w * 4 + q];
    out[0] = (s[0] - s[1]) / (s[0] + s[1]);
    out[1] = s[2] / s[3];
#pragma unroll
    for (int q = 0; q < 4; ++q) out[2 + q] = s[q];  // the grid sums
  }
}

}  // namespace rlbk
