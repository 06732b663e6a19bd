// rlb_kernels.cuh -- GB300 (sm_103a) kernels of the relativistic lattice
// Boltzmann step with a quasiparticle equation of state (Romatschke,
// arXiv:1108.5561, Sec. 3-4).
//
// Thread mapping: one CTA per lattice site, one thread per "xi-line" (the
// n_xi radial nodes at fixed polar index j and azimuth l, contiguous in
// memory), so a warp's loads of a site are contiguous and vectorised.  The
// site's populations are staged in shared memory for the polar (theta-line)
// and azimuthal (phi-line) operators; the per-site FP64 Landau matching and
// EOS inversion run on lane 0 of warp 0 while the other warps apply the
// polar/azimuthal operators.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace rlbk {

enum : int { ERR_LANDAU = 1, ERR_EOS = 2, ERR_NONFINITE = 4 };

// ---------------------------------------------------------------------------
// per-run constants, passed by value (kernel parameter space = constant bank)
// ---------------------------------------------------------------------------
template <class R, int NXI, int NTH, int NPH>
struct Ops {
  R Dr[NXI * NXI];    // Galerkin v.d/dv (radial part of S1, S2)
  R Dth[NTH * NTH];   // Galerkin (mu - mu^3) d/dmu (polar part of S1)
  R Dmu[NTH * NTH];   // collocation d/dmu
  R Dph[NPH * NPH];   // collocation d/dphi
  // radial node constants
  R c[NXI], s[NXI], c_over_s[NXI], inv_cs[NXI], s2[NXI], inv_c[NXI];
  R w0[NXI], w1[NXI], w2[NXI], w3[NXI];  // ecw * {1, c s, c^2, s^2}
  R ecw[NXI];
  // polar
  R mu[NTH], mu2[NTH], sth[NTH], sth_mu[NTH], wj[NTH];  // wj = w^th_j / (2 NPH)
  // azimuth
  R cph[NPH], sph[NPH];
};

struct EosView {
  const double* tab;  // n x 8 doubles, uniform in y = ln T
  double y0, inv_h;
  int n;
};

template <class S, class R, int NXI, int NTH, int NPH>
struct StageArgs {
  const S* f_in;          // populations the right-hand side is evaluated on
  const double* lnM_in;
  const S* f_base;        // corrector: populations at the start of the step
  const double* lnM_base;
  S* f_out;
  double* lnM_out;
  double* Tsite;          // per-site temperature: Newton start in, matched T out
  int* err;
  EosView eos;
  int nx, ny;
  int mode;               // 0 predictor, 1 corrector
  int metric;             // 1 Milne
  double tau, dtau;
  double inv2dx;
  double Z;
  double eta_over_s;
  Ops<R, NXI, NTH, NPH> op;
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

template <class S, class R, int N>
__device__ __forceinline__ void load_line(const S* __restrict__ p, R (&v)[N]) {
  if constexpr (sizeof(S) == 4 && N % 4 == 0) {
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
  if constexpr (sizeof(S) == 4 && N % 4 == 0) {
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
template <class R> __device__ __forceinline__ R fsqrt(R x);
template <> __device__ __forceinline__ float fsqrt<float>(float x) { return sqrtf(x); }
template <> __device__ __forceinline__ double fsqrt<double>(double x) { return sqrt(x); }

// ---------------------------------------------------------------------------
// EOS table: 6-point Lagrange interpolation in y = ln T (offsets -2..3)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void lagrange6(double t, double w[6], double dw[6]) {
  const double fac[6] = {t + 2.0, t + 1.0, t, t - 1.0, t - 2.0, t - 3.0};
  const double den[6] = {-120.0, 24.0, -12.0, 12.0, -24.0, 120.0};
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    double prod = 1.0, dprod = 0.0;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      if (q == m) continue;
      dprod = dprod * fac[q] + prod;
      prod *= fac[q];
    }
    w[m] = prod / den[m];
    dw[m] = dprod / den[m];
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

// Solve table field `field`(y) = target for y by Newton on the interpolant.
__device__ bool eos_invert(const EosView& E, int field, double target, double y, double* y_out) {
  const double ylo = E.y0 + 2.0 / E.inv_h, yhi = E.y0 + (E.n - 4) / E.inv_h;
  if (!(y > ylo && y < yhi)) y = 0.5 * (ylo + yhi);
  int settled = 0;
  for (int it = 0; it < 60; ++it) {
    int i0;
    double t, w[6], dw[6];
    if (!eos_cell(E, y, &i0, &t)) return false;
    lagrange6(t, w, dw);
    double F = 0.0, dF = 0.0;
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      double v = __ldg(E.tab + (size_t)(i0 - 2 + m) * 8 + field);
      F += w[m] * v;
      dF += dw[m] * v;
    }
    dF *= E.inv_h;
    if (!(dF > 0.0)) return false;
    double dy = (F - target) / dF;
    double yn = y - dy;
    if (yn < ylo) yn = 0.5 * (y + ylo);
    if (yn > yhi) yn = 0.5 * (y + yhi);
    y = yn;
    if (fabs(dy) < 1e-13) {
      if (++settled == 2) { *y_out = y; return true; }
    }
  }
  return false;
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
  for (int it = 0; it < 200; ++it) {
    double p = ((lam - c2) * lam + c1) * lam - c0;
    double dp = (3.0 * lam - 2.0 * c2) * lam + c1;
    if (!(dp > 0.0)) break;
    double d = p / dp;
    if (!(d > 0.0)) break;  // no further decrease: converged from above
    lam -= d;
    if (d <= 1e-16 * fabs(lam)) break;
  }
  const double r0[3] = {a00 - lam, a01, a02};
  const double r1[3] = {a10, a11 - lam, a12};
  const double r2[3] = {a20, a21, a22 - lam};
  double cand[3][3];
  const double* rows[3][2] = {{r0, r1}, {r0, r2}, {r1, r2}};
  int best = 0;
  double bn = -1.0;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const double* a = rows[q][0];
    const double* b = rows[q][1];
    cand[q][0] = a[1] * b[2] - a[2] * b[1];
    cand[q][1] = a[2] * b[0] - a[0] * b[2];
    cand[q][2] = a[0] * b[1] - a[1] * b[0];
    double nn = cand[q][0] * cand[q][0] + cand[q][1] * cand[q][1] + cand[q][2] * cand[q][2];
    if (nn > bn) { bn = nn; best = q; }
  }
  double v0 = cand[best][0], v1 = cand[best][1], v2 = cand[best][2];
  double mn = v0 * v0 - v1 * v1 - v2 * v2;
  if (!(mn > 0.0)) return false;
  double r = rsqrt(mn);
  if (v0 < 0) r = -r;
  u[0] = v0 * r; u[1] = v1 * r; u[2] = v2 * r;
  *eps = u[0] * u[0] * tm[0] - 2.0 * u[0] * u[1] * tm[1] - 2.0 * u[0] * u[2] * tm[2] +
         u[1] * u[1] * tm[3] + 2.0 * u[1] * u[2] * tm[4] + u[2] * u[2] * tm[5];
  return *eps > 0.0;
}

struct SiteState {
  double u[3];
  double T, Meq, D, inv_tauR, eps_kin, B;
};

// Matching of one site (FP64): Landau (u, eps_kin), T from e(T) = eps_kin,
// then M(T), dB/deps, tau_R and B(T) from the table.  Returns error bits.
__device__ int match_site(const EosView& E, const double mom[7], double lnM, double Tguess,
                          double eta_over_s, bool want_B, SiteState* o) {
  const double M = exp(lnM);
  const double pref = M * M * M * M * (1.0 / (2.0 * 3.14159265358979323846 * 3.14159265358979323846));
  double tm[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) tm[q] = pref * mom[1 + q];
  int err = 0;
  double eps;
  if (!landau3(tm, o->u, &eps)) {
    err |= ERR_LANDAU;
    o->u[0] = 1.0; o->u[1] = 0.0; o->u[2] = 0.0;
    eps = fmax(tm[0], 1e-300);
  }
  o->eps_kin = eps;
  double y;
  double yg = (Tguess > 0.0) ? log(Tguess) : 0.0;
  if (!eos_invert(E, 0, log(eps), yg, &y)) {
    err |= ERR_EOS;
    y = fmin(fmax(yg, E.y0 + 2.0 / E.inv_h), E.y0 + (E.n - 4) / E.inv_h);
  }
  int i0;
  double t, w[6], dw[6];
  eos_cell(E, y, &i0, &t);
  lagrange6(t, w, dw);
  const double T = exp(y);
  o->T = T;
  o->Meq = eos_field(E, i0, w, 1) * T;
  o->D = eos_field(E, i0, w, 2);
  o->inv_tauR = 1.0 / (eta_over_s * exp(eos_field(E, i0, w, 3)));
  o->B = want_B ? eos_field(E, i0, w, 4) * T * T * T * T : 0.0;
  if (!isfinite(o->T) || !isfinite(o->u[1]) || !isfinite(o->u[2])) err |= ERR_NONFINITE;
  return err;
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

// Sum v over the block into red[0..NV) (valid after the trailing barrier
// inside); red must hold NV * nwarps doubles.
template <int NV, int NT>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* red) {
  constexpr int NW = (NT + 31) / 32;
  warp_sum<NV>(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) red[wid * NV + q] = v[q];
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double s = red[q];
      for (int w = 1; w < NW; ++w) s += red[w * NV + q];
      red[q] = s;
    }
  }
}

__device__ __forceinline__ int wrap(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// Per-thread partial moments of a xi-line: {K, T00, T01, T02, T11, T12, T22}
// (without the M^4/(2 pi^2) prefactor).
template <class R, int NXI, int NTH, int NPH>
__device__ __forceinline__ void line_moments(const Ops<R, NXI, NTH, NPH>& op, const R (&f)[NXI],
                                             int j, int l, double (&mom)[7], double* tzz) {
  R r0 = 0, r1 = 0, r2 = 0, r3 = 0;
#pragma unroll
  for (int k = 0; k < NXI; ++k) {
    r0 += op.w0[k] * f[k];
    r1 += op.w1[k] * f[k];
    r2 += op.w2[k] * f[k];
    r3 += op.w3[k] * f[k];
  }
  const double wj = (double)op.wj[j], st = (double)op.sth[j];
  const double cp = (double)op.cph[l], sp = (double)op.sph[l];
  mom[0] = wj * (double)r0;
  mom[1] = wj * (double)r2;
  mom[2] = wj * (double)r1 * st * cp;
  mom[3] = wj * (double)r1 * st * sp;
  mom[4] = wj * (double)r3 * st * st * cp * cp;
  mom[5] = wj * (double)r3 * st * st * cp * sp;
  mom[6] = wj * (double)r3 * st * st * sp * sp;
  if (tzz) {
    const double mu = (double)op.mu[j];
    *tzz = wj * (double)r3 * mu * mu;
  }
}

// ---------------------------------------------------------------------------
// fused stream-collide stage: evaluates the kinetic right-hand side of one
// site on f_in and writes the predictor or the trapezoid corrector.
//   rhs = -V.grad f + (1/tau) [mu^2 Dr f + Dth f] + g Dr f + T_M f
//         - ((P.U)/E) (f - f_eq) / tau_R
//   T_M = A sin(th) (c/s) Dr f - A sin(th) mu/(c s) Dmu f + A'/(c s sin th) Dph f
//   g   = -D sum w (P^.U)^2 R / (K + D (4 E + Q - K))   (d ln M / d tau)
// ---------------------------------------------------------------------------
template <class S, class R, int NXI, int NTH, int NPH>
__global__ void __launch_bounds__(NTH* NPH)
    stage_kernel(const __grid_constant__ StageArgs<S, R, NXI, NTH, NPH> A) {
  constexpr int NL = NTH * NPH;
  constexpr int NN = NL * NXI;
  constexpr int NW = (NL + 31) / 32;
  constexpr int LINE0 = (NL > 32) ? 32 : 0;  // first thread doing polar/azimuthal lines
  const auto& op = A.op;
  const int site = blockIdx.x;
  const int t = threadIdx.x;
  const int j = t % NTH, l = t / NTH;
  const int x = site % A.nx, y = site / A.nx;
  const int ns = A.nx * A.ny;

  __shared__ R fs[NN];
  __shared__ R pth[NN];
  __shared__ R pph[NN];
  __shared__ double red[8 * NW];
  __shared__ double sc[12];

  // 1. own xi-line and the upwind neighbours for streaming
  R f[NXI];
  load_line<S, R, NXI>(A.f_in + (size_t)site * NN + t * NXI, f);
  const R cp = op.cph[l], sp = op.sph[l];
  const int sx = (cp > (R)0) ? -1 : 1, sy = (sp > (R)0) ? -1 : 1;
  const int sx1 = y * A.nx + wrap(x + sx, A.nx), sx2 = y * A.nx + wrap(x + 2 * sx, A.nx);
  const int sy1 = wrap(y + sy, A.ny) * A.nx + x, sy2 = wrap(y + 2 * sy, A.ny) * A.nx + x;
  R fx1[NXI], fx2[NXI], fy1[NXI], fy2[NXI];
  load_line<S, R, NXI>(A.f_in + (size_t)sx1 * NN + t * NXI, fx1);
  load_line<S, R, NXI>(A.f_in + (size_t)sx2 * NN + t * NXI, fx2);
  load_line<S, R, NXI>(A.f_in + (size_t)sy1 * NN + t * NXI, fy1);
  load_line<S, R, NXI>(A.f_in + (size_t)sy2 * NN + t * NXI, fy2);
  const double lnM = __ldg(A.lnM_in + site);
  const double ax = (__ldg(A.lnM_in + y * A.nx + wrap(x + 1, A.nx)) -
                     __ldg(A.lnM_in + y * A.nx + wrap(x - 1, A.nx))) * A.inv2dx;
  const double ay = (__ldg(A.lnM_in + wrap(y + 1, A.ny) * A.nx + x) -
                     __ldg(A.lnM_in + wrap(y - 1, A.ny) * A.nx + x)) * A.inv2dx;
  (void)ns;

  // 2. moments of the site
  double mom[7];
  line_moments<R, NXI, NTH, NPH>(op, f, j, l, mom, nullptr);
#pragma unroll
  for (int k = 0; k < NXI; ++k) fs[t * NXI + k] = f[k];
  R Drf[NXI];
#pragma unroll
  for (int kp = 0; kp < NXI; ++kp) {
    R acc = 0;
#pragma unroll
    for (int k = 0; k < NXI; ++k) acc += op.Dr[kp * NXI + k] * f[k];
    Drf[kp] = acc;
  }
  block_sum<7, NL>(mom, red);  // contains __syncthreads: fs visible after it

  // 3. FP64 matching on thread 0 while the other warps do the line operators
  const R milne = A.metric ? (R)(1.0 / A.tau) : (R)0;
  auto line_work = [&](int first, int stride) {
    // polar lines (k', l'): Dth and Dmu along j
    for (int it = t - first; it < NXI * NPH; it += stride) {
      const int kq = it % NXI, lq = it / NXI;
      R g[NTH];
#pragma unroll
      for (int jj = 0; jj < NTH; ++jj) g[jj] = fs[(lq * NTH + jj) * NXI + kq];
      const R Aph = (R)ax * op.cph[lq] + (R)ay * op.sph[lq];
      const R bcoef = -Aph * op.inv_cs[kq];
#pragma unroll
      for (int jp = 0; jp < NTH; ++jp) {
        R dth = 0, dmu = 0;
#pragma unroll
        for (int jj = 0; jj < NTH; ++jj) {
          dth += op.Dth[jp * NTH + jj] * g[jj];
          dmu += op.Dmu[jp * NTH + jj] * g[jj];
        }
        pth[(lq * NTH + jp) * NXI + kq] = milne * dth + bcoef * op.sth_mu[jp] * dmu;
      }
    }
    // azimuthal lines (k'', j''): Dph along l
    for (int it = t - first; it < NXI * NTH; it += stride) {
      const int kq = it % NXI, jq = it / NXI;
      R h[NPH];
#pragma unroll
      for (int ll = 0; ll < NPH; ++ll) h[ll] = fs[(ll * NTH + jq) * NXI + kq];
      const R gcoef = op.inv_cs[kq] / op.sth[jq];
#pragma unroll
      for (int lp = 0; lp < NPH; ++lp) {
        R d = 0;
#pragma unroll
        for (int ll = 0; ll < NPH; ++ll) d += op.Dph[lp * NPH + ll] * h[ll];
        const R Aphp = -(R)ax * op.sph[lp] + (R)ay * op.cph[lp];
        pph[(lp * NTH + jq) * NXI + kq] = gcoef * Aphp * d;
      }
    }
  };
  if (t == 0) {
    SiteState ss;
    int e = match_site(A.eos, red, lnM, A.Tsite[site], A.eta_over_s, false, &ss);
    if (e) atomicOr(A.err, e);
    A.Tsite[site] = ss.T;
    sc[0] = ss.u[0]; sc[1] = ss.u[1]; sc[2] = ss.u[2];
    sc[3] = 1.0 / ss.T;
    sc[4] = ss.Meq;
    sc[5] = exp(lnM);
    sc[6] = ss.inv_tauR;
    sc[7] = ss.D;
    sc[8] = red[0];  // K (no prefactor)
  }
  if (LINE0 > 0) {
    if (t >= LINE0) line_work(LINE0, NL - LINE0);
  } else {
    __syncthreads();
    line_work(0, NL);
  }
  __syncthreads();

  // 4. right-hand side on the own xi-line
  const R ut = (R)sc[0], ux = (R)sc[1], uy = (R)sc[2], invT = (R)sc[3];
  const R Meq = (R)sc[4], M = (R)sc[5], itr = (R)sc[6];
  const R st = op.sth[j], mu2 = op.mu2[j];
  const R vu = st * (cp * ux + sp * uy);               // v_perp . u_perp / sinh(xi)
  const R Aph = (R)ax * cp + (R)ay * sp;
  const R ax_abs = st * (cp < 0 ? -cp : cp) * (R)A.inv2dx;
  const R ay_abs = st * (sp < 0 ? -sp : sp) * (R)A.inv2dx;
  const R wj = op.wj[j];
  const R Z = (R)A.Z;
  R Rn[NXI];
  R sA = 0, sQ = 0, sE = 0;
#pragma unroll
  for (int k = 0; k < NXI; ++k) {
    const int n = t * NXI + k;
    const R s = op.s[k], c = op.c[k];
    const R tv = s * op.inv_c[k];  // tanh(xi)
    const R stream = -tv * (ax_abs * ((R)3 * f[k] - (R)4 * fx1[k] + fx2[k]) +
                            ay_abs * ((R)3 * f[k] - (R)4 * fy1[k] + fy2[k]));
    const R radial = (milne * mu2 + Aph * st * op.c_over_s[k]) * Drf[k];
    const R Eeq = fsqrt<R>(Meq * Meq + M * M * op.s2[k]);
    const R PeqU = ut * Eeq - M * s * vu;
    const R feq = Z * fexp<R>(-PeqU * invT);
    const R pu = c * ut - s * vu;
    const R coll = -(pu * op.inv_c[k]) * (f[k] - feq) * itr;
    const R r = stream + radial + pth[n] + pph[n] + coll;
    Rn[k] = r;
    const R wpu2 = wj * op.ecw[k] * pu * pu;
    sA += wpu2 * r;
    sQ += wpu2 * Drf[k];
    sE += wpu2 * f[k];
  }
  double v3[3] = {(double)sA, (double)sQ, (double)sE};
  __syncthreads();  // red reuse
  block_sum<3, NL>(v3, red);
  if (t == 0) {
    const double D = sc[7], K = sc[8];
    const double g = -D * red[0] / (K + D * (4.0 * red[2] + red[1] - K));
    if (!isfinite(g)) atomicOr(A.err, (int)ERR_NONFINITE);
    sc[9] = g;
    const double dt = A.dtau;
    A.lnM_out[site] = A.mode == 0 ? lnM + dt * g : 0.5 * (__ldg(A.lnM_base + site) + lnM + dt * g);
  }
  __syncthreads();
  const R g = (R)sc[9];
  const R dt = (R)A.dtau;
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
  store_line<S, R, NXI>(A.f_out + (size_t)site * NN + t * NXI, out);
}

// ---------------------------------------------------------------------------
// initial condition and observables
// ---------------------------------------------------------------------------
template <class S, class R, int NXI, int NTH, int NPH>
struct InitArgs {
  const double* eps0;  // GeV/fm^3
  double eps_scale;    // (hbar c)^3: GeV/fm^3 -> GeV^4
  S* f;
  double* lnM;
  double* Tsite;
  int* err;
  EosView eos;
  double Z;
  int family;
  double T0;
  Ops<R, NXI, NTH, NPH> op;
};

template <class S, class R, int NXI, int NTH, int NPH>
__global__ void __launch_bounds__(NTH* NPH)
    init_kernel(const __grid_constant__ InitArgs<S, R, NXI, NTH, NPH> A) {
  constexpr int NL = NTH * NPH;
  constexpr int NN = NL * NXI;
  const int site = blockIdx.x, t = threadIdx.x;
  __shared__ double sc[3];
  if (t == 0) {
    double y = 0.0, target = log(__ldg(A.eps0 + site) * A.eps_scale);
    if (!eos_invert(A.eos, 5, target, log(0.3), &y)) {
      atomicOr(A.err, (int)ERR_EOS);
      y = log(0.3);
    }
    int i0;
    double tt, w[6], dw[6];
    eos_cell(A.eos, y, &i0, &tt);
    lagrange6(tt, w, dw);
    const double T = exp(y);
    const double Meq = eos_field(A.eos, i0, w, 1) * T;
    const double M = A.family == 1 ? A.T0 : Meq;
    A.Tsite[site] = T;
    A.lnM[site] = log(M);
    sc[0] = T; sc[1] = Meq; sc[2] = M;
  }
  __syncthreads();
  const double T = sc[0], Meq = sc[1], M = sc[2];
  R out[NXI];
#pragma unroll
  for (int k = 0; k < NXI; ++k) {
    const double s = (double)A.op.s[k];
    out[k] = (R)(A.Z * exp(-sqrt(Meq * Meq + M * M * s * s) / T));
  }
  store_line<S, R, NXI>(A.f + (size_t)site * NN + t * NXI, out);
}

template <class S, class R, int NXI, int NTH, int NPH>
struct MomArgs {
  const S* f;
  const double* lnM;
  const double* Tsite;
  double* out;  // 8 per site
  int* err;
  EosView eos;
  double eta_over_s;
  Ops<R, NXI, NTH, NPH> op;
};

template <class S, class R, int NXI, int NTH, int NPH>
__global__ void __launch_bounds__(NTH* NPH)
    moments_kernel(const __grid_constant__ MomArgs<S, R, NXI, NTH, NPH> A) {
  constexpr int NL = NTH * NPH;
  constexpr int NN = NL * NXI;
  constexpr int NW = (NL + 31) / 32;
  __shared__ double red[8 * NW];
  const int site = blockIdx.x, t = threadIdx.x;
  const int j = t % NTH, l = t / NTH;
  R f[NXI];
  load_line<S, R, NXI>(A.f + (size_t)site * NN + t * NXI, f);
  double mom[8], tzz;
  double m7[7];
  line_moments<R, NXI, NTH, NPH>(A.op, f, j, l, m7, &tzz);
#pragma unroll
  for (int q = 0; q < 7; ++q) mom[q] = m7[q];
  mom[7] = tzz;
  block_sum<8, NL>(mom, red);
  if (t == 0) {
    const double lnM = A.lnM[site];
    SiteState ss;
    int e = match_site(A.eos, red, lnM, A.Tsite[site], A.eta_over_s, true, &ss);
    if (e) atomicOr(A.err, e);
    const double M = exp(lnM);
    const double pref = M * M * M * M * (1.0 / (2.0 * 3.14159265358979323846 * 3.14159265358979323846));
    const double hc = 0.1973269804, h3 = hc * hc * hc;
    double* o = A.out + (size_t)site * 8;
    o[0] = (ss.eps_kin + ss.B) / h3;
    o[1] = ss.T;
    o[2] = ss.u[0];
    o[3] = ss.u[1];
    o[4] = ss.u[2];
    o[5] = M;
    o[6] = (pref * red[7] - ss.B) / h3;
    o[7] = ss.Meq;
  }
}

}  // namespace rlbk
