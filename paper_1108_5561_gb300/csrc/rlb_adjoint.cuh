// rlb_adjoint.cuh -- discrete adjoint of one Heun stage of the scheme
// (Romatschke, arXiv:1108.5561, Sec. 4.4 with the 2+1D terms of the forward
// kernels), for every storage precision, with the per-node work in FP64 or in
// FP32 arithmetic (the per-site matching adjoint is FP64 in both).
//
// Forward stage at a site (nodes n = (k, j, l), per-line constants as in
// stage_kernel; s = site scalars of the matching of f_in):
//   r_n   = tv_k [nsx Sx_n + nsy Sy_n] + (1/tau) [mu_j^2 (Dr f)_n + (Dth f)_n]
//           + feq_n (fc_n + cc_n) - f_n cc_n
//   Sx_n  = 3 f_n(x) - 4 f_n(x + sx) + f_n(x + 2 sx)     (upwind, periodic)
//   feq_n = Z exp(-invT (ut E_k - M vu s_k)),  E_k = sqrt(Meq^2 + M^2 s_k^2)
//   fc_n  = Gp q1_k / E_k + Hp q2_k + Jp / c_k,  cc_n = itr (ut - tv_k vu)
//   Gp = -invT A1 ut M^2,  Hp = invT A1 M vu,  Jp = invT M (a.u)
//   vu = sth (cp ux + sp uy),  A1 = sth (ax cp + ay sp)
//   g  = -D A / (Kh + D (4E + Q - Kh)),  {A, Q, E} = sum_n wj ecw_k pu_n^2 {r, Dr f, f},
//   pu_n = c_k ut - s_k vu
//   out_n = c [f_n + dtau (r_n + g (Dr f)_n)] (+ (1/2) f_base,n),   c = 1 or 1/2
//   ln M_out = c [ln M + dtau g] (+ (1/2) ln M_base)
// The adjoint runs in three launches: adj_stage1 (per site: the adjoints of r,
// of the site-local uses of f and of the site scalars), adj_match (per site: the
// matching -- Landau eigenproblem and EOS inversion -- differentiated
// implicitly, giving the adjoints of the moments, of ln M and of eta/s) and
// adj_stage3 (per site: the transposed streaming stencil and the grad ln M
// terms gathered from the neighbours, plus the moment weights).
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "rlb_kernels.cuh"

namespace rlbk {

// adjoints of the site scalars, per site
constexpr int kAdjS = 12;
enum : int { AS_UT = 0, AS_UX, AS_UY, AS_INVT, AS_MEQ, AS_M, AS_ITR, AS_D, AS_KH, AS_AX, AS_AY, AS_PAD };

// AR: arithmetic of the per-node adjoint work and type of the per-node adjoint
// arrays (double, or float for the FP32-arithmetic adjoint); the per-site
// quantities (site scalars and their adjoints, the matching) stay FP64.
template <class S, class AR, int NXI, int NTH, int NPH>
struct AdjStageArgs {
  const S* f_in;       // stage input populations
  const double* sc;    // FP64 matching of f_in, kSc per site (AR = double)
  const float* scf;    // FP32 matching of f_in, kSc per site (AR = float)
  const AR* ob;        // adjoint of the stage output populations (per node)
  const double* lb;    // adjoint of the stage output ln M (per site)
  AR* rbar;            // out: adjoint of r (per node)
  AR* fbar;            // out: site-local part of the adjoint of f_in (per node)
  double* sbar;        // out: adjoints of the site scalars (kAdjS per site)
  int* err;            // error word (index checks of debug builds)
  GridMap grid;
  AR milne;            // 1/tau of f_in (Milne) or 0
  AR c;                // 1 (predictor) or 1/2 (corrector)
  AR dtau, inv2dx, Z;
  Ops<AR, NXI, NTH, NPH> op;
};

// sum over the block of NV values of type T, result broadcast to every thread
template <int NV, int NT, class T>
__device__ __forceinline__ void block_sum_t(T (&v)[NV], T* red) {
  constexpr int NW = (NT + 31) / 32;
  if constexpr (NT < 32) {
#pragma unroll
    for (int q = 0; q < NV; ++q) red[threadIdx.x * NV + q] = v[q];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      T a = T(0);
      for (int i = 0; i < NT; ++i) a += red[i * NV + q];
      v[q] = a;
    }
    __syncthreads();
  } else {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
      for (int q = 0; q < NV; ++q) v[q] += __shfl_down_sync(0xffffffffu, v[q], off);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
      for (int q = 0; q < NV; ++q) red[wid * NV + q] = v[q];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      T a = T(0);
      for (int w = 0; w < NW; ++w) a += red[w * NV + q];
      v[q] = a;
    }
    __syncthreads();
  }
}

// FP32 on the 768-node lattice: 7 resident blocks of 96 threads (80 registers,
// 16 bytes of spill; gradients 2.5 % faster than uncapped at 120 registers,
// and 1 % faster than 6 blocks at 96 registers without spill)
template <class S, class AR, int NXI, int NTH, int NPH>
__global__ void __launch_bounds__(NTH* NPH, (sizeof(AR) == 4 && NTH * NPH <= 96) ? 7 : 1)
    adj_stage1(const __grid_constant__ AdjStageArgs<S, AR, NXI, NTH, NPH> A) {
  using T = AR;
  constexpr int NL = NTH * NPH;
  constexpr int NN = NL * NXI;
  // polar sums read VEC staged values per shared-memory load when the lines
  // of one azimuth allow it (rows 16-byte aligned)
  constexpr int VEC = (NTH % (16 / (int)sizeof(T)) == 0) ? 16 / (int)sizeof(T) : 1;
  constexpr int LD = NL + (VEC > 1 ? VEC : 1);
  constexpr int NRED = NL < 32 ? NL : (NL + 31) / 32;
  const T k0 = T(0), k1 = T(1), k2 = T(2), k3 = T(3), k4 = T(4);
  const auto& op = A.op;
  SiteLoc L;
  locate_site(A.grid, blockIdx.x, blockIdx.y, &L);
  const int x = L.x, y = L.y, site = idx_checked(L.site, A.grid.n_sites, A.err), nx = L.nx, ny = L.ny;
  const int t = threadIdx.x, j = t % NTH, l = t / NTH;
  __shared__ __align__(16) T fs[NXI * LD];
  // (D fs)_k along the polar lines of this thread's azimuth: Dth row j (trans
  // false) or column j (trans true)
  auto polar = [&](bool trans, T (&out)[NXI]) {
#pragma unroll
    for (int k = 0; k < NXI; ++k) {
      T a = k0;
      const T* row = fs + k * LD + l * NTH;
#pragma unroll
      for (int jj = 0; jj < NTH; jj += VEC) {
        T v[VEC];
        if constexpr (VEC == 4) {
          const float4 q = *reinterpret_cast<const float4*>(row + jj);
          v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
        } else if constexpr (VEC == 2) {
          const double2 q = *reinterpret_cast<const double2*>(row + jj);
          v[0] = q.x; v[1] = q.y;
        } else {
          v[0] = row[jj];
        }
#pragma unroll
        for (int h = 0; h < VEC; ++h)
          a += (trans ? op.Dth[(jj + h) * NTH + j] : op.Dth[j * NTH + jj + h]) * v[h];
      }
      out[k] += a;
    }
  };
  __shared__ T red[16 * NRED];

  // forward recompute
  T f[NXI], fx1[NXI], fx2[NXI], fy1[NXI], fy2[NXI];
  load_line<S, T, NXI>(A.f_in + (size_t)site * NN + t * NXI, f);
  const T cp = op.cph[l], sp = op.sph[l];
  const int sx = (cp > k0) ? -1 : 1, sy = (sp > k0) ? -1 : 1;
  int x1 = x + sx, x2 = x + 2 * sx, y1 = y + sy, y2 = y + 2 * sy;
  x1 += (x1 < 0) ? nx : (x1 >= nx ? -nx : 0);
  x2 += (x2 < 0) ? nx : (x2 >= nx ? -nx : 0);
  x2 += (x2 < 0) ? nx : (x2 >= nx ? -nx : 0);
  y1 += (y1 < 0) ? ny : (y1 >= ny ? -ny : 0);
  y2 += (y2 < 0) ? ny : (y2 >= ny ? -ny : 0);
  y2 += (y2 < 0) ? ny : (y2 >= ny ? -ny : 0);
  const int ns_all = A.grid.n_sites;
  const int i1 = idx_checked(L.base + y * nx + idx_checked(x1, nx, A.err), ns_all, A.err);
  const int i2 = idx_checked(L.base + y * nx + idx_checked(x2, nx, A.err), ns_all, A.err);
  const int i3 = idx_checked(L.base + idx_checked(y1, ny, A.err) * nx + x, ns_all, A.err);
  const int i4 = idx_checked(L.base + idx_checked(y2, ny, A.err) * nx + x, ns_all, A.err);
  load_line<S, T, NXI>(A.f_in + (size_t)i1 * NN + t * NXI, fx1);
  load_line<S, T, NXI>(A.f_in + (size_t)i2 * NN + t * NXI, fx2);
  load_line<S, T, NXI>(A.f_in + (size_t)i3 * NN + t * NXI, fy1);
  load_line<S, T, NXI>(A.f_in + (size_t)i4 * NN + t * NXI, fy2);
  T q[kScUsed];  // site scalars of the matching of f_in
  if constexpr (std::is_same<T, float>::value) {
#pragma unroll
    for (int i = 0; i < kScUsed; ++i) q[i] = A.scf[(size_t)site * kSc + i];
  } else {
#pragma unroll
    for (int i = 0; i < kScUsed; ++i) q[i] = (T)A.sc[(size_t)site * kSc + i];
  }
  const T ut = q[SC_UT], ux = q[SC_UX], uy = q[SC_UY], invT = q[SC_INVT], Meq = q[SC_MEQ];
  const T M = q[SC_M], itr = q[SC_ITR], D = q[SC_D], Kh = q[SC_KH], ax = q[SC_AX], ay = q[SC_AY];
  const T M2 = M * M;
#pragma unroll
  for (int k = 0; k < NXI; ++k) fs[k * LD + t] = f[k];
  T Drf[NXI];
#pragma unroll
  for (int kp = 0; kp < NXI; ++kp) {
    T a = k0;
#pragma unroll
    for (int k = 0; k < NXI; ++k) a += op.Dr[kp * NXI + k] * f[k];
    Drf[kp] = a;
  }
  __syncthreads();
  T pth[NXI];  // (Dth f) on the own line
#pragma unroll
  for (int k = 0; k < NXI; ++k) pth[k] = k0;
  polar(false, pth);
  const T st = op.sth[j], mu2 = op.mu2[j], wj = op.wj[j];
  const T vu = st * (cp * ux + sp * uy), A1 = st * (ax * cp + ay * sp), au = ax * ux + ay * uy;
  const T nsx = -st * fabs(cp) * A.inv2dx, nsy = -st * fabs(sp) * A.inv2dx;
  const T Gp = -invT * A1 * ut * M2, Hp = invT * A1 * M * vu, Jp = invT * M * au;
  // iE = 1/E_eq: one division per node, the other quotients become products
  T E[NXI], iE[NXI], feq[NXI], cc[NXI], fc[NXI], r[NXI], pu[NXI], wp[NXI];
  T sums[3] = {k0, k0, k0};
#pragma unroll
  for (int k = 0; k < NXI; ++k) {
    const T s = op.s[k], c = op.c[k], tv = op.tv[k];
    // FP32 adjoint: the hardware reciprocal square root and exponential (a
    // few ulp; the linearisation point needs no more), FP64: the correctly
    // rounded functions
    if constexpr (std::is_same<T, float>::value) {
      const float e2 = Meq * Meq + M2 * op.s2[k];
      iE[k] = rsqrtf(e2);
      E[k] = e2 * iE[k];
      feq[k] = A.Z * __expf(-invT * (ut * E[k] - M * vu * s));
    } else {
      E[k] = sqrt(Meq * Meq + M2 * op.s2[k]);
      iE[k] = k1 / E[k];
      feq[k] = A.Z * exp(-invT * (ut * E[k] - M * vu * s));
    }
    cc[k] = itr * (ut - tv * vu);
    fc[k] = Gp * op.q1[k] * iE[k] + Hp * op.q2[k] + Jp * op.inv_c[k];
    const T Sx = k3 * f[k] - k4 * fx1[k] + fx2[k], Sy = k3 * f[k] - k4 * fy1[k] + fy2[k];
    r[k] = tv * (nsx * Sx + nsy * Sy) + A.milne * (mu2 * Drf[k] + pth[k]) + feq[k] * (fc[k] + cc[k]) -
           f[k] * cc[k];
    pu[k] = c * ut - s * vu;
    wp[k] = wj * op.ecw[k] * pu[k] * pu[k];
    sums[0] += wp[k] * r[k];
    sums[1] += wp[k] * Drf[k];
    sums[2] += wp[k] * f[k];
  }
  // site sums and sum_n ob_n (Dr f)_n in one reduction
  T ob[NXI];
  load_line<T, T, NXI>(A.ob + (size_t)site * NN + t * NXI, ob);
  T red4[4] = {sums[0], sums[1], sums[2], k0};
#pragma unroll
  for (int k = 0; k < NXI; ++k) red4[3] += ob[k] * Drf[k];
  block_sum_t<4, NL>(red4, red);
  const T SA = red4[0], SQ = red4[1], SE = red4[2];
  const T den = Kh + D * (k4 * SE + SQ - Kh);
  const T g = (D == k0) ? k0 : -D * SA / den;

  // adjoint of g and of its sums (every thread, identical values)
  const T cdt = A.c * A.dtau;
  const T gbar = cdt * (red4[3] + (T)A.lb[site]);
  T Abar = k0, Qbar = k0, Ebar = k0, Dbar = k0, Khbar = k0;
  if (D != k0) {
    const T denbar = D * SA / (den * den) * gbar;
    Abar = -D / den * gbar;
    Dbar = -SA / den * gbar + denbar * (k4 * SE + SQ - Kh);
    Ebar = denbar * k4 * D;
    Qbar = denbar * D;
    Khbar = denbar * (k1 - D);
  }

  // per node
  T rb[NXI], Drfb[NXI], fb[NXI];
  T b_ut = k0, b_vu = k0, b_invT = k0, b_Meq = k0, b_M = k0, b_itr = k0;
  T b_Gp = k0, b_Hp = k0, b_Jp = k0;
#pragma unroll
  for (int k = 0; k < NXI; ++k) {
    const T s = op.s[k], c = op.c[k], tv = op.tv[k];
    const T o = ob[k];
    rb[k] = cdt * o + Abar * wp[k];
    Drfb[k] = cdt * g * o + Qbar * wp[k] + A.milne * mu2 * rb[k];
    fb[k] = A.c * o + Ebar * wp[k] - rb[k] * cc[k] + k3 * tv * (nsx + nsy) * rb[k];
    // pu through the weights of the sums
    const T wpb = Abar * r[k] + Qbar * Drf[k] + Ebar * f[k];
    const T pub = k2 * wj * op.ecw[k] * pu[k] * wpb;
    b_ut += c * pub;
    b_vu -= s * pub;
    // feq, cc, fc
    const T feqb = rb[k] * (fc[k] + cc[k]);
    const T fcb = rb[k] * feq[k];
    const T ccb = rb[k] * (feq[k] - f[k]);
    const T argb = feqb * feq[k];
    b_invT -= argb * (ut * E[k] - M * vu * s);
    b_ut -= argb * invT * E[k];
    T Eb = -argb * invT * ut;
    b_M += argb * invT * vu * s;
    b_vu += argb * invT * M * s;
    b_itr += ccb * (ut - tv * vu);
    b_ut += ccb * itr;
    b_vu -= ccb * itr * tv;
    b_Gp += fcb * op.q1[k] * iE[k];
    Eb -= fcb * Gp * op.q1[k] * iE[k] * iE[k];
    b_Hp += fcb * op.q2[k];
    b_Jp += fcb * op.inv_c[k];
    b_Meq += Eb * Meq * iE[k];
    b_M += Eb * M * op.s2[k] * iE[k];
  }
  T b_A1 = k0, b_au = k0;
  b_invT -= b_Gp * A1 * ut * M2;
  b_A1 -= b_Gp * invT * ut * M2;
  b_ut -= b_Gp * invT * A1 * M2;
  b_M -= b_Gp * invT * A1 * ut * k2 * M;
  b_invT += b_Hp * A1 * M * vu;
  b_A1 += b_Hp * invT * M * vu;
  b_M += b_Hp * invT * A1 * vu;
  b_vu += b_Hp * invT * A1 * M;
  b_invT += b_Jp * M * au;
  b_M += b_Jp * invT * au;
  b_au += b_Jp * invT * M;
  T sb[9];
  sb[0] = b_ut;
  sb[1] = b_vu * st * cp + b_au * ax;   // ux
  sb[2] = b_vu * st * sp + b_au * ay;   // uy
  sb[3] = b_invT;
  sb[4] = b_Meq;
  sb[5] = b_M;
  sb[6] = b_itr;
  sb[7] = b_A1 * st * cp + b_au * ux;   // ax
  sb[8] = b_A1 * st * sp + b_au * uy;   // ay

  // f through Dr^T on the own line and Dth^T along the polar lines
#pragma unroll
  for (int k = 0; k < NXI; ++k) {
    T a = k0;
#pragma unroll
    for (int kp = 0; kp < NXI; ++kp) a += op.Dr[kp * NXI + k] * Drfb[kp];
    fb[k] += a;
  }
#pragma unroll
  for (int k = 0; k < NXI; ++k) fs[k * LD + t] = A.milne * rb[k];  // adjoint of (Dth f)
  __syncthreads();
  polar(true, fb);
  store_line<T, T, NXI>(A.rbar + (size_t)site * NN + t * NXI, rb);
  store_line<T, T, NXI>(A.fbar + (size_t)site * NN + t * NXI, fb);
  // site scalar adjoints
  T s9[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) s9[i] = sb[i];
  block_sum_t<9, NL>(s9, red);
  if (t == 0) {
    double* o = A.sbar + (size_t)site * kAdjS;
    o[AS_UT] = s9[0]; o[AS_UX] = s9[1]; o[AS_UY] = s9[2]; o[AS_INVT] = s9[3]; o[AS_MEQ] = s9[4];
    o[AS_M] = s9[5]; o[AS_ITR] = s9[6]; o[AS_AX] = s9[7]; o[AS_AY] = s9[8];
    o[AS_D] = Dbar; o[AS_KH] = Khbar; o[AS_PAD] = 0.0;
  }
}

// ---------------------------------------------------------------------------
// adjoint of the matching of one site (FP64): from the adjoints of the site
// scalars to those of the moments (mbar, kMom per site), of ln M (local part,
// lbar) and of eta/s (ebar)
// ---------------------------------------------------------------------------
struct AdjMatchArgs {
  const double* mom;   // FP64 moments of f_in, kMom per site (when momf is null)
  const float* momf;   // or their FP32 partial sums, kMom x kMomParts per site
  const double* Tstart;  // Newton start of the EOS inversion (the matching's T)
  const float* scf;    // FP32 adjoint: the FP32 matching of f_in (u and T taken from it)
  const double* lnM;
  const double* sbar;
  double* mbar;
  double* lbar;
  double* ebar;        // per-site eta/s adjoint, accumulated over the stages
  int* err;
  EosView eos;
  GridMap grid;
  int ns;
};

// value and d/dy (y = ln T) of a table field
__device__ __forceinline__ void eos_field_dy(const EosView& E, double y, int field, double* v, double* dv) {
  int i0;
  double t, w[6], dw[6];
  if (!eos_cell(E, y, &i0, &t)) { *v = 0.0; *dv = 0.0; return; }
  lagrange6(t, w);
  lagrange6_d(t, dw);
  double a = 0.0, b = 0.0;
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    const double tv = __ldg(E.tab + (size_t)(i0 - 2 + m) * 8 + field);
    a += w[m] * tv;
    b += dw[m] * tv;
  }
  *v = a;
  *dv = b * E.inv_h;
}

// solve the 4x4 system M x = b by Gaussian elimination with partial pivoting
__device__ __forceinline__ bool solve4(double (&Mx)[4][4], double (&b)[4]) {
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    int p = c;
    for (int r = c + 1; r < 4; ++r)
      if (fabs(Mx[r][c]) > fabs(Mx[p][c])) p = r;
    if (!(fabs(Mx[p][c]) > 0.0)) return false;
    if (p != c) {
      for (int k = 0; k < 4; ++k) { const double tmp = Mx[c][k]; Mx[c][k] = Mx[p][k]; Mx[p][k] = tmp; }
      const double tb = b[c]; b[c] = b[p]; b[p] = tb;
    }
    for (int r = c + 1; r < 4; ++r) {
      const double fct = Mx[r][c] / Mx[c][c];
      for (int k = c; k < 4; ++k) Mx[r][k] -= fct * Mx[c][k];
      b[r] -= fct * b[c];
    }
  }
  for (int c = 3; c >= 0; --c) {
    double a = b[c];
    for (int k = c + 1; k < 4; ++k) a -= Mx[c][k] * b[k];
    b[c] = a / Mx[c][c];
  }
  return true;
}

__global__ void __launch_bounds__(128) adj_match(const AdjMatchArgs A) {
  const int site = blockIdx.x * blockDim.x + threadIdx.x;
  if (site >= A.ns) return;
  double m[kMom];
  if (A.momf) {  // FP32 partials summed in FP64 (exact up to one FP64 rounding per sum)
    const float4* p = reinterpret_cast<const float4*>(A.momf + (size_t)site * kMom * kMomParts);
#pragma unroll
    for (int i = 0; i < kMom; ++i) {
      const float4 v = __ldg(p + i);
      m[i] = ((double)v.x + (double)v.y) + ((double)v.z + (double)v.w);
    }
  } else {
#pragma unroll
    for (int i = 0; i < kMom; ++i) m[i] = A.mom[(size_t)site * kMom + i];
  }
  const double lnM = A.lnM[site], M = exp(lnM);
  const double pref = M * M * M * M * (1.0 / (2.0 * 3.14159265358979323846 * 3.14159265358979323846));
  double tm[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) tm[i] = pref * m[1 + i];
  double u[3], eps;
  int err = 0;
  double y = 0.0;
  if (A.scf) {
    // FP32 adjoint: the velocity and temperature of the FP32 matching of the
    // same moments; eps as the Rayleigh quotient u_mu T^{mu nu} u_nu
    const float* q = A.scf + (size_t)site * kSc;
    u[0] = q[SC_UT]; u[1] = q[SC_UX]; u[2] = q[SC_UY];
    const double g0 = u[0], g1 = -u[1], g2 = -u[2];
    eps = tm[0] * g0 * g0 + 2.0 * (tm[1] * g0 * g1 + tm[2] * g0 * g2 + tm[4] * g1 * g2) + tm[3] * g1 * g1 +
          tm[5] * g2 * g2;
    y = log((double)q[SC_T]);
  } else {
    if (!landau3(tm, u, &eps)) err |= ERR_LANDAU;
    const double T0 = A.Tstart ? A.Tstart[site] : 0.3;
    if (!eos_invert(A.eos, EOS_E, eps, log(T0 > 0.0 ? T0 : 0.3), &y)) err |= ERR_EOS;
  }
  const double T = exp(y);
  double e, de, xv, dx, Dv, dD, ih, dih;
  eos_field_dy(A.eos, y, EOS_E, &e, &de);
  eos_field_dy(A.eos, y, EOS_X, &xv, &dx);
  eos_field_dy(A.eos, y, EOS_D, &Dv, &dD);
  eos_field_dy(A.eos, y, EOS_INVH, &ih, &dih);
  const double* sb = A.sbar + (size_t)site * kAdjS;
  const EventInfo& ev = A.grid.ev[event_of_site(A.grid, site)];
  const double eta = ev.eta_over_s;
  // T from e(T) = eps: Tbar -> epsbar; scalars: invT = 1/T, Meq = x T,
  // D = D(T), itr = (1/h)(T) / eta (d/dT = (1/T) d/dy)
  const double Tbar = -sb[AS_INVT] / (T * T) + sb[AS_MEQ] * (xv + dx) + sb[AS_D] * dD / T +
                      sb[AS_ITR] * dih / (T * eta);
  A.ebar[site] += -sb[AS_ITR] * ih / (eta * eta);  // summed over the stages; over the sites at the end
  const double epsbar = Tbar * T / de;  // de/dT = de/dy / T
  // Landau: F_mu = T^{mu l} (g u)_l - eps u^mu = 0, F_3 = u.g.u - 1 = 0 in
  // z = (u, eps); lambda = J^{-T} zbar, Tbar^{ab} = -lambda_a (g u)_b
  const double gu[3] = {u[0], -u[1], -u[2]};
  const double Tm[3][3] = {{tm[0], tm[1], tm[2]}, {tm[1], tm[3], tm[4]}, {tm[2], tm[4], tm[5]}};
  double Jt[4][4];  // J transposed
#pragma unroll
  for (int mu = 0; mu < 3; ++mu)
#pragma unroll
    for (int nu = 0; nu < 3; ++nu) {
      // J[mu][nu] = T^{mu l} g_{l nu} - eps delta
      const double gnu = nu == 0 ? 1.0 : -1.0;
      Jt[nu][mu] = Tm[mu][nu] * gnu - (mu == nu ? eps : 0.0);
    }
#pragma unroll
  for (int mu = 0; mu < 3; ++mu) {
    Jt[3][mu] = -u[mu];      // J[mu][3]
    Jt[mu][3] = 2.0 * gu[mu];  // J[3][mu]
  }
  Jt[3][3] = 0.0;
  double lam[4] = {sb[AS_UT], sb[AS_UX], sb[AS_UY], epsbar};
  if (!solve4(Jt, lam)) err |= ERR_LANDAU;
  // symmetric moment adjoints: tm = {T00, T01, T02, T11, T12, T22}
  double tb[6];
  tb[0] = -lam[0] * gu[0];
  tb[1] = -(lam[0] * gu[1] + lam[1] * gu[0]);
  tb[2] = -(lam[0] * gu[2] + lam[2] * gu[0]);
  tb[3] = -lam[1] * gu[1];
  tb[4] = -(lam[1] * gu[2] + lam[2] * gu[1]);
  tb[5] = -lam[2] * gu[2];
  double* mb = A.mbar + (size_t)site * kMom;
  mb[0] = sb[AS_KH];
  double lb = sb[AS_M] * M;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    mb[1 + i] = pref * tb[i];
    lb += 4.0 * tb[i] * tm[i];
  }
  mb[7] = 0.0;
  A.lbar[site] = lb;
  if (err) atomicOr(A.err, err);
}

// ---------------------------------------------------------------------------
// assembly: adjoint of f_in (per node) and of ln M_in (per site)
// ---------------------------------------------------------------------------
template <class AR, int NXI, int NTH, int NPH>
struct AdjAssembleArgs {
  const AR* fbar;       // site-local part (adj_stage1)
  const AR* rbar;       // adjoint of r (neighbours gathered)
  const double* mbar;   // moment adjoints (adj_match)
  const double* sbar;   // scalar adjoints (grad ln M gathered)
  const double* lbar;   // ln M local part (adj_match)
  const double* lb;     // adjoint of the stage output ln M
  AR* fout;             // adjoint of f_in
  double* lout;         // adjoint of ln M_in
  AR acc;               // nonzero: fout, lout += acc x their previous values (in place)
  int* err;             // error word (index checks of debug builds)
  GridMap grid;
  double c, inv2dx;
  AR inv2dx_t;          // inv2dx in the arithmetic type
  Ops<AR, NXI, NTH, NPH> op;
};

template <class AR, int NXI, int NTH, int NPH>
__global__ void __launch_bounds__(NTH* NPH)
    adj_stage3(const __grid_constant__ AdjAssembleArgs<AR, NXI, NTH, NPH> A) {
  using T = AR;
  constexpr int NL = NTH * NPH;
  constexpr int NN = NL * NXI;
  const auto& op = A.op;
  SiteLoc L;
  locate_site(A.grid, blockIdx.x, blockIdx.y, &L);
  const int x = L.x, y = L.y, site = idx_checked(L.site, A.grid.n_sites, A.err), nx = L.nx, ny = L.ny;
  const int t = threadIdx.x, j = t % NTH, l = t / NTH;
  const T cp = op.cph[l], sp = op.sph[l], st = op.sth[j], wj = op.wj[j];
  const T i2dx = A.inv2dx_t;
  const T nsx = -st * fabs(cp) * i2dx, nsy = -st * fabs(sp) * i2dx;
  // downwind neighbours: the forward stencil of site i - s uses f(i) with -4,
  // that of i - 2 s with +1 (s = the upwind offset)
  const int sx = (cp > T(0)) ? -1 : 1, sy = (sp > T(0)) ? -1 : 1;
  auto wrap = [](int i, int n) {
    i += (i < 0) ? n : (i >= n ? -n : 0);
    return i + ((i < 0) ? n : (i >= n ? -n : 0));
  };
  const int ns_all = A.grid.n_sites;
  const size_t d1x = idx_checked(L.base + y * nx + idx_checked(wrap(x - sx, nx), nx, A.err), ns_all, A.err);
  const size_t d2x = idx_checked(L.base + y * nx + idx_checked(wrap(x - 2 * sx, nx), nx, A.err), ns_all, A.err);
  const size_t d1y = idx_checked(L.base + idx_checked(wrap(y - sy, ny), ny, A.err) * nx + x, ns_all, A.err);
  const size_t d2y = idx_checked(L.base + idx_checked(wrap(y - 2 * sy, ny), ny, A.err) * nx + x, ns_all, A.err);
  // the moment adjoints of the site, converted once per CTA (a conversion from
  // FP64 occupies the FP64 pipe: per thread it dominated the kernel)
  __shared__ T msh[8];
  if (t < 7) msh[t] = (T)A.mbar[(size_t)site * kMom + t];
  __syncthreads();
  T m[7];
#pragma unroll
  for (int i = 0; i < 7; ++i) m[i] = msh[i];
  const T w0 = wj, w1 = wj * st * cp, w1y = wj * st * sp, w3x = wj * st * st * cp * cp;
  const T w3xy = wj * st * st * cp * sp, w3y = wj * st * st * sp * sp;
  // the per-line moment coefficients of the four radial weights
  const T c0 = m[0] * w0, c2 = m[1] * w0, c1 = m[2] * w1 + m[3] * w1y, c3 = m[4] * w3x + m[5] * w3xy + m[6] * w3y;
  T fb[NXI], r1x[NXI], r2x[NXI], r1y[NXI], r2y[NXI], fo[NXI];
  load_line<T, T, NXI>(A.fbar + (size_t)site * NN + t * NXI, fb);
  load_line<T, T, NXI>(A.rbar + d1x * NN + t * NXI, r1x);
  load_line<T, T, NXI>(A.rbar + d2x * NN + t * NXI, r2x);
  load_line<T, T, NXI>(A.rbar + d1y * NN + t * NXI, r1y);
  load_line<T, T, NXI>(A.rbar + d2y * NN + t * NXI, r2y);
  const T m4 = T(-4);
#pragma unroll
  for (int k = 0; k < NXI; ++k) {
    const T tv = op.tv[k];
    const T a = tv * nsx, b = tv * nsy;
    T v = fb[k];
    v += a * (m4 * r1x[k] + r2x[k]);
    v += b * (m4 * r1y[k] + r2y[k]);
    // moment weights: K, T00, T01, T02, T11, T12, T22 (ecw-scaled radial parts)
    v += c0 * op.w0[k] + c2 * op.w2[k] + c1 * op.w1[k] + c3 * op.w3[k];
    fo[k] = v;
  }
  if (A.acc != T(0)) {  // the adjoint already there, scaled (the corrector's base term), plus this one
    T prev[NXI];
    load_line<T, T, NXI>(A.fout + (size_t)site * NN + t * NXI, prev);
#pragma unroll
    for (int k = 0; k < NXI; ++k) fo[k] = A.acc * prev[k] + fo[k];
  }
  store_line<T, T, NXI>(A.fout + (size_t)site * NN + t * NXI, fo);
  if (t == 0) {
    const double* sb = A.sbar;
    const int xm = wrap(x - 1, nx), xp = wrap(x + 1, nx), ym = wrap(y - 1, ny), yp = wrap(y + 1, ny);
    // ln M(i) enters a_x(i -/+ 1) = (ln M(i) - ln M(i -/+ 2)) / (2 dx) with sign +/-
    const int ns_all = A.grid.n_sites;
    const size_t sxm = idx_checked(L.base + y * nx + xm, ns_all, A.err), sxp = idx_checked(L.base + y * nx + xp, ns_all, A.err);
    const size_t sym = idx_checked(L.base + ym * nx + x, ns_all, A.err), syp = idx_checked(L.base + yp * nx + x, ns_all, A.err);
    const double gx = sb[sxm * kAdjS + AS_AX] - sb[sxp * kAdjS + AS_AX];
    const double gy = sb[sym * kAdjS + AS_AY] - sb[syp * kAdjS + AS_AY];
    const double v = A.c * A.lb[site] + A.lbar[site] + A.inv2dx * (gx + gy);
    A.lout[site] = A.acc != T(0) ? (double)A.acc * A.lout[site] + v : v;
  }
}

// adjoint seed of v2 = NUM / DEN (per-site partials part[4 i + 2], part[4 i + 3]
// = M^3/(2 pi^2) {num_i, den_i}, grid sums in sums[2], sums[3]):
//   fbar_n = M^3/(2 pi^2) w_n s_k sth_j (cos 2phi_l / DEN - NUM / DEN^2)
//   lbar   = 3 (part_num / DEN - part_den NUM / DEN^2)
template <class S, class AR, int NXI, int NTH, int NPH>
struct SeedArgs {
  const double* lnM;
  const double* part;
  const double* tot;   // {.., .., NUM, DEN}
  AR* fbar;
  double* lbar;
  Ops<double, NXI, NTH, NPH> op;
};

template <class S, class AR, int NXI, int NTH, int NPH>
__global__ void __launch_bounds__(NTH* NPH) adj_seed_v2(const __grid_constant__ SeedArgs<S, AR, NXI, NTH, NPH> A) {
  constexpr int NL = NTH * NPH, NN = NL * NXI;
  const int site = blockIdx.x, t = threadIdx.x, j = t % NTH, l = t / NTH;
  const auto& op = A.op;
  const double NUM = A.tot[2], DEN = A.tot[3];
  const double bn = 1.0 / DEN, bd = -NUM / (DEN * DEN);
  const double M = exp(A.lnM[site]);
  const double m3 = M * M * M / (2.0 * 3.14159265358979323846 * 3.14159265358979323846);
  const double cp = op.cph[l], sp = op.sph[l];
  const double wl = m3 * op.wj[j] * op.sth[j] * (bn * (cp * cp - sp * sp) + bd);
  AR* o = A.fbar + (size_t)site * NN + t * NXI;
#pragma unroll
  for (int k = 0; k < NXI; ++k) o[k] = (AR)(wl * op.ecw[k] * op.s[k]);
  if (t == 0) A.lbar[site] = 3.0 * (bn * A.part[(size_t)site * 4 + 2] + bd * A.part[(size_t)site * 4 + 3]);
}

// adjoint of the initial condition (Sec. 4.4: f = Z exp(-M cosh xi / T) at
// rest, M = x(T) T, eps_EOS(T) = eps0): from the adjoints of f and ln M of the
// initial state to that of eps0 [GeV/fm^3], per site
template <class S, class AR, int NXI, int NTH, int NPH>
struct AdjIcArgs {
  const double* eps0;
  const AR* fbar;
  const double* lbar;
  double* epsbar;
  int* err;
  EosView eos;
  double eps_scale, Z;
  Ops<double, NXI, NTH, NPH> op;
};

template <class S, class AR, int NXI, int NTH, int NPH>
__global__ void __launch_bounds__(NTH* NPH) adj_ic(const __grid_constant__ AdjIcArgs<S, AR, NXI, NTH, NPH> A) {
  constexpr int NL = NTH * NPH, NN = NL * NXI;
  constexpr int NRED = NL < 32 ? NL : (NL + 31) / 32;
  __shared__ double red[NRED * 2];
  __shared__ double sT[2];
  const int site = blockIdx.x, t = threadIdx.x;
  const auto& op = A.op;
  if (t == 0) {
    double y = 0.0;
    if (!eos_invert(A.eos, EOS_EPS, A.eps0[site] * A.eps_scale, log(0.3), &y)) atomicOr(A.err, (int)ERR_EOS);
    double xv, dx;
    eos_field_dy(A.eos, y, EOS_X, &xv, &dx);
    sT[0] = y;
    sT[1] = xv;
  }
  __syncthreads();
  const double xv = sT[1];
  const AR* fb = A.fbar + (size_t)site * NN + t * NXI;
  double a[1] = {0.0};
#pragma unroll
  for (int k = 0; k < NXI; ++k) {
    const double fk = A.Z * exp(-xv * op.c[k]);
    a[0] += (double)fb[k] * fk * (-op.c[k]);  // d f / d x
  }
  block_sum_t<1, NL>(a, red);
  if (t == 0) {
    const double y = sT[0], T = exp(y);
    double xx, dx, ee, de;
    eos_field_dy(A.eos, y, EOS_X, &xx, &dx);
    eos_field_dy(A.eos, y, EOS_EPS, &ee, &de);
    // x(T), ln M = ln x + ln T;  d/dT = (1/T) d/dy
    const double Tbar = a[0] * dx / T + A.lbar[site] * (dx / xx + 1.0) / T;
    A.epsbar[site] = Tbar * T / de * A.eps_scale;
  }
}

// out[i] = sum_s basis[i * ns + s] epsbar[s]  (one block per row, fixed order)
__global__ void __launch_bounds__(1024) project_kernel(const double* basis, const double* v, size_t ns, double* out) {
  __shared__ double red[32];
  const double* b = basis + (size_t)blockIdx.x * ns;
  double a[1] = {0.0};
  for (size_t s = threadIdx.x; s < ns; s += 1024) a[0] += b[s] * v[s];
  warp_sum<1>(a);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a[0];
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 32; ++w) s += red[w];
    out[blockIdx.x] = s;
  }
}

// out[i] = (T) in[i]
template <class T>
__global__ void convert_kernel(T* out, const double* in, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (T)in[i];
}

// sum of n doubles into out[0] (one block, fixed order)
__global__ void __launch_bounds__(1024) sum_kernel(const double* in, size_t n, double* out, int accumulate) {
  __shared__ double red[32];
  double a[1] = {0.0};
  for (size_t i = threadIdx.x; i < n; i += 1024) a[0] += in[i];
  warp_sum<1>(a);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a[0];
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 32; ++w) s += red[w];
    out[0] = accumulate ? out[0] + s : s;
  }
}

}  // namespace rlbk
