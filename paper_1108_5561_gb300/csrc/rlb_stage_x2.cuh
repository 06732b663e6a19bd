// rlb_stage_x2.cuh -- the fused stream-collide stage in FP32 arithmetic with
// packed pairs of radial nodes (FFMA2 / FADD2 / FMUL2, sm_100 and later).
//
// Same right-hand side as stage_kernel (Romatschke, arXiv:1108.5561, Sec. 4.3,
// Eq. Bmilne with the BGK term of Sec. 4.1, Heun stages of Sec. 4.4):
//   rhs = -V.grad f + (1/tau) [mu^2 Dr f + Dth f] + g Dr f + T_M f_eq
//         - ((P.U)/E) (f - f_eq) / tau_R
// Each thread owns one (theta_j, phi_l) line of radial nodes and holds it as
// NXI/2 float2 pairs (xi_2p, xi_2p+1), so every per-node operation acts on two
// nodes per instruction.  The per-node constants are stored as the matching
// pairs in parameter space; the per-line scalars are broadcast to pairs once.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "rlb_kernels.cuh"

namespace rlbk {

__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// Per-run constants of the paired kernel (parameter space).
template <int NXI, int NTH, int NPH>
struct OpsX2 {
  static constexpr int NP = NXI / 2;
  float2 Drb[NXI * NP];    // [k * NP + p] = (Dr[2p][k], Dr[2p+1][k])
  float2 Dthb[NTH * NTH];  // [jp * NTH + jj] = Dth[jp][jj] in both halves
  float2 tv[NP], s[NP], q2[NP], ic[NP];  // tanh, sinh, sinh^2/cosh, 1/cosh
  float2 Cw[NP], Sw[NP];                 // cosh sqrt(ecw), sinh sqrt(ecw)
  float2 w0[NP], w1[NP], w2[NP], w3[NP];  // ecw * {1, c s, c^2, s^2}
  float s2[NXI], q1[NXI];                 // sinh^2, sinh (sinh^2 + 1)/cosh
  float sth[NTH], mu[NTH], mu2[NTH], wj[NTH];
  float cph[NPH], sph[NPH];
};

template <class S, int NXI, int NTH, int NPH>
struct StageArgsX2 {
  const S* f_in;
  const double* lnM_in;
  const float* scf;       // FP32 matching of f_in, kSc per site
  const S* f_base;        // corrector: populations at the start of the step
  const double* lnM_base;
  S* f_out;
  double* lnM_out;
  float* momf_out;        // moments of f_out: one partial sum per warp (kMomParts slots)
  int* err;
  GridMap grid;
  const Clock* clock;     // proper time of f_in
  int milne_on;           // Milne metric (1/tau terms) or Minkowski
  int mode;               // 0 predictor, 1 corrector
  double dtau;
  float dtau_r, inv2dx_r, log2Z;
  OpsX2<NXI, NTH, NPH> op;
};

// 32 bytes per thread in one 256-bit access (p 32-byte aligned: a line of 8
// FP32 values at a multiple of 8 elements in a 256-byte aligned array).  With
// two 128-bit accesses per line, each touches all 32 sectors of the warp's
// 1 KB and the second finds them in L1: twice the L1 requests and sector
// traffic (the 256-bit form measured 9 % faster on the stage).
__device__ __forceinline__ void ldg_v8(const float* p, float2& a, float2& b, float2& c, float2& d) {
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(a.x), "=f"(a.y), "=f"(b.x), "=f"(b.y), "=f"(c.x), "=f"(c.y), "=f"(d.x), "=f"(d.y)
      : "l"(p));
}
__device__ __forceinline__ void stg_v8(float* p, float2 a, float2 b, float2 c, float2 d) {
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(a.x), "f"(a.y), "f"(b.x),
               "f"(b.y), "f"(c.x), "f"(c.y), "f"(d.x), "f"(d.y)
               : "memory");
}

// line of NXI stored values -> NXI/2 FP32 pairs (vector loads where aligned)
template <class S, int NP>
__device__ __forceinline__ void load_pairs(const S* __restrict__ p, float2 (&v)[NP]) {
  if constexpr (sizeof(S) == 4) {
    if constexpr (NP % 4 == 0) {
#pragma unroll
      for (int i = 0; i < NP / 4; ++i) ldg_v8(p + 8 * i, v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    } else if constexpr (NP % 2 == 0) {
      const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
      for (int i = 0; i < NP / 2; ++i) {
        const float4 a = __ldg(q + i);
        v[2 * i] = make_float2(a.x, a.y);
        v[2 * i + 1] = make_float2(a.z, a.w);
      }
    } else {
      const float2* q = reinterpret_cast<const float2*>(p);
#pragma unroll
      for (int i = 0; i < NP; ++i) v[i] = __ldg(q + i);
    }
  } else {
    static_assert(sizeof(S) == 2, "FP32 or BF16 storage");
    if constexpr (NP % 4 == 0) {
      const uint4* q = reinterpret_cast<const uint4*>(p);
#pragma unroll
      for (int i = 0; i < NP / 4; ++i) {
        uint4 a = __ldg(q + i);
        const __nv_bfloat162* b = reinterpret_cast<const __nv_bfloat162*>(&a);
#pragma unroll
        for (int h = 0; h < 4; ++h) v[4 * i + h] = __bfloat1622float2(b[h]);
      }
    } else {
      const __nv_bfloat162* q = reinterpret_cast<const __nv_bfloat162*>(p);
#pragma unroll
      for (int i = 0; i < NP; ++i) v[i] = __bfloat1622float2(q[i]);
    }
  }
}

// FP32 pairs -> storage; returns in v what was stored (rounded to S)
template <class S, int NP>
__device__ __forceinline__ void store_pairs(S* __restrict__ p, float2 (&v)[NP]) {
  if constexpr (sizeof(S) == 4) {
    if constexpr (NP % 4 == 0) {
#pragma unroll
      for (int i = 0; i < NP / 4; ++i) stg_v8(p + 8 * i, v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    } else if constexpr (NP % 2 == 0) {
      float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
      for (int i = 0; i < NP / 2; ++i) q[i] = make_float4(v[2 * i].x, v[2 * i].y, v[2 * i + 1].x, v[2 * i + 1].y);
    } else {
      float2* q = reinterpret_cast<float2*>(p);
#pragma unroll
      for (int i = 0; i < NP; ++i) q[i] = v[i];
    }
  } else {
    __nv_bfloat162 b[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      b[i] = __float22bfloat162_rn(v[i]);
      v[i] = __bfloat1622float2(b[i]);
    }
    if constexpr (NP % 4 == 0) {
      uint4* q = reinterpret_cast<uint4*>(p);
#pragma unroll
      for (int i = 0; i < NP / 4; ++i) {
        uint4 u;
        u.x = *reinterpret_cast<const unsigned*>(&b[4 * i]);
        u.y = *reinterpret_cast<const unsigned*>(&b[4 * i + 1]);
        u.z = *reinterpret_cast<const unsigned*>(&b[4 * i + 2]);
        u.w = *reinterpret_cast<const unsigned*>(&b[4 * i + 3]);
        q[i] = u;
      }
    } else {
      __nv_bfloat162* q = reinterpret_cast<__nv_bfloat162*>(p);
#pragma unroll
      for (int i = 0; i < NP; ++i) q[i] = b[i];
    }
  }
}

// Sites of one CTA.  SPT = 1: the site of locate_site.  SPT = 2: sites (2c, y)
// and (2c + 1, y) of a grid row (launch grid (ny, ceil(nx / 2)), CTA (y, c)), or
// sites 2b and 2b + 1 of a batch (launch grid ceil(ns / 2)); a missing second
// site (odd row length or site count) repeats the first and stores nothing.
template <int SPT>
__device__ __forceinline__ void locate_sites(const GridMap& G, int bx, int by, SiteLoc (&L)[SPT],
                                             bool* has2) {
  if constexpr (SPT == 1) {
    locate_site(G, bx, by, &L[0]);
    *has2 = false;
  } else {
    static_assert(SPT == 2, "one or two sites per CTA");
    if (G.n_events == 1) {
      const int x0 = 2 * by;
      *has2 = x0 + 1 < G.nx0;
      locate_site(G, bx, x0, &L[0]);
      locate_site(G, bx, *has2 ? x0 + 1 : x0, &L[1]);
    } else {
      const int s0 = 2 * bx;
      *has2 = s0 + 1 < G.n_sites;
      locate_site(G, s0, 0, &L[0]);
      locate_site(G, *has2 ? s0 + 1 : s0, 0, &L[1]);
    }
  }
}

// SPT sites per CTA: with two, every per-node constant a thread loads (radial
// and polar operator entries, radial tables) and every per-line scalar serves
// both sites, and the warp reductions carry both sites' sums; each site goes
// through the same operations as with one.  On the 768-node lattice two sites
// per CTA measured slower (0.211 against 0.191 ms per stage at 256^2: the
// doubled live state leaves 7 resident CTAs instead of 12); the autotuner
// keeps both.
// MINB resident blocks per SM bound the registers.  768 nodes (96 threads):
// 12 blocks, 56 registers; measured at 160^2: 75 us against 79 us uncapped (72
// registers) and 89-93 us at 40 registers, which spill.  2048 nodes (128
// threads): 5 blocks, 96 registers; at 512^2 a BF16 stage takes 1.65 ms
// against 1.80 ms with 4 blocks (114 registers) and 1.73 ms with 6 (80,
// spilling).  The autotuner also times the uncapped kernel.
template <class S, int NXI, int NTH, int NPH, int SPT = 1, int MINB = (NTH * NPH <= 96 ? 12 : 5)>
__global__ void __launch_bounds__(NTH* NPH, MINB)
    stage_kernel_x2(const __grid_constant__ StageArgsX2<S, NXI, NTH, NPH> A) {
  static_assert(NXI % 2 == 0 && NTH % 2 == 0, "paired radial nodes, half polar lines");
  static_assert(SPT == 1 || SPT == 2, "one or two sites per CTA");
  constexpr int NL = NTH * NPH;
  constexpr int NN = NL * NXI;
  constexpr int NP = NXI / 2;
  constexpr int NW = (NL + 31) / 32;
  static_assert(NL % 32 == 0, "whole warps (the warp reductions use every lane)");
  static_assert(NW <= kMomParts, "one moment slot per warp");
  constexpr int H = NTH / 2;
  // staged site: pair p of line (l, j) at p * LDK + l * LDL + j (float2 units),
  // LDL = NTH and LDK = NPH NTH + 1 (odd).  The polar items of a warp are the
  // (pair, half) of its own LPW lines of fixed phi, half fastest across the
  // lanes: with this layout the line-wise stores and loads of the owners and
  // the item loads and stores all run at the minimum number of shared-memory
  // wavefronts (768 nodes: 120 per site against 168 with the padded layout;
  // 1.1 % faster stage).
  constexpr int LDL = NTH;
  constexpr int LDK = NPH * NTH + 1;
  constexpr int LPW = 32 / NTH;  // lines of one phi per warp
  static_assert(32 % NTH == 0, "the lines of one phi inside one warp");
  const auto& op = A.op;
  SiteLoc L[SPT];
  bool has2;
  locate_sites<SPT>(A.grid, blockIdx.x, blockIdx.y, L, &has2);
#pragma unroll
  for (int s = 0; s < SPT; ++s) L[s].site = idx_checked(L[s].site, A.grid.n_sites, A.err);
  const int t = threadIdx.x;
  const int j = t % NTH, l = t / NTH;
  // 1/tau of f_in, issued first: its latency hides behind the population loads
  const float milne = A.milne_on ? A.clock->inv_tau_f : 0.f;

  __shared__ float2 fs[SPT][NP * LDK];
  __shared__ float2 pth[SPT][NP * LDK];
  __shared__ float4 tab[SPT][NP];  // (E_eq at 2p, 2p+1;  q1/E_eq at 2p, 2p+1)
  __shared__ float4 red[SPT][NW];  // per-warp partial sums for d ln M / d tau
  __shared__ double lnm_s[4];      // ln M of f_in, f_base per site (lnm_fetch)
  if (t == 0) {
#pragma unroll
    for (int s = 0; s < SPT; ++s)
      if (s == 0 || has2) lnm_fetch(lnm_s + s, A.lnM_in, A.lnM_base, L[s].site, A.mode);
  }

  // 1. own line and the upwind neighbours (periodic), and the streaming term
  //    right away: the neighbour lines die here instead of staying live across
  //    the barriers below (fewer registers, more resident blocks)
  const float cp = op.cph[l], sp = op.sph[l];
  const int sx = (cp > 0.f) ? -1 : 1, sy = (sp > 0.f) ? -1 : 1;
  float2 f[SPT][NP], strm[SPT][NP];
  {
    const float st0 = op.sth[j];
    const float2 nsx0 = bc2(-st0 * fabsf(cp) * A.inv2dx_r), nsy0 = bc2(-st0 * fabsf(sp) * A.inv2dx_r);
    const float2 three0 = bc2(3.f), mfour0 = bc2(-4.f);
#pragma unroll
    for (int s = 0; s < SPT; ++s) {
      const int x = L[s].x, y = L[s].y, nx = L[s].nx, ny = L[s].ny;
      load_pairs<S, NP>(A.f_in + (size_t)L[s].site * NN + t * NXI, f[s]);
      int x1 = x + sx, x2 = x + 2 * sx, y1 = y + sy, y2 = y + 2 * sy;
      x1 += (x1 < 0) ? nx : (x1 >= nx ? -nx : 0);
      x2 += (x2 < 0) ? nx : (x2 >= nx ? -nx : 0);
      x2 += (x2 < 0) ? nx : (x2 >= nx ? -nx : 0);  // grids of one site
      y1 += (y1 < 0) ? ny : (y1 >= ny ? -ny : 0);
      y2 += (y2 < 0) ? ny : (y2 >= ny ? -ny : 0);
      y2 += (y2 < 0) ? ny : (y2 >= ny ? -ny : 0);
      float2 fx1[NP], fx2[NP], fy1[NP], fy2[NP];
      const int ns_all = A.grid.n_sites, b0 = L[s].base;
      const int i1 = idx_checked(b0 + y * nx + idx_checked(x1, nx, A.err), ns_all, A.err);
      const int i2 = idx_checked(b0 + y * nx + idx_checked(x2, nx, A.err), ns_all, A.err);
      const int i3 = idx_checked(b0 + idx_checked(y1, ny, A.err) * nx + x, ns_all, A.err);
      const int i4 = idx_checked(b0 + idx_checked(y2, ny, A.err) * nx + x, ns_all, A.err);
      const S* fl = A.f_in + t * NXI;
      load_pairs<S, NP>(fl + (size_t)i1 * NN, fx1);
      load_pairs<S, NP>(fl + (size_t)i2 * NN, fx2);
      load_pairs<S, NP>(fl + (size_t)i3 * NN, fy1);
      load_pairs<S, NP>(fl + (size_t)i4 * NN, fy2);
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        const float2 Sx = fma2(mfour0, fx1[p], fma2(three0, f[s][p], fx2[p]));
        const float2 Sy = fma2(mfour0, fy1[p], fma2(three0, f[s][p], fy2[p]));
        strm[s][p] = mul2(op.tv[p], fma2(nsy0, Sy, mul2(nsx0, Sx)));
      }
    }
  }

  // site scalars of the matching of f_in
  float ut[SPT], ux[SPT], uy[SPT], invT[SPT], M[SPT], itr[SPT], ax[SPT], ay[SPT], Dm[SPT], Kh[SPT];
#pragma unroll
  for (int s = 0; s < SPT; ++s) {
    static_assert(kSc == 16 && SC_UT == 0 && SC_MEQ == 4 && SC_B == 8 && SC_AX == 12, "float4 groups");
    const float4* q = reinterpret_cast<const float4*>(A.scf + (size_t)L[s].site * kSc);
    const float4 q0 = __ldg(q), q1 = __ldg(q + 1), q2 = __ldg(q + 2), q3 = __ldg(q + 3);
    ut[s] = q0.x; ux[s] = q0.y; uy[s] = q0.z; invT[s] = q0.w;  // SC_UT .. SC_INVT
    M[s] = q1.y; itr[s] = q1.z; Dm[s] = q1.w;                  // SC_MEQ .. SC_D
    Kh[s] = q2.z;                                              // SC_B .. SC_T
    ax[s] = q3.x; ay[s] = q3.y;                                // SC_AX, SC_AY
    if (t < NP) {  // per-site radial table
      const float Meq = q1.x, M2 = M[s] * M[s];
      const float e0 = sqrtf(Meq * Meq + M2 * op.s2[2 * t]), e1 = sqrtf(Meq * Meq + M2 * op.s2[2 * t + 1]);
      tab[s][t] = make_float4(e0, e1, op.q1[2 * t] / e0, op.q1[2 * t + 1] / e1);
    }
  }

  // 2. stage the sites for the polar operator; radial operator on the own lines
#pragma unroll
  for (int s = 0; s < SPT; ++s)
#pragma unroll
    for (int p = 0; p < NP; ++p) fs[s][p * LDK + l * LDL + j] = f[s][p];
  float2 Drf[SPT][NP];
#pragma unroll
  for (int s = 0; s < SPT; ++s)
#pragma unroll
    for (int p = 0; p < NP; ++p) Drf[s][p] = make_float2(0.f, 0.f);
#pragma unroll
  for (int k = 0; k < NXI; ++k) {
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const float2 d = op.Drb[k * NP + p];
#pragma unroll
      for (int s = 0; s < SPT; ++s) Drf[s][p] = fma2(d, bc2((k & 1) ? f[s][k >> 1].y : f[s][k >> 1].x), Drf[s][p]);
    }
  }
  __syncthreads();
  const bool pol = milne != 0.f;
  if (pol) {  // polar lines (pair, l), one half of the outputs per item
    for (int it = (t & 31); it < LPW * NXI; it += 32) {  // this warp's items
      const int lq = (t >> 5) * LPW + it / NXI, r = it % NXI, kp = r / 2, half = r % 2;
      const int base = kp * LDK + lq * LDL;
      float2 g[SPT][NTH];
#pragma unroll
      for (int s = 0; s < SPT; ++s)
#pragma unroll
        for (int jj = 0; jj < NTH; ++jj) g[s][jj] = fs[s][base + jj];
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        if (half != hh) continue;
#pragma unroll
        for (int qq = 0; qq < H; ++qq) {
          const int jp = hh * H + qq;
          float2 acc[SPT];
#pragma unroll
          for (int s = 0; s < SPT; ++s) acc[s] = mul2(op.Dthb[jp * NTH], g[s][0]);
#pragma unroll
          for (int jj = 1; jj < NTH; ++jj) {
            const float2 d = op.Dthb[jp * NTH + jj];
#pragma unroll
            for (int s = 0; s < SPT; ++s) acc[s] = fma2(d, g[s][jj], acc[s]);
          }
#pragma unroll
          for (int s = 0; s < SPT; ++s) pth[s][base + jp] = acc[s];
        }
      }
    }
  }
  __syncthreads();

  // 3. right-hand side on the own lines (same algebra as stage_kernel):
  //    f_eq = Z 2^(c1 E_eq + c2 sinh),  force = f_eq [Gp q1/E_eq + Hp q2 + Jp/cosh],
  //    collision = -(f - f_eq) cc,  cc = (u^tau - tanh vu)/tau_R
  const float st = op.sth[j];
  const float2 mmu2 = bc2(milne * op.mu2[j]), milne2 = bc2(milne);
  constexpr float kLog2e = 1.4426950408889634f;
  const float2 lZ = bc2(A.log2Z);
  float2 c1[SPT], c2[SPT], Gp[SPT], Hp[SPT], Jp[SPT], cc0[SPT], cc1[SPT], ncc0[SPT], ncc1[SPT], utb[SPT], nvub[SPT];
#pragma unroll
  for (int s = 0; s < SPT; ++s) {
    const float vu = st * (cp * ux[s] + sp * uy[s]);
    const float A1 = st * (ax[s] * cp + ay[s] * sp);
    const float au = ax[s] * ux[s] + ay[s] * uy[s];
    const float M2 = M[s] * M[s];
    c1[s] = bc2(-kLog2e * invT[s] * ut[s]); c2[s] = bc2(kLog2e * invT[s] * M[s] * vu);
    Gp[s] = bc2(-invT[s] * A1 * ut[s] * M2); Hp[s] = bc2(invT[s] * A1 * M[s] * vu); Jp[s] = bc2(invT[s] * M[s] * au);
    cc0[s] = bc2(ut[s] * itr[s]); cc1[s] = bc2(-vu * itr[s]);
    ncc0[s] = bc2(-ut[s] * itr[s]); ncc1[s] = bc2(vu * itr[s]);
    utb[s] = bc2(ut[s]); nvub[s] = bc2(-vu);
  }
  float2 Rn[SPT][NP];
  float2 sA[SPT], sQ[SPT], sE[SPT];
#pragma unroll
  for (int s = 0; s < SPT; ++s) sA[s] = sQ[s] = sE[s] = make_float2(0.f, 0.f);
#pragma unroll
  for (int p = 0; p < NP; ++p) {
#pragma unroll
    for (int s = 0; s < SPT; ++s) {
      const float4 tb = tab[s][p];
      const float2 E = make_float2(tb.x, tb.y), QE = make_float2(tb.z, tb.w);
      float2 r = fma2(mmu2, Drf[s][p], strm[s][p]);
      if (pol) r = fma2(milne2, pth[s][p * LDK + l * LDL + j], r);
      const float2 ex = fma2(c1[s], E, fma2(c2[s], op.s[p], lZ));
      const float2 feq = make_float2(ex2_ftz(ex.x), ex2_ftz(ex.y));
      const float2 cc = fma2(cc1[s], op.tv[p], cc0[s]), ncc = fma2(ncc1[s], op.tv[p], ncc0[s]);
      const float2 fcc = fma2(Gp[s], QE, fma2(Hp[s], op.q2[p], fma2(Jp[s], op.ic[p], cc)));
      r = fma2(f[s][p], ncc, fma2(feq, fcc, r));
      Rn[s][p] = r;
      const float2 pu = fma2(op.Sw[p], nvub[s], mul2(op.Cw[p], utb[s]));
      const float2 w = mul2(pu, pu);
      sA[s] = fma2(w, r, sA[s]);
      sQ[s] = fma2(w, Drf[s][p], sQ[s]);
      sE[s] = fma2(w, f[s][p], sE[s]);
    }
  }
  const float wj = op.wj[j];
  // warp partial sums, then every thread combines the NW partials itself;
  // after the halving reduction of 4 SPT values the site-s sums sit on lanes
  // s 4d, s 4d + d and s 4d + 2d (d = 8 / SPT lanes per value)
  const int lane = t & 31, wid = t >> 5;
  {
    constexpr int K = 4 * SPT, dl = 32 / K;
    float v[K];
#pragma unroll
    for (int s = 0; s < SPT; ++s) {
      v[4 * s] = wj * (sA[s].x + sA[s].y);
      v[4 * s + 1] = wj * (sQ[s].x + sQ[s].y);
      v[4 * s + 2] = wj * (sE[s].x + sE[s].y);
      v[4 * s + 3] = 0.f;
    }
    warp_reduce_halving<K>(v, lane);
    const float s1 = __shfl_down_sync(0xffffffffu, v[0], dl), s2 = __shfl_down_sync(0xffffffffu, v[0], 2 * dl);
    if (lane % (4 * dl) == 0) red[lane / (4 * dl)][wid] = make_float4(v[0], s1, s2, 0.f);
  }
  __syncthreads();
  float2 gb[SPT];
#pragma unroll
  for (int s = 0; s < SPT; ++s) {
    float Af = 0.f, Qf = 0.f, Ef = 0.f;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      const float4 rw = red[s][w];
      Af += rw.x; Qf += rw.y; Ef += rw.z;
    }
    // d ln M / d tau from the consistency condition
    const float D = Dm[s];
    // (fast quotient, 2 ulp: the denominator is a moment sum far inside its range;
    // 1 % faster stage than the IEEE division)
    const float g = (D == 0.f) ? 0.f : __fdividef(-D * Af, Kh[s] + D * (4.f * Ef + Qf - Kh[s]));
    if (t == 0 && (s == 0 || has2)) {
      const int site = L[s].site;
      if (!isfinite(g)) atomicOr(A.err, (int)ERR_NONFINITE);
      lnm_wait();
      const double lnM = lnm_s[s], gd = (double)g;
      A.lnM_out[site] = A.mode == 0 ? lnM + A.dtau * gd : 0.5 * (lnm_s[2 + s] + lnM + A.dtau * gd);
    }
    gb[s] = bc2(g);
  }
  const float2 dt = bc2(A.dtau_r);
  float2 out[SPT][NP];
  if (A.mode == 0) {
#pragma unroll
    for (int s = 0; s < SPT; ++s)
#pragma unroll
      for (int p = 0; p < NP; ++p) out[s][p] = fma2(dt, fma2(gb[s], Drf[s][p], Rn[s][p]), f[s][p]);
  } else {
    const float2 half = bc2(0.5f), hdt = bc2(0.5f * A.dtau_r);
#pragma unroll
    for (int s = 0; s < SPT; ++s) {
      float2 fb[NP];
      load_pairs<S, NP>(A.f_base + (size_t)L[s].site * NN + t * NXI, fb);
#pragma unroll
      for (int p = 0; p < NP; ++p)
        out[s][p] = fma2(hdt, fma2(gb[s], Drf[s][p], Rn[s][p]), mul2(half, add2(fb[p], f[s][p])));
    }
  }
#pragma unroll
  for (int s = 0; s < SPT; ++s) {  // out now holds the stored values
    if (s == 0 || has2) store_pairs<S, NP>(A.f_out + (size_t)L[s].site * NN + t * NXI, out[s]);
    finite_checked(reinterpret_cast<const float*>(out[s]), 2 * NP, A.err);
  }

  // 4. moments of what was stored
  const float mu = op.mu[j];
  constexpr int KM = kMom * SPT, dm = 32 / KM;
  float mom[KM];
#pragma unroll
  for (int s = 0; s < SPT; ++s) {
    float2 r0 = make_float2(0.f, 0.f), r1 = r0, r2 = r0, r3 = r0;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      r0 = fma2(op.w0[p], out[s][p], r0);
      r1 = fma2(op.w1[p], out[s][p], r1);
      r2 = fma2(op.w2[p], out[s][p], r2);
      r3 = fma2(op.w3[p], out[s][p], r3);
    }
    const float a1 = wj * (r1.x + r1.y) * st, a3 = wj * (r3.x + r3.y) * st * st;
    float* m = mom + kMom * s;
    m[0] = wj * (r0.x + r0.y); m[1] = wj * (r2.x + r2.y); m[2] = a1 * cp; m[3] = a1 * sp;
    m[4] = a3 * cp * cp; m[5] = a3 * cp * sp; m[6] = a3 * sp * sp; m[7] = wj * (r3.x + r3.y) * mu * mu;
  }
  warp_reduce_halving<KM>(mom, lane);  // lanes dm qq .. dm qq + dm - 1 hold value qq
  // slot wid of moment qq % kMom of site qq / kMom; warp 0 also clears the
  // slots no warp owns
  const int qq = lane / dm, sq = qq / kMom, r = lane % dm;
  if (sq == 0 || has2) {
    const int site = (SPT == 1 || sq == 0) ? L[0].site : L[SPT - 1].site;
    float* dst = A.momf_out + ((size_t)site * kMom + (qq % kMom)) * kMomParts;
    if (r == 0) dst[wid] = mom[0];
    else if (wid == 0 && r == 1) {
#pragma unroll
      for (int w = NW; w < kMomParts; ++w) dst[w] = 0.f;
    }
  }
}

}  // namespace rlbk
