// rlb_stage_mp.cuh -- the fused stream-collide stage in FP32 arithmetic with
// mirror-paired polar lines (Romatschke, arXiv:1108.5561, Sec. 4.3-4.4).
//
// Same right-hand side as stage_kernel and stage_kernel_x2 (Eq. Bmilne with the
// BGK term of Sec. 4.1, Heun stages of Sec. 4.4):
//   rhs = -V.grad f + (1/tau) [mu^2 Dr f + Dth f] + g Dr f + T_M f_eq
//         - ((P.U)/E) (f - f_eq) / tau_R
// Each thread owns the two radial lines (theta_j, phi_l) and (pi - theta_j,
// phi_l).  The Gauss-Legendre nodes are symmetric, mu_{N-1-j} = -mu_j, and in
// the boost-invariant problem nothing but the Milne polar operator sees the
// sign of mu: the transverse velocity V, hence the upwind neighbours, the
// equilibrium f_eq on the moving nodes, the mass-gradient force, the
// collision rate and the moment weights are the same for both lines, and are
// computed once for the two.  The polar operator Dth of Sec. 4.4 commutes with
// the reflection mu -> -mu (its Galerkin kernel (mu - mu^3) d/dmu + 1 - 3 mu^2
// is even), so on the even and odd parts e = f_j + f_{N-1-j}, o = f_j -
// f_{N-1-j} it splits into two N/2 x N/2 blocks,
//   (Dth f)_j = Ae e + Ao o,  (Dth f)_{N-1-j} = Ae e - Ao o,
//   Ae[j][i] = (Dth[j][i] + Dth[j][N-1-i]) / 2,  Ao[j][i] = (Dth[j][i] - Dth[j][N-1-i]) / 2,
// half the multiply-adds of the full operator; the N/2 threads of one azimuth
// exchange e and o through shared memory inside their warp (no CTA barrier).
// Radial nodes are held as packed FP32 pairs (FFMA2).  A site takes
// TS = (N_theta/2) N_phi threads; with TS not a multiple of 32 a CTA holds two
// sites (the 8 x 8 x 12 lattice: 48 threads per site, 96 per CTA).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "rlb_kernels.cuh"
#include "rlb_stage_x2.cuh"

namespace rlbk {

// Per-run radial constants (parameter space; every lane reads the same entry).
template <int NXI>
struct OpsMP {
  static constexpr int NP = NXI / 2;
  float2 Drb[NXI * NP];                   // [k * NP + p] = (Dr[2p][k], Dr[2p+1][k])
  float2 tv[NP], s[NP], q2[NP], ic[NP];   // tanh, sinh, sinh^2/cosh, 1/cosh
  float2 Cw[NP], Sw[NP];                  // cosh sqrt(ecw), sinh sqrt(ecw)
  float2 w0[NP], w1[NP], w2[NP], w3[NP];  // ecw * {1, c s, c^2, s^2}
  float2 s2[NP], q1[NP];                  // sinh^2, sinh (sinh^2 + 1)/cosh
};

// Line constants (device memory), stored field by field so that the lanes of
// a warp read contiguous entries:
//   a[q] = (sin theta_j, mu_j^2, polar weight / (2 N_phi), cos phi_l)
//   b[q] = (sin phi_l, -sin theta_j |cos phi_l| / (2 dx), -sin theta_j |sin phi_l| / (2 dx), 0)
// for the thread slot q = l * (N_theta/2) + j of a site, and the even and odd
// polar blocks, ae[i * H + j] = (Ae[j][i], Ae[j][i]) (likewise ao), which
// depend on j only: the lanes of a warp read H distinct entries (one or two
// sectors) instead of one 96-byte record each.
template <int H, int TS>
struct alignas(16) LinesMP {
  float4 a[TS], b[TS];
  float2 ae[H * H], ao[H * H];
};

template <int NTH, int NPH>
struct MPShape {
  static constexpr int H = NTH / 2;                    // mirror pairs of polar lines
  static constexpr int TS = H * NPH;                   // threads per site
  static constexpr int SPC = (TS % 32 == 0) ? 1 : 2;   // sites per CTA
  static constexpr int NT = SPC * TS;                  // threads per CTA
  static constexpr int G = TS / 16;                    // 16-lane reduction groups per site
};

template <class S, int NXI, int NTH, int NPH>
struct StageArgsMP {
  const S* f_in;
  const double* lnM_in;
  const float* scf;       // FP32 matching of f_in, kSc per site
  const S* f_base;        // corrector: populations at the start of the step
  const double* lnM_base;
  S* f_out;
  double* lnM_out;
  float* momf_out;        // moments of f_out: one partial sum per 16-lane group
  int* err;
  const LinesMP<NTH / 2, (NTH / 2) * NPH>* lines;
  GridMap grid;
  const Clock* clock;     // proper time of f_in
  int milne_on;           // Milne metric (1/tau terms) or Minkowski
  int mode;               // 0 predictor, 1 corrector
  int prefetch_ahead;     // L2 prefetch of the sites of the CTA launched this many CTAs later (0: none)
  double dtau;
  float dtau_r;
  float Zh, Zl;           // Z / (1 + mean error of the hardware 2^x), as FP32 hi + lo
  OpsMP<NXI> op;
};

// Sum of NV values over each group of GL consecutive lanes by halving: value q
// ends on the lanes with (lane % GL) / (GL / NV) == q.
template <int NV, int GL>
__device__ __forceinline__ void group_reduce_halving(float (&v)[NV], int lane) {
  constexpr int L = NV >= 16 ? 4 : NV >= 8 ? 3 : NV >= 4 ? 2 : NV >= 2 ? 1 : 0;
  static_assert((1 << L) == NV && NV <= GL && (GL & (GL - 1)) == 0 && GL <= 32, "powers of two");
#pragma unroll
  for (int lev = 0; lev < L; ++lev) {
    const int h = NV >> (lev + 1), off = (GL / 2) >> lev;
    const bool upper = (lane & off) != 0;
#pragma unroll
    for (int q = 0; q < h; ++q) {
      const float keep = upper ? v[q + h] : v[q];
      const float send = upper ? v[q] : v[q + h];
      v[q] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
#pragma unroll
  for (int off = (GL / 2) >> L; off > 0; off >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], off);
}

// Bring [p, p + bytes) into L2 without waiting (bytes a multiple of 16, p
// 16-byte aligned).
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// The populations of the CTA launched `ahead` CTAs after this one (launch
// order: blockIdx.x fastest; one grid: CTA (y, c) holds sites (SPC c .. SPC c +
// SPC - 1, y) of a row; a batch: CTA b holds sites SPC b ..), into L2 by one
// thread: by the time that CTA runs, its own lines and the lines its
// neighbours read are L2 hits.
template <class S, int NN, int SPC>
__device__ __forceinline__ void prefetch_ahead_sites(const GridMap& G, const S* f, int ahead) {
  const unsigned b = blockIdx.y * gridDim.x + blockIdx.x + (unsigned)ahead;  // 32-bit division (thread 0 waits on it)
  long long s0, n;
  if (G.n_events == 1) {
    const unsigned c = b / gridDim.x, y = b - c * gridDim.x;
    if (c >= gridDim.y) return;
    s0 = (long long)y * G.nx0 + SPC * (long long)c;
    n = G.nx0 - SPC * (long long)c;
  } else {
    if (b >= gridDim.x) return;
    s0 = SPC * (long long)b;
    n = G.n_sites - s0;
  }
  n = n < SPC ? n : SPC;
  if (n > 0) prefetch_l2(f + s0 * NN, (unsigned)(n * NN * sizeof(S)));
}

__device__ __forceinline__ float2 rsqrt2_nr(float2 x) {
  // 1/sqrt(x) per half: the hardware approximation and one Newton step
  // r <- r (3 - x r^2) / 2 (about 1 ulp)
  float2 r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r.x) : "f"(x.x));
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r.y) : "f"(x.y));
  const float2 xr2 = __fmul2_rn(__fmul2_rn(x, r), r);
  return __fmul2_rn(r, __ffma2_rn(make_float2(-0.5f, -0.5f), xr2, make_float2(1.5f, 1.5f)));
}

// Site of a thread: position, event base, and whether it stores (a CTA whose
// second site is missing repeats its first and stores nothing).
struct MPSite {
  int site, x, y, nx, ny, base;
  bool owner;
};

// The CTA's site pair `pair` (one grid: row pair / ceil(nx / 2), columns 2c and
// 2c + 1; a batch: sites 2 pair, 2 pair + 1), or the CTA's own site when a CTA
// holds one site.
template <int SPC>
__device__ __forceinline__ MPSite mp_locate(const GridMap& G, int bx, int by, int sl, int* err) {
  SiteLoc L[SPC];
  bool has2;
  locate_sites<SPC>(G, bx, by, L, &has2);
  MPSite m;
  m.site = idx_checked(sl ? L[SPC - 1].site : L[0].site, G.n_sites, err);
  m.x = sl ? L[SPC - 1].x : L[0].x;
  m.y = sl ? L[SPC - 1].y : L[0].y;
  m.nx = sl ? L[SPC - 1].nx : L[0].nx;
  m.ny = sl ? L[SPC - 1].ny : L[0].ny;
  m.base = sl ? L[SPC - 1].base : L[0].base;
  m.owner = (sl == 0) || has2;
  return m;
}

// Element offsets (into a population array) of the ten lines a thread reads:
// its own lines A = (j, l) and B = (N_theta - 1 - j, l), then A and B at the
// upwind neighbours x - sx, x - 2 sx, y - sy, y - 2 sy (periodic; the same
// neighbours for both lines: V depends on sin theta, not on its sign), in the
// order A x1, A x2, B x1, B x2, A y1, A y2, B y1, B y2.
template <int NXI, int NTH, int NPH>
__device__ __forceinline__ void mp_offsets(const MPSite& m, int l, int jp, float cp, float sp, int n_sites,
                                           int* err, size_t (&o)[10]) {
  constexpr int NN = NXI * NTH * NPH;
  const size_t offA = (size_t)(l * NTH + jp) * NXI, offB = (size_t)(l * NTH + NTH - 1 - jp) * NXI;
  const int x = m.x, y = m.y, nx = m.nx, ny = m.ny, b0 = m.base;
  const int sx = (cp > 0.f) ? -1 : 1, sy = (sp > 0.f) ? -1 : 1;
  int x1 = x + sx, x2 = x + 2 * sx, y1 = y + sy, y2 = y + 2 * sy;
  x1 += (x1 < 0) ? nx : (x1 >= nx ? -nx : 0);
  x2 += (x2 < 0) ? nx : (x2 >= nx ? -nx : 0);
  x2 += (x2 < 0) ? nx : (x2 >= nx ? -nx : 0);  // grids of one site
  y1 += (y1 < 0) ? ny : (y1 >= ny ? -ny : 0);
  y2 += (y2 < 0) ? ny : (y2 >= ny ? -ny : 0);
  y2 += (y2 < 0) ? ny : (y2 >= ny ? -ny : 0);
  const size_t i0 = (size_t)m.site * NN;
  const size_t i1 = (size_t)idx_checked(b0 + y * nx + idx_checked(x1, nx, err), n_sites, err) * NN;
  const size_t i2 = (size_t)idx_checked(b0 + y * nx + idx_checked(x2, nx, err), n_sites, err) * NN;
  const size_t i3 = (size_t)idx_checked(b0 + idx_checked(y1, ny, err) * nx + x, n_sites, err) * NN;
  const size_t i4 = (size_t)idx_checked(b0 + idx_checked(y2, ny, err) * nx + x, n_sites, err) * NN;
  o[0] = i0 + offA; o[1] = i0 + offB;
  o[2] = i1 + offA; o[3] = i2 + offA; o[4] = i1 + offB; o[5] = i2 + offB;
  o[6] = i3 + offA; o[7] = i4 + offA; o[8] = i3 + offB; o[9] = i4 + offB;
}

// The stage at one site for the thread's two lines.  ld(i, v) delivers line i
// of the ten of mp_offsets (i < 10) or, in the corrector, the thread's own
// lines A (i = 10) and B (i = 11) of f_base.  The streaming term comes first
// (the neighbour lines die before the site's own work; computing it last, so
// that the neighbour loads overlap the own-line work, keeps them live and
// measured 3 % slower).  sc holds the site's FP32 matching
// (four float4); eo is the CTA's polar exchange area (NXI/2 + 1 16-byte chunks per
// thread) and red its per-group partial sums; lnm_s[sl] and lnm_s[2 + sl]
// receive ln M of f_in and f_base at site sl (lnm_fetch at the top of the
// kernel).  Contains one CTA barrier.
template <class S, int NXI, int NTH, int NPH, class LD>
__device__ __forceinline__ void mp_body(const StageArgsMP<S, NXI, NTH, NPH>& A, const MPSite& me,
                                        const size_t (&off)[10], int t, int q, int sl, float milne,
                                        const LinesMP<NTH / 2, (NTH / 2) * NPH>& lt, float4 la, float4 lb,
                                        const float4 (&sc)[4], LD&& ld, uint4* eo,
                                        float4* red, const double* lnm_s) {
  using Sh = MPShape<NTH, NPH>;
  constexpr int H = Sh::H, G = Sh::G;
  constexpr int NP = NXI / 2;
  constexpr int EOC = NP + 1;  // 16-byte chunks per thread in eo: e (NP/2), o (NP/2), one of padding
  static_assert(EOC % 2 == 1, "odd stride: bank-conflict free");
  const auto& op = A.op;
  const int lane = t & 31, jp = q % H;
  const float st = la.x, mu2 = la.y, wj = la.z, cp = la.w, sp = lb.x;

  float2 fA[NP], fB[NP], RA[NP], RB[NP];
  ld(0, fA);
  ld(1, fB);

  // 1. streaming -V.grad f from the upwind neighbour lines (periodic) into R
  //    right away: the neighbour lines die here, before the site's own work
  {
    const float2 nsx = bc2(lb.y), nsy = bc2(lb.z), three = bc2(3.f), mfour = bc2(-4.f);
    float2 n1[NP], n2[NP];
    ld(2, n1);  // x, line A
    ld(3, n2);
#pragma unroll
    for (int p = 0; p < NP; ++p) RA[p] = mul2(mul2(op.tv[p], nsx), fma2(mfour, n1[p], fma2(three, fA[p], n2[p])));
    ld(4, n1);  // x, line B
    ld(5, n2);
#pragma unroll
    for (int p = 0; p < NP; ++p) RB[p] = mul2(mul2(op.tv[p], nsx), fma2(mfour, n1[p], fma2(three, fB[p], n2[p])));
    ld(6, n1);  // y, line A
    ld(7, n2);
#pragma unroll
    for (int p = 0; p < NP; ++p) RA[p] = fma2(mul2(op.tv[p], nsy), fma2(mfour, n1[p], fma2(three, fA[p], n2[p])), RA[p]);
    ld(8, n1);  // y, line B
    ld(9, n2);
#pragma unroll
    for (int p = 0; p < NP; ++p) RB[p] = fma2(mul2(op.tv[p], nsy), fma2(mfour, n1[p], fma2(three, fB[p], n2[p])), RB[p]);
  }

  // site scalars of the matching of f_in
  static_assert(kSc == 16 && SC_UT == 0 && SC_MEQ == 4 && SC_B == 8 && SC_AX == 12 && SC_L2T == 14,
                "float4 groups");
  const float ut = sc[0].x, ux = sc[0].y, uy = sc[0].z, invT = sc[0].w;
  const float Meq = sc[1].x, M = sc[1].y, itr = sc[1].z, Dm = sc[1].w, Kh = sc[2].z, ax = sc[3].x, ay = sc[3].y;

  // 2. radial operator on both lines; Milne term mu^2 Dr f / tau into R
  float2 DA[NP], DB[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) DA[p] = DB[p] = make_float2(0.f, 0.f);
#pragma unroll
  for (int k = 0; k < NXI; ++k) {
    const float2 a = bc2((k & 1) ? fA[k >> 1].y : fA[k >> 1].x);
    const float2 b = bc2((k & 1) ? fB[k >> 1].y : fB[k >> 1].x);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const float2 d = op.Drb[k * NP + p];
      DA[p] = fma2(d, a, DA[p]);
      DB[p] = fma2(d, b, DB[p]);
    }
  }
  const float2 mmu2 = bc2(milne * mu2);
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    RA[p] = fma2(mmu2, DA[p], RA[p]);
    RB[p] = fma2(mmu2, DB[p], RB[p]);
  }

  // 3. polar operator on the even and odd parts, exchanged among the H
  //    threads of this azimuth (same warp).  Thread u's chunks lie EOC = NP + 1
  //    chunks apart (odd): 8 consecutive threads store to 8 distinct bank
  //    groups, the two azimuths of a quarter warp read from distinct ones, and
  //    every address is a constant offset from the thread's or its group's
  //    base (an XOR swizzle of the unpadded layout cost integer work per
  //    access; the padded layout measured 2.4 % faster)
  if (milne != 0.f) {
    auto eoc = [&](int u, int c) -> uint4& { return eo[u * EOC + c]; };
#pragma unroll
    for (int p = 0; p < NP; p += 2) {
      const float2 e0 = add2(fA[p], fB[p]), e1 = add2(fA[p + 1], fB[p + 1]);
      const float2 o0 = fma2(bc2(-1.f), fB[p], fA[p]), o1 = fma2(bc2(-1.f), fB[p + 1], fA[p + 1]);
      eoc(t, p / 2) = make_uint4(__float_as_uint(e0.x), __float_as_uint(e0.y), __float_as_uint(e1.x), __float_as_uint(e1.y));
      eoc(t, NP / 2 + p / 2) =
          make_uint4(__float_as_uint(o0.x), __float_as_uint(o0.y), __float_as_uint(o1.x), __float_as_uint(o1.y));
    }
    __syncwarp();
    float2 Ev[NP], Ov[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) Ev[p] = Ov[p] = make_float2(0.f, 0.f);
    const int g0 = t - jp;  // thread of (l, j = 0)
#pragma unroll
    for (int i = 0; i < H; ++i) {
      const float2 ae = __ldg(&lt.ae[i * H + jp]), ao = __ldg(&lt.ao[i * H + jp]);
#pragma unroll
      for (int p = 0; p < NP; p += 2) {
        const uint4 ev = eoc(g0 + i, p / 2), ov = eoc(g0 + i, NP / 2 + p / 2);
        Ev[p] = fma2(ae, make_float2(__uint_as_float(ev.x), __uint_as_float(ev.y)), Ev[p]);
        Ev[p + 1] = fma2(ae, make_float2(__uint_as_float(ev.z), __uint_as_float(ev.w)), Ev[p + 1]);
        Ov[p] = fma2(ao, make_float2(__uint_as_float(ov.x), __uint_as_float(ov.y)), Ov[p]);
        Ov[p + 1] = fma2(ao, make_float2(__uint_as_float(ov.z), __uint_as_float(ov.w)), Ov[p + 1]);
      }
    }
    const float2 ml = bc2(milne);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      RA[p] = fma2(ml, add2(Ev[p], Ov[p]), RA[p]);
      RB[p] = fma2(ml, fma2(bc2(-1.f), Ov[p], Ev[p]), RB[p]);
    }
  }

  // 4. equilibrium, force and collision (shared by the two lines), and the
  //    energy-weighted sums for d ln M / d tau:
  //    f_eq = Z e2, e2 = 2^(c1 E_eq + c2 sinh), force = f_eq [Gp q1/E_eq + Hp q2 + Jp/cosh],
  //    collision = -(f - f_eq) cc, cc = (u^tau - tanh vu)/tau_R.
  //    Z multiplies the per-line coefficients of e2 (hi + lo product, about
  //    an ulp) instead of entering the exponent as an FP32 log2 Z, whose
  //    rounding would scale every f_eq by the same factor (7.7e-8 for the
  //    QCD degeneracy); the factor also takes out the mean error of the
  //    hardware 2^x, measured when the buffers are bound.
  const float L2T = sc[3].z;  // log2(e) / T
  const float vu = st * (cp * ux + sp * uy);
  const float A1 = st * (ax * cp + ay * sp);
  const float au = ax * ux + ay * uy;
  const float M2 = M * M;
  auto zs = [&](float v) { return bc2(fmaf(A.Zh, v, A.Zl * v)); };
  const float2 c1 = bc2(-L2T * ut), c2 = bc2(L2T * M * vu);
  const float2 Gp = zs(-invT * A1 * ut * M2), Hp = zs(invT * A1 * M * vu), Jp = zs(invT * M * au);
  const float2 cc0 = zs(ut * itr), cc1 = zs(-vu * itr), ncc0 = bc2(-ut * itr), ncc1 = bc2(vu * itr);
  const float2 utb = bc2(ut), nvub = bc2(-vu), M2b = bc2(M2), Meq2 = bc2(Meq * Meq);
  float2 sA = make_float2(0.f, 0.f), sQ = sA, sE = sA;
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    // per-site radial table: E_eq = sqrt(M_eq^2 + M^2 sinh^2), q1 / E_eq.
    // E_eq = e2 / sqrt(e2) from the Newton-refined reciprocal square root,
    // then one residual step E += (e2 - E^2) / (2 E): the FP32 Newton step
    // leaves 1/sqrt 1.5e-8 low on average (rounding near 1 is coarser above
    // than below), which the exponent E_eq / T ~ 10 would turn into an f_eq
    // 2e-7 too large at every node; after the residual step E_eq is within
    // half an ulp with no mean error
    const float2 e2 = fma2(M2b, op.s2[p], Meq2);
    const float2 ie = rsqrt2_nr(e2);
    float2 E = mul2(e2, ie);
    E = fma2(mul2(bc2(0.5f), ie), fma2(mul2(bc2(-1.f), E), E, e2), E);  // e2 - E^2 in one rounding
    const float2 QE = mul2(op.q1[p], ie);
    const float2 ex = fma2(c1, E, mul2(c2, op.s[p]));
    const float2 feq = make_float2(ex2_ftz(ex.x), ex2_ftz(ex.y));
    const float2 cc = fma2(cc1, op.tv[p], cc0), ncc = fma2(ncc1, op.tv[p], ncc0);
    const float2 fcc = fma2(Gp, QE, fma2(Hp, op.q2[p], fma2(Jp, op.ic[p], cc)));
    RA[p] = fma2(fA[p], ncc, fma2(feq, fcc, RA[p]));
    RB[p] = fma2(fB[p], ncc, fma2(feq, fcc, RB[p]));
    const float2 pu = fma2(op.Sw[p], nvub, mul2(op.Cw[p], utb));
    const float2 w = mul2(pu, pu);
    sA = fma2(w, RA[p], fma2(w, RB[p], sA));
    sQ = fma2(w, DA[p], fma2(w, DB[p], sQ));
    sE = fma2(w, fA[p], fma2(w, fB[p], sE));
  }

  // Heun base: predictor f + dtau R, corrector (f_base + f)/2 + dtau R / 2;
  // g Dr f is added once g is known
  if (A.mode == 0) {
    const float2 dt = bc2(A.dtau_r);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      RA[p] = fma2(dt, RA[p], fA[p]);
      RB[p] = fma2(dt, RB[p], fB[p]);
    }
  } else {
    float2 bA[NP], bB[NP];
    ld(10, bA);
    ld(11, bB);
    const float2 half = bc2(0.5f), hdt = bc2(0.5f * A.dtau_r);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      RA[p] = fma2(hdt, RA[p], mul2(half, add2(bA[p], fA[p])));
      RB[p] = fma2(hdt, RB[p], mul2(half, add2(bB[p], fB[p])));
    }
  }

  // 5. d ln M / d tau: 16-lane partial sums, combined per site by every thread
  const int gi = q >> 4;  // 16-lane group of this thread within its site
  {
    float v[4] = {wj * (sA.x + sA.y), wj * (sQ.x + sQ.y), wj * (sE.x + sE.y), 0.f};
    group_reduce_halving<4, 16>(v, lane);  // value i on lanes 4i .. 4i + 3 of the group
    const float s1v = __shfl_down_sync(0xffffffffu, v[0], 4), s2w = __shfl_down_sync(0xffffffffu, v[0], 8);
    if ((lane & 15) == 0) red[sl * G + gi] = make_float4(v[0], s1v, s2w, 0.f);
  }
  lnm_wait();  // ln M (long arrived)
  __syncthreads();
  float Af = 0.f, Qf = 0.f, Ef = 0.f;
#pragma unroll
  for (int w = 0; w < G; ++w) {
    const float4 rw = red[sl * G + w];
    Af += rw.x; Qf += rw.y; Ef += rw.z;
  }
  // consistency condition (fast quotient, 2 ulp: the denominator is a moment
  // sum far inside its range)
  const float g = (Dm == 0.f) ? 0.f : __fdividef(-Dm * Af, Kh + Dm * (4.f * Ef + Qf - Kh));
  const int site = me.site;
  if (q == 0 && me.owner) {
    if (!isfinite(g)) atomicOr(A.err, (int)ERR_NONFINITE);
    const double lnM = lnm_s[sl], gd = (double)g;
    A.lnM_out[site] = A.mode == 0 ? lnM + A.dtau * gd : 0.5 * (lnm_s[2 + sl] + lnM + A.dtau * gd);
  }
  const float2 gs = bc2((A.mode == 0 ? A.dtau_r : 0.5f * A.dtau_r) * g);
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    RA[p] = fma2(gs, DA[p], RA[p]);
    RB[p] = fma2(gs, DB[p], RB[p]);
  }
  if (me.owner) {  // RA, RB then hold the stored (rounded) values
    store_pairs<S, NP>(A.f_out + off[0], RA);
    store_pairs<S, NP>(A.f_out + off[1], RB);
  }
  finite_checked(reinterpret_cast<const float*>(RA), 2 * NP, A.err);
  finite_checked(reinterpret_cast<const float*>(RB), 2 * NP, A.err);

  // 6. moments of what was stored (the two lines have the same weights)
  float mom[kMom];
  {
    float2 r0 = make_float2(0.f, 0.f), r1 = r0, r2 = r0, r3 = r0;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const float2 o = add2(RA[p], RB[p]);
      r0 = fma2(op.w0[p], o, r0);
      r1 = fma2(op.w1[p], o, r1);
      r2 = fma2(op.w2[p], o, r2);
      r3 = fma2(op.w3[p], o, r3);
    }
    const float a1 = wj * (r1.x + r1.y) * st, a3 = wj * (r3.x + r3.y) * st * st;
    mom[0] = wj * (r0.x + r0.y); mom[1] = wj * (r2.x + r2.y); mom[2] = a1 * cp; mom[3] = a1 * sp;
    mom[4] = a3 * cp * cp; mom[5] = a3 * cp * sp; mom[6] = a3 * sp * sp; mom[7] = wj * (r3.x + r3.y) * mu2;
  }
  group_reduce_halving<kMom, 16>(mom, lane);  // value i on lanes 2i, 2i + 1 of the group
  if (me.owner) {
    const int r = lane & 15, mi = r >> 1;
    float* dst = A.momf_out + ((size_t)site * kMom + mi) * kMomParts;
    if ((r & 1) == 0) dst[gi] = mom[0];
    else if (gi == 0) {
#pragma unroll
      for (int w = G; w < kMomParts; ++w) dst[w] = 0.f;
    }
  }
}

// MINB resident CTAs per SM bound the registers (8 x 8 x 12: 96 threads; 5
// CTAs, 128 registers).
#ifndef RLB_MP_MINB
#define RLB_MP_MINB 5
#endif
template <class S, int NXI, int NTH, int NPH, int MINB = RLB_MP_MINB>
__global__ void __launch_bounds__(MPShape<NTH, NPH>::NT, MINB)
    stage_kernel_mp(const __grid_constant__ StageArgsMP<S, NXI, NTH, NPH> A) {
  using Sh = MPShape<NTH, NPH>;
  constexpr int H = Sh::H, TS = Sh::TS, SPC = Sh::SPC;
  constexpr int NP = NXI / 2;
  static_assert(NXI % 2 == 0 && NTH % 2 == 0, "paired radial nodes, mirrored polar lines");
  static_assert(Sh::NT % 32 == 0 && TS % 16 == 0 && 16 % H == 0, "whole warps, 16-lane groups");
  static_assert(Sh::G <= kMomParts, "one moment slot per 16-lane group");
  const int t = threadIdx.x;
  const int sl = (SPC == 1) ? 0 : t / TS;  // site of this thread within the CTA
  const int q = t - sl * TS, l = q / H, jp = q - l * H;
  const MPSite me = mp_locate<SPC>(A.grid, blockIdx.x, blockIdx.y, sl, A.err);
  if (A.prefetch_ahead > 0 && t == 0) {
    constexpr int NN = NXI * NTH * NPH;
    prefetch_ahead_sites<S, NN, SPC>(A.grid, A.f_in, A.prefetch_ahead);
    if (A.mode == 1) prefetch_ahead_sites<S, NN, SPC>(A.grid, A.f_base, A.prefetch_ahead);
  }
  const float milne = A.milne_on ? A.clock->inv_tau_f : 0.f;
  const auto& lt = *A.lines;
  const float4 la = __ldg(&lt.a[q]), lb = __ldg(&lt.b[q]);
  __shared__ uint4 eo[Sh::NT * (NP + 1)];  // polar exchange: e and o of every thread
  __shared__ float4 red[SPC * Sh::G];  // per-group partial sums for d ln M / d tau
  // ln M of the site(s), needed after the barrier: copied to shared memory
  // now, so that the owner thread does not wait there for a global load
  // (measured 8 % of the stage)
  __shared__ double lnm_s[4];
  if (q == 0 && me.owner) lnm_fetch(lnm_s + sl, A.lnM_in, A.lnM_base, me.site, A.mode);
  size_t off[10];
  mp_offsets<NXI, NTH, NPH>(me, l, jp, la.w, lb.x, A.grid.n_sites, A.err, off);
  if (A.mode == 1) {  // the corrector's base lines, read after the site's own work: into L1 now
    asm volatile("prefetch.global.L1 [%0];" ::"l"(A.f_base + off[0]));
    asm volatile("prefetch.global.L1 [%0];" ::"l"(A.f_base + off[1]));
  }
  const float4* scq = reinterpret_cast<const float4*>(A.scf + (size_t)me.site * kSc);
  const float4 sc[4] = {__ldg(scq), __ldg(scq + 1), __ldg(scq + 2), __ldg(scq + 3)};
  auto ld = [&](int i, float2 (&v)[NP]) {
    if (i < 10) load_pairs<S, NP>(A.f_in + off[i], v);
    else load_pairs<S, NP>(A.f_base + off[i - 10], v);
  };
  mp_body<S, NXI, NTH, NPH>(A, me, off, t, q, sl, milne, lt, la, lb, sc, ld, eo, red, lnm_s);
}

}  // namespace rlbk
