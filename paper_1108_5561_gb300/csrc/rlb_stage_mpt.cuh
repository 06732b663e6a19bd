// rlb_stage_mpt.cuh -- the mirror-paired stage of rlb_stage_mp.cuh with the
// populations a CTA reads staged in shared memory by bulk asynchronous copies
// (the TMA engine: cp.async.bulk completing on one mbarrier), one grid, FP32
// storage, an even number of sites per row (Romatschke, arXiv:1108.5561, Sec.
// 4.3-4.4: the same right-hand side, Heun stages and reductions).
//
// A CTA holds the two sites (x0, y), (x0 + 1, y).  Streaming is second-order
// upwind, so a line at azimuth phi_l reads the same line at x - 2 sx .. x - sx
// and y - 2 sy .. y - sy with sx = -1 where cos phi_l > 0 (else +1), likewise
// sy with sin phi_l.  The azimuths split into four classes by those signs,
// X+ (cos > 0), X- (cos <= 0), Y+ (sin > 0), Y- (sin <= 0); each is an arc of
// the azimuth circle, at most two runs of consecutive l, and a site's lines
// of one azimuth are one contiguous chunk of N_theta N_xi values.  The CTA
// copies, before any thread reads:
//   its own two sites (contiguous);
//   the X+ chunks of the sites x0 - 1, x0 - 2 and the X- chunks of x0 + 2,
//   x0 + 3 (the other x-neighbours are the CTA's own sites);
//   the Y+ chunks of both sites' columns in rows y - 1, y - 2 and the Y-
//   chunks in rows y + 1, y + 2;
//   in the corrector, its two sites of f_base,
// eight (ten) sites' worth of chunks, each needed chunk once per CTA, in 26
// copies issued by the lanes of warp 0.  Every thread then reads its ten
// (twelve) lines from shared memory.
#pragma once

#include "rlb_stage_mp.cuh"

namespace rlbk {

// Device error bit: a bounded wait of a kernel expired (rlb_check reports
// RLB_ERR_TIMEOUT).
constexpr int ERR_TIMEOUT = 16;

// The four azimuth classes (X+, X-, Y+, Y-) as runs of consecutive l.
struct HaloRuns {
  int start[4][2], count[4][2];
  int n[4];  // chunks per class
};

template <class S, int NXI, int NTH, int NPH>
struct StageArgsMPT {
  StageArgsMP<S, NXI, NTH, NPH> m;
  HaloRuns runs;
};

// Staging layout in chunks of NTH * NXI values: the own sites, the x halo
// (X+ of x0 - 1, x0 - 2; X- of x0 + 2, x0 + 3), the y halo (Y+ of sites 0, 1
// in rows y - 1, then y - 2; Y- likewise in rows y + 1, y + 2), the
// corrector's base sites.
template <int NPH>
struct MPTLayout {
  static constexpr int OWN = 0, XP1 = 2 * NPH;
  int xp2, xm2, xm3, yp, ym, base;
  __device__ MPTLayout(const HaloRuns& R) {
    xp2 = XP1 + R.n[0];
    xm2 = xp2 + R.n[0];
    xm3 = xm2 + R.n[1];
    yp = xm3 + R.n[1];     // + (2 (r - 1) + s) n[2] for site s, row y - r
    ym = yp + 4 * R.n[2];  // + (2 (r - 1) + s) n[3]
    base = ym + 4 * R.n[3];
  }
};
constexpr int kMPTCopies = 26;  // own, 12 halo groups x 2 runs, base

// Copy c of the CTA at (x0, y): destination chunk, source site, first
// azimuth, chunks (0: nothing to copy), and whether it reads f_base.
template <int NPH>
__device__ __forceinline__ int mpt_copy(int c, const HaloRuns& R, const MPTLayout<NPH>& Ly, int x0, int y, int nx,
                                        int ny, int* dst, int* site, int* l0, bool* from_base) {
  *from_base = false;
  if (c == 0 || c == kMPTCopies - 1) {
    *dst = c == 0 ? Ly.OWN : Ly.base;
    *site = y * nx + x0;
    *l0 = 0;
    *from_base = c != 0;
    return 2 * NPH;  // both sites: x0 + 1 < nx (nx even)
  }
  const int g = (c - 1) >> 1, r = (c - 1) & 1;
  int cls, dx, dy, d;
  if (g < 4) {  // x halo
    cls = g < 2 ? 0 : 1;
    dx = g == 0 ? -1 : g == 1 ? -2 : g == 2 ? 2 : 3;
    dy = 0;
    d = g == 0 ? Ly.XP1 : g == 1 ? Ly.xp2 : g == 2 ? Ly.xm2 : Ly.xm3;
  } else {  // y halo: g - 4 = 4 (class Y-) + 2 (row - 1) + site
    const int h = g - 4, s = h & 1, rr = ((h >> 1) & 1) + 1;
    cls = h < 4 ? 2 : 3;
    dx = s;
    dy = cls == 2 ? -rr : rr;
    d = (cls == 2 ? Ly.yp : Ly.ym) + (2 * (rr - 1) + s) * R.n[cls];
  }
  const int xs = ((x0 + dx) % nx + nx) % nx, ys = ((y + dy) % ny + ny) % ny;
  *dst = d + (r == 1 ? R.count[cls][0] : 0);
  *site = ys * nx + xs;
  *l0 = R.start[cls][r];
  return R.count[cls][r];
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for phase 0 of the mbarrier for at most limit_ns; false on expiry.
__device__ __forceinline__ bool mbar_wait0(unsigned bar, unsigned long long limit_ns) {
  const unsigned long long t0 = global_ns();
  while (true) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar)
        : "memory");
    if (done) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

// 8 x 8 x 12 FP32: 96 threads (two sites), 30 KB staged, five CTAs per SM.
template <int NXI, int NTH, int NPH, int MINB = RLB_MP_MINB>
__global__ void __launch_bounds__(MPShape<NTH, NPH>::NT, MINB)
    stage_kernel_mpt(const __grid_constant__ StageArgsMPT<float, NXI, NTH, NPH> P) {
  using Sh = MPShape<NTH, NPH>;
  constexpr int H = Sh::H, TS = Sh::TS, NP = NXI / 2, CH = NTH * NXI, NN = CH * NPH;
  static_assert(Sh::SPC == 2 && NXI % 8 == 0, "two sites per CTA, 32-byte lines");
  const auto& A = P.m;
  const int t = threadIdx.x;
  const int sl = t / TS;
  const int q = t - sl * TS, l = q / H, jp = q - l * H;
  const int y = blockIdx.x, x0 = 2 * blockIdx.y, nx = A.grid.nx0, ny = A.grid.ny0;
  MPSite me;
  me.site = idx_checked(y * nx + x0 + sl, A.grid.n_sites, A.err);
  me.x = x0 + sl; me.y = y; me.nx = nx; me.ny = ny; me.base = 0; me.owner = true;

  __shared__ __align__(128) float stg[10 * NN];
  __shared__ __align__(8) unsigned long long bar;
  const MPTLayout<NPH> Ly(P.runs);
  const unsigned bar_s = (unsigned)__cvta_generic_to_shared(&bar);
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_s) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (t < 32) {
    if (t == 0) {
      const unsigned bytes = (unsigned)((A.mode == 1 ? 10 : 8) * NN * sizeof(float));
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_s), "r"(bytes) : "memory");
    }
    __syncwarp();
    if (t < kMPTCopies) {
      int dst, site, l0;
      bool fb;
      const int n = mpt_copy<NPH>(t, P.runs, Ly, x0, y, nx, ny, &dst, &site, &l0, &fb);
      if (n > 0 && (!fb || A.mode == 1)) {
        const float* src = (fb ? A.f_base : A.f_in) + (size_t)idx_checked(site, A.grid.n_sites, A.err) * NN +
                           (size_t)l0 * CH;
        const unsigned d = (unsigned)__cvta_generic_to_shared(stg + (size_t)dst * CH);
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(d),
            "l"(src), "r"((unsigned)(n * CH * sizeof(float))), "r"(bar_s)
            : "memory");
      }
    }
  }
  if (A.prefetch_ahead > 0 && t == 0) {
    prefetch_ahead_sites<float, NN, 2>(A.grid, A.f_in, A.prefetch_ahead);
    if (A.mode == 1) prefetch_ahead_sites<float, NN, 2>(A.grid, A.f_base, A.prefetch_ahead);
  }
  const float milne = A.milne_on ? A.clock->inv_tau_f : 0.f;
  const auto& lt = *A.lines;
  const float4 la = __ldg(&lt.a[q]), lb = __ldg(&lt.b[q]);
  __shared__ uint4 eo[Sh::NT * (NP + 1)];
  __shared__ float4 red[2 * Sh::G];
  __shared__ double lnm_s[4];
  if (q == 0) lnm_fetch(lnm_s + sl, A.lnM_in, A.lnM_base, me.site, A.mode);
  const float4* scq = reinterpret_cast<const float4*>(A.scf + (size_t)me.site * kSc);
  const float4 sc[4] = {__ldg(scq), __ldg(scq + 1), __ldg(scq + 2), __ldg(scq + 3)};

  // line offsets: the global ones of the own lines (stores), the staged ones
  // of all twelve (chunk * CH + j * NXI)
  size_t off[10] = {};
  const int jA = jp, jB = NTH - 1 - jp;
  off[0] = (size_t)me.site * NN + (size_t)(l * NTH + jA) * NXI;
  off[1] = (size_t)me.site * NN + (size_t)(l * NTH + jB) * NXI;
  int so[6];  // chunks: own, x1, x2, y1, y2, base
  {
    const int code = __float_as_int(lb.w);  // class bits and the index of l in its X and Y classes
    const bool xm = code & 1, ym = code & 2;
    const int hx = (code >> 4) & 0xff, hy = (code >> 12) & 0xff;
    so[0] = Ly.OWN + sl * NPH + l;
    if (!xm) {
      so[1] = sl == 0 ? Ly.XP1 + hx : Ly.OWN + l;
      so[2] = sl == 0 ? Ly.xp2 + hx : Ly.XP1 + hx;
    } else {
      so[1] = sl == 0 ? Ly.OWN + NPH + l : Ly.xm2 + hx;
      so[2] = sl == 0 ? Ly.xm2 + hx : Ly.xm3 + hx;
    }
    const int yb = ym ? Ly.ym : Ly.yp, ny_ = P.runs.n[ym ? 3 : 2];
    so[3] = yb + sl * ny_ + hy;
    so[4] = yb + (2 + sl) * ny_ + hy;
    so[5] = Ly.base + sl * NPH + l;
  }
  // every wait is bounded (1 s); the CTA leaves together if any expired,
  // after a second bounded wait for copies still in flight
  const bool ok = mbar_wait0(bar_s, 1000000000ull);
  if (__syncthreads_or(!ok)) {
    if (t == 0) atomicOr(A.err, ERR_TIMEOUT);
    if (ok == false) mbar_wait0(bar_s, 1000000000ull);
    return;
  }
  auto ld = [&](int i, float2 (&v)[NP]) {
    // i: 0, 1 own A, B; 2 x1 A, 3 x2 A, 4 x1 B, 5 x2 B; 6 y1 A, 7 y2 A, 8 y1 B, 9 y2 B; 10, 11 base A, B
    const int c = i < 2 ? so[0] : i < 6 ? so[1 + ((i - 2) & 1)] : i < 10 ? so[3 + ((i - 6) & 1)] : so[5];
    const int j = (i < 2 ? i : i < 10 ? ((i - 2) >> 1) & 1 : i - 10) ? jB : jA;
    const float4* s = reinterpret_cast<const float4*>(stg + c * CH + j * NXI);
#pragma unroll
    for (int h = 0; h < NP / 2; ++h) {
      const float4 a = s[h];
      v[2 * h] = make_float2(a.x, a.y);
      v[2 * h + 1] = make_float2(a.z, a.w);
    }
  };
  mp_body<float, NXI, NTH, NPH>(A, me, off, t, q, sl, milne, lt, la, lb, sc, ld, eo, red, lnm_s);
}

}  // namespace rlbk

namespace rlbk {

// The staging barrier on its own (one CTA): an mbarrier expecting 16 bytes
// from one bulk copy, issued only when `deliver` is set, then the bounded wait
// of the stage kernel.  out[0] = 1 if the wait expired, out[1] = the copied
// value (src[0] when delivered).
__global__ void wait_selftest_kernel(const float* src, int deliver, unsigned long long limit_ns, int* out) {
  __shared__ __align__(16) float buf[4];
  __shared__ __align__(8) unsigned long long bar;
  const unsigned bar_s = (unsigned)__cvta_generic_to_shared(&bar);
  if (threadIdx.x == 0) {
    buf[0] = -1.f;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_s) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_s), "r"(16u) : "memory");
    if (deliver) {
      const unsigned d = (unsigned)__cvta_generic_to_shared(buf);
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], 16, [%2];" ::"r"(d),
          "l"(src), "r"(bar_s)
          : "memory");
    }
  }
  const bool ok = mbar_wait0(bar_s, limit_ns);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) out[0] = 1;
    return;
  }
  if (threadIdx.x == 0) {
    out[0] = 0;
    out[1] = __float_as_int(buf[0]);
  }
}

}  // namespace rlbk
