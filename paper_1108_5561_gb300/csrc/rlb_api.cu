// rlb_api.cu -- C ABI (include/rlb.h) of the GB300 lattice Boltzmann step.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <string>
#include <mutex>
#include <type_traits>
#include <utility>
#include <vector>

#include "../../include/rlb.h"
#include "rlb_host.hpp"
#include "rlb_kernels.cuh"
#include "rlb_stage_x2.cuh"
#include "rlb_stage_mpt.cuh"
#include "rlb_adjoint.cuh"
#include "rlb_peaks.cuh"

struct rlb_ctx {
  int device = 0;
  std::string err;
  bool eos_ok = false, grid_ok = false, bound = false, inited = false;
  rlb::EosParams eosp;
  rlb::EosTable tab;
  rlb_grid_params gp{};
  rlb::Lattice lat;
  size_t ns = 0, nn = 0, pop_bytes = 0;
  size_t f_off = 0, lnM_off = 0;  // state
  size_t fs_off = 0, lnMs_off = 0, T_off = 0, err_off = 0, tab_off = 0, eps_off = 0;  // scratch
  size_t mom_off = 0, moms_off = 0, sc_off = 0, tabf_off = 0, scf_off = 0;
  size_t ev_off = 0, loc_off = 0, clock_off = 0, lines_off = 0;
  // rlb_moments_async: two device staging slots of ns x 8 doubles (allocated
  // at the first call), a copy stream, per slot the events "observables ready"
  // and "copy done", the next slot
  char* mstage = nullptr;
  cudaStream_t cstream = nullptr;
  cudaEvent_t cev_ready[2] = {nullptr, nullptr}, cev_done[2] = {nullptr, nullptr};
  int cslot = 0;
  // line constants of the mirror-paired stage kernel (rlbk::LinesMP)
  std::vector<unsigned char> lines_mp;
  // events: one for a single grid, n for a batch (with a per-site locator)
  std::vector<rlbk::EventInfo> events;
  std::vector<int2> loc;
  char* state = nullptr;
  char* scratch = nullptr;
  double tau = 0.0;
  // one step captured as a CUDA graph (on the first rlb_step), replayed after
  bool graphs = true;
  cudaStream_t gstream = nullptr;
  cudaGraphExec_t gexec = nullptr;     // the full step
  cudaGraphExec_t gexec_nm = nullptr;  // the step without its first matching (scf_fresh)
  // the FP32/FP64 site scalars hold the matching of the current state (set by
  // rlb_moments, which matches it anyway): the next step skips its first
  // matching, which would repeat the same work with the same result
  bool scf_fresh = false;
  cudaEvent_t gev[2] = {nullptr, nullptr};
  int stage_variant = -1;  // rlb_autotune's choice (see Stager); -1: the default of the lattice
  // mean relative error of the hardware 2^x of the FP32 stage kernels on this
  // device (ex2_bias_kernel), measured once per context
  double ex2_bias = 0.0;
  bool ex2_measured = false;
  // adjoint workspace (caller-owned): offsets in bytes; per-node adjoints in
  // FP64 or FP32 (adj_prec, RLB_F64 or RLB_F32), per-site quantities in FP64
  char* adj = nullptr;
  int adj_prec = RLB_F64;
  size_t a_f = 0, a_l = 0, a_fb = 0, a_rb = 0, a_lin = 0, a_lbar = 0, a_sbar = 0, a_mbar = 0;
  size_t a_ebar = 0, a_mom = 0, a_sc = 0, a_T = 0, a_tot = 0, a_eps = 0, a_eta = 0;
  size_t a_momf = 0, a_scf = 0;  // FP32 adjoint: moment partials and site scalars of the stage input
  // optional per-kernel timing (CUDA events on the launch stream)
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;  // kind, (start, end)
  double t_ms[3] = {0, 0, 0};
  long t_n[3] = {0, 0, 0};
};

namespace {

// matching: one site per thread; 64-thread blocks spread the FP64-heavy sites
// evenly over the SMs (65,536 sites: 1,024 blocks, 6.7 per SM)
constexpr int kMatchThreads = 64;

// forget the captured steps (buffers, variant or matching state changed)
void drop_graphs(rlb_ctx* ctx) {
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  if (ctx->gexec_nm) cudaGraphExecDestroy(ctx->gexec_nm);
  ctx->gexec = ctx->gexec_nm = nullptr;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

rlb_status fail(rlb_ctx* c, rlb_status s, const std::string& m) {
  if (c) c->err = m;
  return s;
}

rlb_status cuda_fail(rlb_ctx* c, cudaError_t e, const char* what) {
  return fail(c, RLB_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define RLB_CUDA(call, what)                       \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
  } while (0)

size_t pop_size(int prec) { return prec == RLB_F64 ? 8 : (prec == RLB_F32 ? 4 : 2); }

bool supported_shape(int nxi, int nth, int nph) {
  return (nxi == 8 && nth == 8 && nph == 12) || (nxi == 16 && nth == 8 && nph == 16) ||
         (nxi == 5 && nth == 5 && nph == 2) || (nxi == 6 && nth == 4 && nph == 6) ||
         (nxi == 8 && nth == 8 && nph == 2);
}

// L2 prefetch distance of the mirror-paired stage kernel, in waves of resident
// CTAs: a CTA prefetches the populations of the CTA launched this many waves
// after it
constexpr int kPrefetchWaves = 1;

// room for the line constants of the mirror-paired stage kernel: (N_theta/2)
// N_phi entries of 32 + 8 N_theta bytes (the largest lattice: 64 x 96 B)
constexpr size_t kLinesBytes = 16384;

// sites and events of a configuration (one grid or a batch of events)
struct Shape {
  size_t ns, events;
};
Shape grid_shape(const rlb_grid_params& g) { return {(size_t)g.nx * g.ny, 1}; }

void layout(const rlb_grid_params& g, const Shape& sh, size_t table_points, size_t* state_b,
            size_t* scratch_b, rlb_ctx* c) {
  const size_t ns = sh.ns;
  const size_t nn = (size_t)g.n_xi * g.n_theta * 2 * g.n_phi_half;
  const size_t fb = align256(ns * nn * pop_size(g.prec));
  const size_t mb = align256(ns * sizeof(double));
  size_t off = 0;
  size_t f_off = off; off += fb;
  size_t lnM_off = off; off += mb;
  *state_b = off;
  off = 0;
  size_t fs_off = off; off += fb;
  size_t lnMs_off = off; off += mb;
  size_t T_off = off; off += mb;
  size_t eps_off = off; off += mb;
  // moments: kMom doubles per site (FP64 storage) or kMom x kMomParts floats
  const size_t momb = align256(ns * std::max(rlbk::kMom * sizeof(double), rlbk::kMom * rlbk::kMomParts * sizeof(float)));
  size_t mom_off = off; off += momb;
  size_t moms_off = off; off += momb;
  size_t sc_off = off; off += align256(ns * rlbk::kSc * sizeof(double));
  size_t err_off = off; off += 256;
  size_t tab_off = off; off += align256((table_points + 6) * rlb::kFields * sizeof(double));
  // FP32 table: hi parts, then lo parts (hi + lo = the FP64 table to 2^-48)
  size_t tabf_off = off; off += align256(2 * (table_points + 6) * rlb::kFields * sizeof(float));
  size_t scf_off = off; off += align256(ns * rlbk::kSc * sizeof(float));
  size_t ev_off = off; off += align256(sh.events * sizeof(rlbk::EventInfo));
  size_t loc_off = off; off += sh.events > 1 ? align256(ns * sizeof(int2)) : 0;
  size_t clock_off = off; off += 256;
  size_t lines_off = off; off += kLinesBytes;
  *scratch_b = off;
  if (c) {
    c->ev_off = ev_off; c->loc_off = loc_off; c->clock_off = clock_off; c->lines_off = lines_off;
    c->f_off = f_off; c->lnM_off = lnM_off;
    c->fs_off = fs_off; c->lnMs_off = lnMs_off; c->T_off = T_off; c->eps_off = eps_off;
    c->err_off = err_off; c->tab_off = tab_off;
    c->mom_off = mom_off; c->moms_off = moms_off; c->sc_off = sc_off;
    c->tabf_off = tabf_off; c->scf_off = scf_off;
  }
}

// adjoint workspace: FP64 adjoints of f (twice), of r, and per-site arrays
size_t adj_layout(rlb_ctx* c) {
  const size_t pe = c->adj_prec == RLB_F32 ? sizeof(float) : sizeof(double);
  const size_t ns = c->ns, pn = align256(ns * c->nn * pe), s1 = align256(ns * sizeof(double));
  size_t off = 0;
  c->a_f = off; off += pn;
  c->a_fb = off; off += pn;
  c->a_rb = off; off += pn;
  c->a_l = off; off += s1;
  c->a_lin = off; off += s1;
  c->a_lbar = off; off += s1;
  c->a_ebar = off; off += s1;
  c->a_T = off; off += s1;
  c->a_eps = off; off += s1;
  c->a_sbar = off; off += align256(ns * rlbk::kAdjS * sizeof(double));
  c->a_mbar = off; off += align256(ns * rlbk::kMom * sizeof(double));
  c->a_mom = off; off += align256(ns * rlbk::kMom * sizeof(double));
  c->a_sc = off; off += align256(ns * rlbk::kSc * sizeof(double));
  const bool f32 = c->adj_prec == RLB_F32;
  c->a_momf = off; off += f32 ? align256(ns * rlbk::kMom * rlbk::kMomParts * sizeof(float)) : 0;
  c->a_scf = off; off += f32 ? align256(ns * rlbk::kSc * sizeof(float)) : 0;
  c->a_tot = off; off += 256;
  c->a_eta = off; off += 256;
  return off;
}

template <class R, int NXI, int NTH, int NPH>
rlbk::Ops<R, NXI, NTH, NPH> make_ops(const rlb::Lattice& L) {
  rlbk::Ops<R, NXI, NTH, NPH> o;
  for (int i = 0; i < NXI * NXI; ++i) o.Dr[i] = (R)L.Dr[i];
  for (int i = 0; i < NTH * NTH; ++i) o.Dth[i] = (R)L.Dth[i];
  for (int k = 0; k < NXI; ++k) {
    const double c = L.c[k], s = L.s[k], e = L.ecw[k];
    o.c[k] = (R)c; o.s[k] = (R)s; o.s2[k] = (R)(s * s); o.inv_c[k] = (R)(1.0 / c);
    o.tv[k] = (R)(s / c); o.q1[k] = (R)(s * (s * s + 1.0) / c); o.q2[k] = (R)(s * s / c);
    o.w0[k] = (R)e; o.w1[k] = (R)(e * c * s); o.w2[k] = (R)(e * c * c); o.w3[k] = (R)(e * s * s);
    o.ecw[k] = (R)e;
  }
  for (int j = 0; j < NTH; ++j) {
    o.mu[j] = (R)L.mu[j]; o.mu2[j] = (R)(L.mu[j] * L.mu[j]); o.sth[j] = (R)L.sth[j];
    o.sth_mu[j] = (R)(L.sth[j] * L.mu[j]); o.wj[j] = (R)(L.wth[j] / (2.0 * NPH));
  }
  for (int l = 0; l < NPH; ++l) { o.cph[l] = (R)L.cph[l]; o.sph[l] = (R)L.sph[l]; }
  return o;
}

template <int NXI, int NTH, int NPH>
rlbk::OpsX2<NXI, NTH, NPH> make_ops_x2(const rlb::Lattice& L) {
  rlbk::OpsX2<NXI, NTH, NPH> o;
  constexpr int NP = NXI / 2;
  auto pr = [](double a, double b) { return make_float2((float)a, (float)b); };
  for (int k = 0; k < NXI; ++k)
    for (int p = 0; p < NP; ++p) o.Drb[k * NP + p] = pr(L.Dr[(2 * p) * NXI + k], L.Dr[(2 * p + 1) * NXI + k]);
  for (int i = 0; i < NTH * NTH; ++i) o.Dthb[i] = pr(L.Dth[i], L.Dth[i]);
  for (int p = 0; p < NP; ++p) {
    double c[2], s[2], e[2];
    for (int h = 0; h < 2; ++h) { c[h] = L.c[2 * p + h]; s[h] = L.s[2 * p + h]; e[h] = L.ecw[2 * p + h]; }
    o.tv[p] = pr(s[0] / c[0], s[1] / c[1]);
    o.s[p] = pr(s[0], s[1]);
    o.q2[p] = pr(s[0] * s[0] / c[0], s[1] * s[1] / c[1]);
    o.ic[p] = pr(1.0 / c[0], 1.0 / c[1]);
    o.Cw[p] = pr(c[0] * std::sqrt(e[0]), c[1] * std::sqrt(e[1]));
    o.Sw[p] = pr(s[0] * std::sqrt(e[0]), s[1] * std::sqrt(e[1]));
    o.w0[p] = pr(e[0], e[1]);
    o.w1[p] = pr(e[0] * c[0] * s[0], e[1] * c[1] * s[1]);
    o.w2[p] = pr(e[0] * c[0] * c[0], e[1] * c[1] * c[1]);
    o.w3[p] = pr(e[0] * s[0] * s[0], e[1] * s[1] * s[1]);
  }
  for (int k = 0; k < NXI; ++k) {
    const double c = L.c[k], s = L.s[k];
    o.s2[k] = (float)(s * s);
    o.q1[k] = (float)(s * (s * s + 1.0) / c);
  }
  for (int j = 0; j < NTH; ++j) {
    o.sth[j] = (float)L.sth[j]; o.mu[j] = (float)L.mu[j]; o.mu2[j] = (float)(L.mu[j] * L.mu[j]);
    o.wj[j] = (float)(L.wth[j] / (2.0 * NPH));
  }
  for (int l = 0; l < NPH; ++l) { o.cph[l] = (float)L.cph[l]; o.sph[l] = (float)L.sph[l]; }
  return o;
}

// Line constants of stage_kernel_mp (rlbk::LinesMP<H, TS>, H = N_theta/2,
// TS = H N_phi): thread slot q = l H + j of a site owns the polar lines j and
// N_theta - 1 - j at azimuth l.  The mirror lines share sin(theta), mu^2 and
// the polar weight (averaged over the pair, equal up to rounding), and the
// even and odd blocks of the polar operator come from its rows j < H.
std::vector<unsigned char> make_lines_mp(const rlb::Lattice& L, double dx) {
  const int nth = L.nth, nph = L.nph, H = nth / 2, TS = H * nph;
  std::vector<unsigned char> out(32 * (size_t)TS + 16 * (size_t)H * H, 0);
  float* a = reinterpret_cast<float*>(out.data());
  float* b = a + 4 * TS;
  float* ae = b + 4 * TS;
  float* ao = ae + 2 * H * H;
  for (int l = 0; l < nph; ++l)
    for (int jp = 0; jp < H; ++jp) {
      const int q = l * H + jp, jb = nth - 1 - jp;
      const double st = 0.5 * (L.sth[jp] + L.sth[jb]);
      const double mu2 = 0.5 * (L.mu[jp] * L.mu[jp] + L.mu[jb] * L.mu[jb]);
      const double wj = 0.5 * (L.wth[jp] + L.wth[jb]) / (2.0 * nph);
      const double cp = L.cph[l], sp = L.sph[l];
      float* e = a + 4 * q;
      e[0] = (float)st; e[1] = (float)mu2; e[2] = (float)wj; e[3] = (float)cp;
      e = b + 4 * q;
      e[0] = (float)sp; e[1] = (float)(-st * std::fabs(cp) / (2.0 * dx));
      e[2] = (float)(-st * std::fabs(sp) / (2.0 * dx));
      // halo staging (stage_kernel_mpt): bit 0 cos <= 0 (class X-), bit 1
      // sin <= 0 (Y-), bits 4-11 and 12-19 the index of l in its X and Y class
      int hx = 0, hy = 0;
      for (int m = 0; m < l; ++m) {
        hx += (L.cph[m] > 0) == (cp > 0);
        hy += (L.sph[m] > 0) == (sp > 0);
      }
      const int code = (cp > 0 ? 0 : 1) | (sp > 0 ? 0 : 2) | (hx << 4) | (hy << 12);
      std::memcpy(&e[3], &code, sizeof code);
    }
  for (int jp = 0; jp < H; ++jp)
    for (int i = 0; i < H; ++i) {
      const double d0 = L.Dth[jp * nth + i], d1 = L.Dth[jp * nth + (nth - 1 - i)];
      const size_t k = 2 * ((size_t)i * H + jp);
      ae[k] = ae[k + 1] = (float)(0.5 * (d0 + d1));
      ao[k] = ao[k + 1] = (float)(0.5 * (d0 - d1));
    }
  return out;
}

// The azimuth classes of the halo-staged kernel (X+: cos > 0, X-, Y+: sin > 0,
// Y-) as runs of consecutive l; false when a class has more than two runs.
bool make_halo_runs(const rlb::Lattice& L, rlbk::HaloRuns* R) {
  std::memset(R, 0, sizeof *R);
  for (int c = 0; c < 4; ++c) {
    int runs = 0;
    for (int l = 0; l < L.nph; ++l) {
      const double v = c < 2 ? L.cph[l] : L.sph[l];
      const bool in = (c % 2 == 0) ? v > 0 : !(v > 0);
      if (!in) continue;
      ++R->n[c];
      const double pv = l > 0 ? (c < 2 ? L.cph[l - 1] : L.sph[l - 1]) : 0.0;
      const bool prev_in = l > 0 && ((c % 2 == 0) ? pv > 0 : !(pv > 0));
      if (!prev_in) {
        if (runs == 2) return false;
        R->start[c][runs++] = l;
      }
      R->count[c][runs - 1]++;
    }
  }
  return true;
}

template <int NXI>
rlbk::OpsMP<NXI> make_ops_mp(const rlb::Lattice& L) {
  rlbk::OpsMP<NXI> o;
  constexpr int NP = NXI / 2;
  auto pr = [](double a, double b) { return make_float2((float)a, (float)b); };
  for (int k = 0; k < NXI; ++k)
    for (int p = 0; p < NP; ++p) o.Drb[k * NP + p] = pr(L.Dr[(2 * p) * NXI + k], L.Dr[(2 * p + 1) * NXI + k]);
  for (int p = 0; p < NP; ++p) {
    double c[2], s[2], e[2];
    for (int h = 0; h < 2; ++h) { c[h] = L.c[2 * p + h]; s[h] = L.s[2 * p + h]; e[h] = L.ecw[2 * p + h]; }
    o.tv[p] = pr(s[0] / c[0], s[1] / c[1]);
    o.s[p] = pr(s[0], s[1]);
    o.q2[p] = pr(s[0] * s[0] / c[0], s[1] * s[1] / c[1]);
    o.ic[p] = pr(1.0 / c[0], 1.0 / c[1]);
    o.Cw[p] = pr(c[0] * std::sqrt(e[0]), c[1] * std::sqrt(e[1]));
    o.Sw[p] = pr(s[0] * std::sqrt(e[0]), s[1] * std::sqrt(e[1]));
    o.w0[p] = pr(e[0], e[1]);
    o.w1[p] = pr(e[0] * c[0] * s[0], e[1] * c[1] * s[1]);
    o.w2[p] = pr(e[0] * c[0] * c[0], e[1] * c[1] * c[1]);
    o.w3[p] = pr(e[0] * s[0] * s[0], e[1] * s[1] * s[1]);
    o.s2[p] = pr(s[0] * s[0], s[1] * s[1]);
    o.q1[p] = pr(s[0] * (s[0] * s[0] + 1.0) / c[0], s[1] * (s[1] * s[1] + 1.0) / c[1]);
  }
  return o;
}

// Mean relative error of the hardware approximation of 2^x used for the
// equilibrium in the FP32 stage kernels (ex2.approx.ftz), over x in [-60, 0]
// (the exponents of f_eq): 65,536 arguments against the FP64 exp2, summed in
// FP64 into *out (zeroed by the caller).  The errors of the approximation are
// not centred on zero (-5.2e-8 on GB300), and a factor common to every f_eq
// makes the collision term create or remove energy at that rate, so the
// stage kernel divides Z by 1 + the mean.
__global__ void ex2_bias_kernel(double* out) {
  constexpr int N = 1 << 16;
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const float x = -60.f * ((float)i + 0.5f) / (float)N;
    acc += (double)rlbk::ex2_ftz(x) / exp2((double)x) - 1.0;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, acc / N);
}

// Measure ex2_bias_kernel's mean once per context, using 8 bytes of `scr` at
// `off` (free at the time of the call) and synchronising the stream.
rlb_status measure_ex2_bias(rlb_ctx* ctx, char* scr, size_t off, cudaStream_t st) {
  if (ctx->ex2_measured) return RLB_OK;
  double* d = reinterpret_cast<double*>(scr + off);
  RLB_CUDA(cudaMemsetAsync(d, 0, sizeof(double), st), "ex2 bias reset");
  ex2_bias_kernel<<<64, 256, 0, st>>>(d);
  RLB_CUDA(cudaGetLastError(), "ex2_bias_kernel launch");
  double b = 0.0;
  RLB_CUDA(cudaMemcpyAsync(&b, d, sizeof(double), cudaMemcpyDeviceToHost, st), "ex2 bias read");
  RLB_CUDA(cudaStreamSynchronize(st), "ex2 bias synchronise");
  if (!(std::fabs(b) < 1e-6)) return fail(ctx, RLB_ERR_NUMERIC, "hardware 2^x error outside its expected range");
  ctx->ex2_bias = b;
  ctx->ex2_measured = true;
  return RLB_OK;
}

// Table geometry of an EosView, including the split constants of the FP32 cell
// location (see EosView).
void eos_geometry(const rlb::EosTable& tab, rlbk::EosView* v) {
  v->y0 = tab.y0;
  v->inv_h = 1.0 / tab.h;
  v->n = tab.n;
  v->ih_hi = (float)v->inv_h;
  v->ih_lo = (float)(v->inv_h - (double)v->ih_hi);
  const double c = tab.y0 * v->inv_h;
  v->c_hi = (float)std::nearbyint(c);
  v->c_lo = (float)(c - (double)v->c_hi);
  v->ylo_f = (float)(tab.y0 + 2.0 * tab.h);
  v->yhi_f = (float)(tab.y0 + (tab.n - 4) * tab.h);
  v->y0_hi = (float)tab.y0;
  v->y0_lo = (float)(tab.y0 - (double)v->y0_hi);
}

// The FP32 table in device order: hi parts of every entry, then lo parts.
std::vector<float> table_hi_lo(const rlb::EosTable& tab) {
  const size_t n = tab.data.size();
  std::vector<float> t(2 * n);
  for (size_t i = 0; i < n; ++i) {
    t[i] = (float)tab.data[i];
    t[n + i] = (float)(tab.data[i] - (double)t[i]);
  }
  return t;
}

rlbk::EosView eos_view(const rlb_ctx* c) {
  rlbk::EosView v;
  v.tab = reinterpret_cast<const double*>(c->scratch + c->tab_off);
  v.tabf = reinterpret_cast<const float*>(c->scratch + c->tabf_off);
  v.tabl = v.tabf + c->tab.data.size();
  eos_geometry(c->tab, &v);
  return v;
}

Shape ctx_shape(const rlb_ctx* c) { return {c->ns, c->events.size()}; }

// CTA grid of the per-site kernels (see rlbk::locate_site)
dim3 site_grid(const rlb_ctx* c) {
  if (c->events.size() == 1) return dim3((unsigned)c->events[0].ny, (unsigned)c->events[0].nx, 1);
  return dim3((unsigned)c->ns, 1, 1);
}

// The same for kernels with two sites per CTA (rlbk::locate_sites<2>).
dim3 site_pair_grid(const rlb_ctx* c) {
  if (c->events.size() == 1) return dim3((unsigned)c->events[0].ny, (unsigned)(c->events[0].nx + 1) / 2, 1);
  return dim3((unsigned)((c->ns + 1) / 2), 1, 1);
}

rlbk::GridMap grid_map(const rlb_ctx* c, char* scr) {
  rlbk::GridMap g;
  g.ev = reinterpret_cast<const rlbk::EventInfo*>(scr + c->ev_off);
  g.loc = reinterpret_cast<const int2*>(scr + c->loc_off);
  g.n_events = (int)c->events.size();
  g.nx0 = c->events[0].nx;
  g.ny0 = c->events[0].ny;
  g.n_sites = (int)c->ns;
  return g;
}

// event, row and clock tables into a scratch block (host memory of the context)
rlb_status upload_tables(rlb_ctx* ctx, char* scr, cudaStream_t st) {
  if (!ctx->lines_mp.empty())
    RLB_CUDA(cudaMemcpyAsync(scr + ctx->lines_off, ctx->lines_mp.data(), ctx->lines_mp.size(),
                             cudaMemcpyHostToDevice, st), "line table upload");
  RLB_CUDA(cudaMemcpyAsync(scr + ctx->ev_off, ctx->events.data(), ctx->events.size() * sizeof(rlbk::EventInfo),
                           cudaMemcpyHostToDevice, st), "event table upload");
  if (ctx->events.size() > 1)
    RLB_CUDA(cudaMemcpyAsync(scr + ctx->loc_off, ctx->loc.data(), ctx->loc.size() * sizeof(int2),
                             cudaMemcpyHostToDevice, st), "site locator upload");
  return RLB_OK;
}

// the clock value travels as a kernel parameter: enqueued on the stream
// without a host copy that could synchronise it
__global__ void set_clock_kernel(rlbk::Clock* dst, rlbk::Clock v) { *dst = v; }

rlb_status set_clock(rlb_ctx* ctx, char* scr, double tau, cudaStream_t st) {
  const rlbk::Clock c{tau, 1.0 / tau, (float)(1.0 / tau), 0.f};
  set_clock_kernel<<<1, 1, 0, st>>>(reinterpret_cast<rlbk::Clock*>(scr + ctx->clock_off), c);
  RLB_CUDA(cudaGetLastError(), "clock upload");
  return RLB_OK;
}

// events of a configuration and, for a batch, the per-site locator (ctx->gp
// holds the shared parameters)
void set_events(rlb_ctx* ctx, const std::vector<rlbk::EventInfo>& ev) {
  ctx->events = ev;
  ctx->loc.clear();
  size_t ns = 0;
  for (size_t e = 0; e < ev.size(); ++e) ns += (size_t)ev[e].nx * ev[e].ny;
  ctx->ns = ns;
  if (ev.size() > 1) {
    ctx->loc.reserve(ns);
    for (size_t e = 0; e < ev.size(); ++e)
      for (int y = 0; y < ev[e].ny; ++y)
        for (int x = 0; x < ev[e].nx; ++x) ctx->loc.push_back(make_int2((int)e, (y << 16) | x));
  }
}

enum Kind { K_STAGE = 0, K_MATCH = 1, K_INIT = 2 };


// Event bracket around one launch when timing is enabled.
struct Timed {
  rlb_ctx* c;
  int kind;
  cudaStream_t st;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  Timed(rlb_ctx* c_, int k, cudaStream_t s) : c(c_), kind(k), st(s) {
    if (!c->timing) return;
    e0 = take();
    e1 = take();
    if (e0) cudaEventRecord(e0, st);
  }
  cudaEvent_t take() {
    if (c->ev_pool.empty()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
      return e;
    }
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  ~Timed() {
    if (!c->timing || !e0 || !e1) return;
    cudaEventRecord(e1, st);
    c->ev_pending.push_back({kind, {e0, e1}});
  }
};

rlbk::MatchArgs match_args(rlb_ctx* ctx, const double* mom, const double* lnM, double* obs) {
  rlbk::MatchArgs a;
  a.mom = mom;
  a.momf = reinterpret_cast<const float*>(mom);  // FP32 storage keeps kMomParts partial sums here
  a.inv2dx = 1.0 / (2.0 * ctx->gp.dx);
  a.grid = grid_map(ctx, ctx->scratch);
  a.clock = nullptr;
  a.dtau = ctx->gp.dtau;
  a.lnM = lnM;
  a.Tsite = reinterpret_cast<double*>(ctx->scratch + ctx->T_off);
  a.sc = reinterpret_cast<double*>(ctx->scratch + ctx->sc_off);
  a.scf = reinterpret_cast<float*>(ctx->scratch + ctx->scf_off);
  a.obs = obs;
  a.err = reinterpret_cast<int*>(ctx->scratch + ctx->err_off);
  a.eos = eos_view(ctx);
  a.ns = (int)ctx->ns;
  return a;
}

// One stage-kernel launch per call: the paired FP32 kernel where the lattice
// allows it (FP32 arithmetic, even N_xi and N_theta, whole warps per site), the
// generic one otherwise.
template <class S, class R, int NXI, int NTH, int NPH>
struct Stager {
  static constexpr bool kX2 =
      std::is_same<R, float>::value && NXI % 2 == 0 && NTH % 2 == 0 && (NTH * NPH) % 32 == 0;
  using MPS = rlbk::MPShape<NTH, NPH>;
  static constexpr bool kMP = kX2 && NXI <= 8 && MPS::NT % 32 == 0 && MPS::TS % 16 == 0 && 16 % MPS::H == 0;
  static constexpr int NL = NTH * NPH;
  // mirror-paired with the halo staged in shared memory by bulk copies: FP32
  // storage, two sites per CTA, 32-byte lines
  static constexpr bool kMPT = kMP && std::is_same<S, float>::value && MPS::SPC == 2 && NXI % 8 == 0;
  // variants the autotuner times: packed kernel with the register cap, packed
  // without it, generic kernel, packed with two sites per CTA (capped,
  // uncapped), mirror-paired kernel, mirror-paired with the staged halo (one
  // grid with an even number of sites per row; otherwise it runs the
  // mirror-paired kernel) (lattices the packed kernel does not take: generic
  // only)
  static constexpr int kVariants = kMPT ? 7 : kMP ? 6 : (kX2 ? 5 : 1);
  static constexpr int kDefault = kMP ? 5 : 0;  // used until rlb_autotune or rlb_set_stage_variant choose
  static_assert(kVariants <= RLB_MAX_STAGE_VARIANTS, "rlb_autotune output size");
  rlbk::StageArgs<S, R, NXI, NTH, NPH> a;
  rlbk::StageArgsX2<S, NXI, NTH, NPH> b;
  rlbk::StageArgsMP<S, NXI, NTH, NPH> c;
  rlbk::StageArgsMPT<S, NXI, NTH, NPH> d;
  bool mpt_ok = false;  // variant 6 applies to this grid
  // variant v launches another variant's kernel on this configuration
  bool runs_elsewhere(int v) const { return kMPT && v == 6 && !mpt_ok; }
  int mpt_prefetch = 0;
  dim3 grid, grid2;
  int variant = 0;

  // scr: the scratch block holding the event tables and the clock
  Stager(const rlb_ctx* ctx, char* scr, const double* sc, const float* scf, int* err) {
    variant = (ctx->stage_variant >= 0 && ctx->stage_variant < kVariants) ? ctx->stage_variant : kDefault;
    grid = site_grid(ctx);
    grid2 = site_pair_grid(ctx);
    const double dtau = ctx->gp.dtau, inv2dx = 1.0 / (2.0 * ctx->gp.dx);
    const rlbk::GridMap gm = grid_map(ctx, scr);
    const rlbk::Clock* clock = reinterpret_cast<const rlbk::Clock*>(scr + ctx->clock_off);
    if constexpr (kX2) {
      b.scf = scf;
      b.err = err;
      b.grid = gm;
      // the generic kernel as well, for variant 2
      a.sc = sc; a.scf = scf; a.err = err; a.grid = gm; a.clock = clock;
      a.milne_on = ctx->gp.metric == RLB_MILNE;
      a.dtau = dtau; a.inv2dx = inv2dx; a.dtau_r = (R)dtau; a.inv2dx_r = (R)inv2dx;
      a.Z = (R)ctx->eosp.Z;
      a.op = make_ops<R, NXI, NTH, NPH>(ctx->lat);
      b.clock = clock;
      b.milne_on = ctx->gp.metric == RLB_MILNE;
      b.dtau = dtau;
      b.dtau_r = (float)dtau;
      b.inv2dx_r = (float)inv2dx;
      b.log2Z = (float)std::log2(ctx->eosp.Z);
      b.op = make_ops_x2<NXI, NTH, NPH>(ctx->lat);
      if constexpr (kMP) {
        c.scf = scf; c.err = err; c.grid = gm; c.clock = clock;
        c.lines = reinterpret_cast<const rlbk::LinesMP<NTH / 2, (NTH / 2) * NPH>*>(scr + ctx->lines_off);
        c.milne_on = ctx->gp.metric == RLB_MILNE;
        c.dtau = dtau;
        c.dtau_r = (float)dtau;
        {
          const double zf = ctx->eosp.Z / (1.0 + ctx->ex2_bias);
          c.Zh = (float)zf;
          c.Zl = (float)(zf - (double)c.Zh);
        }
        c.op = make_ops_mp<NXI>(ctx->lat);
        c.prefetch_ahead = 0;
        int per_sm = 0, sms = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rlbk::stage_kernel_mp<S, NXI, NTH, NPH>,
                                                          MPS::NT, 0) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device) == cudaSuccess)
          c.prefetch_ahead = kPrefetchWaves * per_sm * sms;
        if constexpr (kMPT) {
          mpt_ok = ctx->events.size() == 1 && ctx->events[0].nx % 2 == 0 && make_halo_runs(ctx->lat, &d.runs);
          per_sm = 0;
          if (mpt_ok && cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                            &per_sm, rlbk::stage_kernel_mpt<NXI, NTH, NPH>, MPS::NT, 0) == cudaSuccess)
            mpt_prefetch = kPrefetchWaves * per_sm * sms;
        }
      }
    } else {
      a.sc = sc;
      a.scf = scf;
      a.err = err;
      a.grid = gm;
      a.clock = clock;
      a.milne_on = ctx->gp.metric == RLB_MILNE;
      a.dtau = dtau;
      a.inv2dx = inv2dx;
      a.dtau_r = (R)dtau;
      a.inv2dx_r = (R)inv2dx;
      a.Z = (R)ctx->eosp.Z;
      a.op = make_ops<R, NXI, NTH, NPH>(ctx->lat);
    }
  }

  // mode 0: predictor f_out = f_in + dtau rhs(f_in); mode 1: corrector
  // f_out = (f_base + f_in + dtau rhs(f_in)) / 2.  The time of f_in is the
  // device clock's.
  void launch(const S* f_in, const double* lnM_in, const S* f_base, const double* lnM_base, S* f_out,
              double* lnM_out, double* mom_out, int mode, cudaStream_t st) {
    if constexpr (kMP) {
      if (variant == 5) {
        c.f_in = f_in; c.lnM_in = lnM_in; c.f_base = f_base; c.lnM_base = lnM_base;
        c.f_out = f_out; c.lnM_out = lnM_out; c.momf_out = reinterpret_cast<float*>(mom_out);
        c.mode = mode;
        rlbk::stage_kernel_mp<S, NXI, NTH, NPH><<<MPS::SPC == 2 ? grid2 : grid, MPS::NT, 0, st>>>(c);
        return;
      }
      if constexpr (kMPT) {
        if (variant == 6) {
          c.f_in = f_in; c.lnM_in = lnM_in; c.f_base = f_base; c.lnM_base = lnM_base;
          c.f_out = f_out; c.lnM_out = lnM_out; c.momf_out = reinterpret_cast<float*>(mom_out);
          c.mode = mode;
          if (mpt_ok) {
            d.m = c;
            d.m.prefetch_ahead = mpt_prefetch;
            rlbk::stage_kernel_mpt<NXI, NTH, NPH><<<grid2, MPS::NT, 0, st>>>(d);
          } else {
            rlbk::stage_kernel_mp<S, NXI, NTH, NPH><<<grid2, MPS::NT, 0, st>>>(c);
          }
          return;
        }
      }
    }
    if constexpr (kX2) {
      if (variant != 2) {
        constexpr int kMinb2 = NL <= 96 ? 6 : 2;  // two sites per CTA: resident blocks per SM
        b.f_in = f_in; b.lnM_in = lnM_in; b.f_base = f_base; b.lnM_base = lnM_base;
        b.f_out = f_out; b.lnM_out = lnM_out; b.momf_out = reinterpret_cast<float*>(mom_out);
        b.mode = mode;
        if (variant == 0) rlbk::stage_kernel_x2<S, NXI, NTH, NPH><<<grid, NL, 0, st>>>(b);
        else if (variant == 1) rlbk::stage_kernel_x2<S, NXI, NTH, NPH, 1, 1><<<grid, NL, 0, st>>>(b);
        else if (variant == 3) rlbk::stage_kernel_x2<S, NXI, NTH, NPH, 2, kMinb2><<<grid2, NL, 0, st>>>(b);
        else rlbk::stage_kernel_x2<S, NXI, NTH, NPH, 2, 1><<<grid2, NL, 0, st>>>(b);
        return;
      }
    }
    {
      a.f_in = f_in; a.lnM_in = lnM_in; a.f_base = f_base; a.lnM_base = lnM_base;
      a.f_out = f_out; a.lnM_out = lnM_out; a.mom_out = mom_out; a.momf_out = reinterpret_cast<float*>(mom_out);
      a.mode = mode;
      rlbk::stage_kernel<S, R, NXI, NTH, NPH><<<grid, NL, 0, st>>>(a);
    }
  }
};

// clock: advanced by dtau in the launch (corrector matching) when non-null
rlb_status match(rlb_ctx* ctx, const double* mom, const double* lnM, double* obs, cudaStream_t st,
                 rlbk::Clock* clock = nullptr) {
  rlbk::MatchArgs a = match_args(ctx, mom, lnM, obs);
  a.clock = clock;
  {
    Timed tm(ctx, K_MATCH, st);
    const unsigned nb = (unsigned)((ctx->ns + kMatchThreads - 1) / kMatchThreads);
    if (ctx->gp.prec == RLB_F64) rlbk::match_kernel<false><<<nb, kMatchThreads, 0, st>>>(a);
    else rlbk::match_kernel<true><<<nb, kMatchThreads, 0, st>>>(a);
  }
  RLB_CUDA(cudaGetLastError(), "match_kernel launch");
  return RLB_OK;
}

template <class S, class R, int NXI, int NTH, int NPH>
struct Runner {
  static constexpr int NL = NTH * NPH;

  static rlb_status init(rlb_ctx* ctx, const double* eps_dev, cudaStream_t st) {
    ctx->scf_fresh = false;
    rlbk::InitArgs<S, R, NXI, NTH, NPH> a;
    a.eps0 = eps_dev;
    a.eps_scale = rlb::kHbarc * rlb::kHbarc * rlb::kHbarc;
    a.f = reinterpret_cast<S*>(ctx->state + ctx->f_off);
    a.lnM = reinterpret_cast<double*>(ctx->state + ctx->lnM_off);
    a.Tsite = reinterpret_cast<double*>(ctx->scratch + ctx->T_off);
    a.mom = reinterpret_cast<double*>(ctx->scratch + ctx->mom_off);
    a.momf = reinterpret_cast<float*>(ctx->scratch + ctx->mom_off);
    a.err = reinterpret_cast<int*>(ctx->scratch + ctx->err_off);
    a.eos = eos_view(ctx);
    a.Z = ctx->eosp.Z;
    a.family = ctx->gp.family;
    a.T0 = ctx->gp.T0;
    a.op = make_ops<R, NXI, NTH, NPH>(ctx->lat);
    for (int k = 0; k < NXI; ++k) a.s2d[k] = ctx->lat.s[k] * ctx->lat.s[k];
    // (T, M_eq, M) per site in the FP64 site-scalar scratch (free until the first matching)
    double* tsm = reinterpret_cast<double*>(ctx->scratch + ctx->sc_off);
    a.tsm = tsm;
    rlbk::InitSiteArgs b;
    b.eps0 = eps_dev; b.eps_scale = a.eps_scale; b.lnM = a.lnM; b.Tsite = a.Tsite; b.tsm = tsm; b.err = a.err;
    b.eos = a.eos; b.family = a.family; b.T0 = a.T0; b.ns = (int)ctx->ns;
    {
      Timed tm(ctx, K_INIT, st);
      rlbk::init_site_kernel<<<(unsigned)((ctx->ns + 127) / 128), 128, 0, st>>>(b);
      rlbk::init_kernel<S, R, NXI, NTH, NPH><<<(unsigned)ctx->ns, NL, 0, st>>>(a);
    }
    RLB_CUDA(cudaGetLastError(), "init_kernel launch");
    return RLB_OK;
  }

  // One predictor-corrector step = match(f) -> stage(f -> f*) -> match(f*) -> stage(f*, f -> f),
  // enqueued on st (the host clock is not advanced here).
  static rlb_status enqueue_step(rlb_ctx* ctx, cudaStream_t st, bool first_match = true) {
    S* f = reinterpret_cast<S*>(ctx->state + ctx->f_off);
    S* fs = reinterpret_cast<S*>(ctx->scratch + ctx->fs_off);
    double* m = reinterpret_cast<double*>(ctx->state + ctx->lnM_off);
    double* ms = reinterpret_cast<double*>(ctx->scratch + ctx->lnMs_off);
    double* mom = reinterpret_cast<double*>(ctx->scratch + ctx->mom_off);
    double* moms = reinterpret_cast<double*>(ctx->scratch + ctx->moms_off);
    Stager<S, R, NXI, NTH, NPH> sg(ctx, ctx->scratch, reinterpret_cast<const double*>(ctx->scratch + ctx->sc_off),
                                   reinterpret_cast<const float*>(ctx->scratch + ctx->scf_off),
                                   reinterpret_cast<int*>(ctx->scratch + ctx->err_off));
    rlbk::Clock* clock = reinterpret_cast<rlbk::Clock*>(ctx->scratch + ctx->clock_off);
    // predictor: f* = f + dtau RHS(f) at tau
    rlb_status r = first_match ? match(ctx, mom, m, nullptr, st) : RLB_OK;
    if (r) return r;
    {
      Timed tm(ctx, K_STAGE, st);
      sg.launch(f, m, f, m, fs, ms, moms, 0, st);
    }
    RLB_CUDA(cudaGetLastError(), "stage kernel (predictor) launch");
    // corrector: f = (f + f* + dtau RHS(f*))/2 at tau + dtau, in place over f;
    // its matching moves the device clock to tau + dtau
    r = match(ctx, moms, ms, nullptr, st, clock);
    if (r) return r;
    {
      Timed tm(ctx, K_STAGE, st);
      sg.launch(fs, ms, f, m, f, m, mom, 1, st);
    }
    RLB_CUDA(cudaGetLastError(), "stage kernel (corrector) launch");
    return RLB_OK;
  }

  // One step captured once as a CUDA graph on the context's own stream (all of
  // its launch parameters are the same from step to step: the time lives in the
  // device clock).  A failed capture turns graphs off for the context.
  static rlb_status ensure_graph(rlb_ctx* ctx, bool first_match = true) {
    cudaGraphExec_t* ge = first_match ? &ctx->gexec : &ctx->gexec_nm;
    if (*ge) return RLB_OK;
    if (!ctx->gstream) {
      RLB_CUDA(cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking), "graph stream");
      RLB_CUDA(cudaEventCreateWithFlags(&ctx->gev[0], cudaEventDisableTiming), "graph event");
      RLB_CUDA(cudaEventCreateWithFlags(&ctx->gev[1], cudaEventDisableTiming), "graph event");
    }
    RLB_CUDA(cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeThreadLocal), "graph capture");
    const rlb_status r = enqueue_step(ctx, ctx->gstream, first_match);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(ctx->gstream, &g);
    if (r != RLB_OK || e != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      ctx->graphs = false;
      return r != RLB_OK ? r : cuda_fail(ctx, e, "graph capture");
    }
    const cudaError_t ei = cudaGraphInstantiate(ge, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      *ge = nullptr;
      ctx->graphs = false;
      return cuda_fail(ctx, ei, "graph instantiate");
    }
    return RLB_OK;
  }

  static rlb_status step(rlb_ctx* ctx, int nsteps, cudaStream_t st) {
    if (nsteps <= 0) return RLB_OK;
    const bool skip = ctx->scf_fresh;  // the first step's matching is already done
    ctx->scf_fresh = false;
    const bool graphs = ctx->graphs && !ctx->timing && (!skip || ensure_graph(ctx, false) == RLB_OK) &&
                        ((skip && nsteps == 1) || ensure_graph(ctx) == RLB_OK);
    if (graphs) {
      RLB_CUDA(cudaEventRecord(ctx->gev[0], st), "graph order");
      RLB_CUDA(cudaStreamWaitEvent(ctx->gstream, ctx->gev[0], 0), "graph order");
      for (int s = 0; s < nsteps; ++s) {
        RLB_CUDA(cudaGraphLaunch(s == 0 && skip ? ctx->gexec_nm : ctx->gexec, ctx->gstream), "graph launch");
        ctx->tau += ctx->gp.dtau;
      }
      RLB_CUDA(cudaEventRecord(ctx->gev[1], ctx->gstream), "graph order");
      RLB_CUDA(cudaStreamWaitEvent(st, ctx->gev[1], 0), "graph order");
      return RLB_OK;
    }
    for (int s = 0; s < nsteps; ++s) {
      rlb_status r = enqueue_step(ctx, st, !(s == 0 && skip));
      if (r) return r;
      ctx->tau += ctx->gp.dtau;
    }
    return RLB_OK;
  }

  // Time every stage-kernel variant on predictor launches over the current state
  // and keep the fastest; f, ln M and the clock are untouched, the Newton
  // starting temperatures are restored.
  static rlb_status autotune(rlb_ctx* ctx, double* ms, int* nvar, cudaStream_t st) {
    constexpr int NV = Stager<S, R, NXI, NTH, NPH>::kVariants;
    S* f = reinterpret_cast<S*>(ctx->state + ctx->f_off);
    S* fs = reinterpret_cast<S*>(ctx->scratch + ctx->fs_off);
    double* m = reinterpret_cast<double*>(ctx->state + ctx->lnM_off);
    double* ms_ = reinterpret_cast<double*>(ctx->scratch + ctx->lnMs_off);
    double* mom = reinterpret_cast<double*>(ctx->scratch + ctx->mom_off);
    double* moms = reinterpret_cast<double*>(ctx->scratch + ctx->moms_off);
    double* Tsite = reinterpret_cast<double*>(ctx->scratch + ctx->T_off);
    double* Tsave = reinterpret_cast<double*>(ctx->scratch + ctx->eps_off);  // free between steps
    RLB_CUDA(cudaMemcpyAsync(Tsave, Tsite, ctx->ns * sizeof(double), cudaMemcpyDeviceToDevice, st), "autotune save");
    rlb_status r = match(ctx, mom, m, nullptr, st);
    if (r) return r;
    cudaEvent_t e0, e1;
    RLB_CUDA(cudaEventCreate(&e0), "autotune event");
    RLB_CUDA(cudaEventCreate(&e1), "autotune event");
    const int keep = ctx->stage_variant;
    int best = 0;
    for (int v = 0; v < NV; ++v) {
      ctx->stage_variant = v;
      Stager<S, R, NXI, NTH, NPH> sg(ctx, ctx->scratch, reinterpret_cast<const double*>(ctx->scratch + ctx->sc_off),
                                     reinterpret_cast<const float*>(ctx->scratch + ctx->scf_off),
                                     reinterpret_cast<int*>(ctx->scratch + ctx->err_off));
      if (sg.runs_elsewhere(v)) {  // not a kernel of its own here: never chosen
        if (ms) ms[v] = -1.0;
        continue;
      }
      sg.launch(f, m, f, m, fs, ms_, moms, 0, st);  // warm-up
      cudaEventRecord(e0, st);
      for (int k = 0; k < 3; ++k) sg.launch(f, m, f, m, fs, ms_, moms, 0, st);
      cudaEventRecord(e1, st);
      const cudaError_t ce = cudaEventSynchronize(e1);
      if (ce != cudaSuccess) {
        ctx->stage_variant = keep;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return cuda_fail(ctx, ce, "autotune launch");
      }
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      if (ms) ms[v] = t / 3.0;
      if (v > 0 && ms && ms[v] < ms[best]) best = v;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    RLB_CUDA(cudaMemcpyAsync(Tsite, Tsave, ctx->ns * sizeof(double), cudaMemcpyDeviceToDevice, st), "autotune restore");
    RLB_CUDA(cudaStreamSynchronize(st), "autotune synchronise");
    ctx->stage_variant = best;
    drop_graphs(ctx);  // the captured step used the previous choice
    ctx->scf_fresh = false;
    if (nvar) *nvar = NV;
    return RLB_OK;
  }
};

// Grid observables of the current state into out_dev[2] (device): matching of
// the stored moments (for B), per-site partial sums, one fixed-order reduction.
template <class S, class R, int NXI, int NTH, int NPH>
rlb_status observables(rlb_ctx* ctx, double* out_dev, cudaStream_t st) {
  constexpr int NL = NTH * NPH;
  const double* mom = reinterpret_cast<const double*>(ctx->scratch + ctx->mom_off);
  const double* lnM = reinterpret_cast<const double*>(ctx->state + ctx->lnM_off);
  rlb_status r = match(ctx, mom, lnM, nullptr, st);
  if (r) return r;
  rlbk::ObsArgs<S, R, NXI, NTH, NPH> a;
  a.f = reinterpret_cast<const S*>(ctx->state + ctx->f_off);
  a.lnM = lnM;
  a.sc = ctx->gp.prec == RLB_F64 ? reinterpret_cast<const double*>(ctx->scratch + ctx->sc_off) : nullptr;
  a.scf = reinterpret_cast<const float*>(ctx->scratch + ctx->scf_off);
  a.part = reinterpret_cast<double*>(ctx->scratch + ctx->moms_off);  // free between steps
  a.op = make_ops<R, NXI, NTH, NPH>(ctx->lat);
  rlbk::observables_kernel<S, R, NXI, NTH, NPH><<<(unsigned)ctx->ns, NL, 0, st>>>(a);
  RLB_CUDA(cudaGetLastError(), "observables_kernel launch");
  rlbk::observables_reduce_kernel<<<1, 1024, 0, st>>>(a.part, (int)ctx->ns, out_dev);
  RLB_CUDA(cudaGetLastError(), "observables_reduce_kernel launch");
  return RLB_OK;
}

// ---------------------------------------------------------------------------
// adjoint of the step (FP64 arithmetic): see rlb_adjoint.cuh
// ---------------------------------------------------------------------------
template <class S, class R, int NXI, int NTH, int NPH>
struct Adjoint {
  static constexpr int NL = NTH * NPH;
  static double* D(rlb_ctx* c, size_t off) { return reinterpret_cast<double*>(c->adj + off); }
  template <class AR>
  static AR* P(rlb_ctx* c, size_t off) { return reinterpret_cast<AR*>(c->adj + off); }

  // adjoint of one stage with input (f_in, lnM_in): from (ob, lb) to (fout, lout);
  // AR: arithmetic of the per-node adjoint work and type of the per-node arrays
  // acc nonzero: fout, lout += acc x their previous values (instead of overwriting them).
  // FP32 adjoint on the FP32-arithmetic storage paths: the moments, the
  // matching and its temperature of f_in may come from the forward recompute
  // (momf_src, scf_src, T_src), the exact point the forward step used, instead
  // of being recomputed here.
  template <class AR>
  static rlb_status stage(rlb_ctx* ctx, const S* f_in, const double* lnM_in, double milne, double c,
                          const AR* ob, const double* lb, AR* fout, double* lout, cudaStream_t st,
                          double acc = 0.0, const float* momf_src = nullptr, const float* scf_src = nullptr,
                          double* T_src = nullptr) {
    const auto opd = make_ops<double, NXI, NTH, NPH>(ctx->lat);
    const auto opa = make_ops<AR, NXI, NTH, NPH>(ctx->lat);
    const rlbk::GridMap gm = grid_map(ctx, ctx->scratch);
    int* err = reinterpret_cast<int*>(ctx->scratch + ctx->err_off);
    constexpr bool kF32 = std::is_same<AR, float>::value;
    const unsigned nbm = (unsigned)((ctx->ns + kMatchThreads - 1) / kMatchThreads);
    const bool given = kF32 && scf_src;
    const float* momf_use = given ? momf_src : P<float>(ctx, ctx->a_momf);
    const float* scf_use = given ? scf_src : P<float>(ctx, ctx->a_scf);
    double* T_use = given ? T_src : D(ctx, ctx->a_T);
    if (given) {
    } else if constexpr (kF32) {  // FP32 moment partials and the FP32 matching (double-FP32 final steps) of f_in
      rlbk::MomentsArgs<S, float, NXI, NTH, NPH> a;
      a.f = f_in;
      a.mom = nullptr;
      a.momf = P<float>(ctx, ctx->a_momf);
      a.op = opa;
      rlbk::moments_kernel<S, float, NXI, NTH, NPH><<<(unsigned)ctx->ns, NL, 0, st>>>(a);
      RLB_CUDA(cudaGetLastError(), "adjoint moments launch");
      rlbk::MatchArgs ma = match_args(ctx, nullptr, lnM_in, nullptr);
      ma.momf = P<float>(ctx, ctx->a_momf);
      ma.Tsite = D(ctx, ctx->a_T);
      ma.sc = nullptr;
      ma.scf = P<float>(ctx, ctx->a_scf);
      rlbk::match_kernel<true><<<nbm, kMatchThreads, 0, st>>>(ma);
      RLB_CUDA(cudaGetLastError(), "adjoint matching launch");
    } else {  // FP64 moments and matching of f_in
      rlbk::MomentsArgs<S, double, NXI, NTH, NPH> a;
      a.f = f_in;
      a.mom = D(ctx, ctx->a_mom);
      a.momf = nullptr;
      a.op = opd;
      rlbk::moments_kernel<S, double, NXI, NTH, NPH><<<(unsigned)ctx->ns, NL, 0, st>>>(a);
      RLB_CUDA(cudaGetLastError(), "adjoint moments launch");
      rlbk::MatchArgs ma = match_args(ctx, D(ctx, ctx->a_mom), lnM_in, nullptr);
      ma.Tsite = D(ctx, ctx->a_T);
      ma.sc = D(ctx, ctx->a_sc);
      ma.scf = nullptr;
      rlbk::match_kernel<false><<<nbm, kMatchThreads, 0, st>>>(ma);
      RLB_CUDA(cudaGetLastError(), "adjoint matching launch");
    }
    {
      rlbk::AdjStageArgs<S, AR, NXI, NTH, NPH> a;
      a.f_in = f_in; a.sc = D(ctx, ctx->a_sc); a.scf = kF32 ? scf_use : nullptr;
      a.ob = ob; a.lb = lb;
      a.rbar = P<AR>(ctx, ctx->a_rb); a.fbar = P<AR>(ctx, ctx->a_fb); a.sbar = D(ctx, ctx->a_sbar);
      a.err = err; a.grid = gm; a.milne = (AR)milne; a.c = (AR)c; a.dtau = (AR)ctx->gp.dtau;
      a.inv2dx = (AR)(1.0 / (2.0 * ctx->gp.dx)); a.Z = (AR)ctx->eosp.Z; a.op = opa;
      rlbk::adj_stage1<S, AR, NXI, NTH, NPH><<<site_grid(ctx), NL, 0, st>>>(a);
      RLB_CUDA(cudaGetLastError(), "adj_stage1 launch");
    }
    {
      rlbk::AdjMatchArgs a;
      a.mom = D(ctx, ctx->a_mom); a.momf = kF32 ? momf_use : nullptr;
      a.Tstart = kF32 ? T_use : D(ctx, ctx->a_T);  // the matching made: the EOS inversion starts there
      a.scf = kF32 ? scf_use : nullptr;  // FP32: u and T from that matching
      a.lnM = lnM_in; a.sbar = D(ctx, ctx->a_sbar); a.mbar = D(ctx, ctx->a_mbar);
      a.lbar = D(ctx, ctx->a_lbar); a.ebar = D(ctx, ctx->a_ebar); a.err = err; a.eos = eos_view(ctx);
      a.grid = gm; a.ns = (int)ctx->ns;
      // one warp per CTA: the FP64-bound per-site work spread over as many SMs as possible
      rlbk::adj_match<<<(unsigned)((ctx->ns + 31) / 32), 32, 0, st>>>(a);
      RLB_CUDA(cudaGetLastError(), "adj_match launch");

    }
    {
      rlbk::AdjAssembleArgs<AR, NXI, NTH, NPH> a;
      a.fbar = P<AR>(ctx, ctx->a_fb); a.rbar = P<AR>(ctx, ctx->a_rb); a.mbar = D(ctx, ctx->a_mbar);
      a.sbar = D(ctx, ctx->a_sbar); a.lbar = D(ctx, ctx->a_lbar); a.lb = lb; a.fout = fout; a.lout = lout;
      a.acc = (AR)acc;
      a.err = err; a.grid = gm; a.c = c; a.inv2dx = 1.0 / (2.0 * ctx->gp.dx); a.op = opa;
      a.inv2dx_t = (AR)a.inv2dx;
      rlbk::adj_stage3<AR, NXI, NTH, NPH><<<site_grid(ctx), NL, 0, st>>>(a);
      RLB_CUDA(cudaGetLastError(), "adj_stage3 launch");
    }
    return RLB_OK;
  }


  // the adjoint buffers hold the adjoints of a step's output; the context state
  // is that step's input (at ctx->tau): replace them by the adjoints of the input
  // the step's input state: the context's (null pointers) or a device blob's
  struct Input {
    const S* f = nullptr;
    const double* lnM = nullptr;
    const double* mom = nullptr;
  };
  static rlb_status step(rlb_ctx* ctx, cudaStream_t st, Input in = Input()) {
    ctx->scf_fresh = false;
    return ctx->adj_prec == RLB_F32 ? step_t<float>(ctx, st, in) : step_t<double>(ctx, st, in);
  }
  template <class AR>
  static rlb_status step_t(rlb_ctx* ctx, cudaStream_t st, Input in) {
    const S* f = in.f ? in.f : reinterpret_cast<S*>(ctx->state + ctx->f_off);
    S* fs = reinterpret_cast<S*>(ctx->scratch + ctx->fs_off);
    const double* m = in.lnM ? in.lnM : reinterpret_cast<double*>(ctx->state + ctx->lnM_off);
    double* ms = reinterpret_cast<double*>(ctx->scratch + ctx->lnMs_off);
    const double* mom = in.mom ? in.mom : reinterpret_cast<double*>(ctx->scratch + ctx->mom_off);
    double* moms = reinterpret_cast<double*>(ctx->scratch + ctx->moms_off);
    // the predictor output f*, ln M* exactly as the forward run made it
    rlb_status r = match(ctx, mom, m, nullptr, st);
    if (r) return r;
    Stager<S, R, NXI, NTH, NPH> sg(ctx, ctx->scratch, reinterpret_cast<const double*>(ctx->scratch + ctx->sc_off),
                                   reinterpret_cast<const float*>(ctx->scratch + ctx->scf_off),
                                   reinterpret_cast<int*>(ctx->scratch + ctx->err_off));
    sg.launch(f, m, f, m, fs, ms, moms, 0, st);
    RLB_CUDA(cudaGetLastError(), "adjoint predictor recompute");
    const double tau = ctx->tau, dt = ctx->gp.dtau;
    const bool milne = ctx->gp.metric == RLB_MILNE;
    // FP32 adjoint on an FP32-arithmetic storage path: the matchings of f and
    // f* as the forward step made them (moment partials of the stage kernels,
    // the same Newton starts), no recomputed moments
    constexpr bool kReuse = std::is_same<AR, float>::value && std::is_same<R, float>::value;
    float* scf = reinterpret_cast<float*>(ctx->scratch + ctx->scf_off);
    double* Tsite = reinterpret_cast<double*>(ctx->scratch + ctx->T_off);
    if constexpr (kReuse) {  // matching of f* into the adjoint's buffers, from T(f) as the forward did
      RLB_CUDA(cudaMemcpyAsync(D(ctx, ctx->a_T), Tsite, ctx->ns * sizeof(double), cudaMemcpyDeviceToDevice, st),
               "adjoint Newton start copy");
      rlbk::MatchArgs ma = match_args(ctx, moms, ms, nullptr);
      ma.Tsite = D(ctx, ctx->a_T);
      ma.sc = nullptr;
      ma.scf = P<float>(ctx, ctx->a_scf);
      rlbk::match_kernel<true><<<(unsigned)((ctx->ns + kMatchThreads - 1) / kMatchThreads), kMatchThreads, 0, st>>>(ma);
      RLB_CUDA(cudaGetLastError(), "adjoint matching launch");
    }
    // corrector f_new = (f + f* + dtau RHS(f*)) / 2
    r = stage<AR>(ctx, fs, ms, milne ? 1.0 / (tau + dt) : 0.0, 0.5, P<AR>(ctx, ctx->a_f), D(ctx, ctx->a_l),
                  P<AR>(ctx, ctx->a_fb), D(ctx, ctx->a_lin), st, 0.0,
                  kReuse ? reinterpret_cast<const float*>(moms) : nullptr,
                  kReuse ? P<float>(ctx, ctx->a_scf) : nullptr, kReuse ? D(ctx, ctx->a_T) : nullptr);
    if (r) return r;
    // predictor f* = f + dtau RHS(f); its adjoint adds to the corrector's base
    // term (1/2) fbar_new, ln M likewise (in the assembly kernel, in place)
    return stage<AR>(ctx, f, m, milne ? 1.0 / tau : 0.0, 1.0, P<AR>(ctx, ctx->a_fb), D(ctx, ctx->a_lin),
                     P<AR>(ctx, ctx->a_f), D(ctx, ctx->a_l), st, 0.5,
                     kReuse ? reinterpret_cast<const float*>(mom) : nullptr, kReuse ? scf : nullptr,
                     kReuse ? Tsite : nullptr);
  }

  // seed: adjoints of v2 (p_perp-weighted) of the current state; out[0] = v2
  static rlb_status seed(rlb_ctx* ctx, double* out, cudaStream_t st) {
    return ctx->adj_prec == RLB_F32 ? seed_t<float>(ctx, out, st) : seed_t<double>(ctx, out, st);
  }
  template <class AR>
  static rlb_status seed_t(rlb_ctx* ctx, double* out, cudaStream_t st) {
    double* dev = reinterpret_cast<double*>(ctx->scratch + ctx->eps_off);
    rlb_status r = observables<S, R, NXI, NTH, NPH>(ctx, dev, st);
    if (r) return r;
    rlbk::SeedArgs<S, AR, NXI, NTH, NPH> a;
    a.lnM = reinterpret_cast<const double*>(ctx->state + ctx->lnM_off);
    a.part = reinterpret_cast<const double*>(ctx->scratch + ctx->moms_off);
    a.tot = dev + 2;
    a.fbar = P<AR>(ctx, ctx->a_f);
    a.lbar = D(ctx, ctx->a_l);
    a.op = make_ops<double, NXI, NTH, NPH>(ctx->lat);
    rlbk::adj_seed_v2<S, AR, NXI, NTH, NPH><<<(unsigned)ctx->ns, NL, 0, st>>>(a);
    RLB_CUDA(cudaGetLastError(), "adjoint seed launch");
    RLB_CUDA(cudaMemsetAsync(D(ctx, ctx->a_eta), 0, sizeof(double), st), "adjoint eta reset");
    RLB_CUDA(cudaMemsetAsync(D(ctx, ctx->a_ebar), 0, ctx->ns * sizeof(double), st), "adjoint eta reset");
    RLB_CUDA(cudaMemcpyAsync(out, dev + 1, sizeof(double), cudaMemcpyDeviceToHost, st), "v2 download");
    RLB_CUDA(cudaStreamSynchronize(st), "adjoint seed synchronise");
    return RLB_OK;
  }

  // initial condition: p[0] = eps0 (device, GeV/fm^3), p[1] = basis (device,
  // n x ns), p[2] = n, p[3] = output (host, n + 1: dJ/dA_i, then dJ/d(eta/s))
  static rlb_status ic(rlb_ctx* ctx, const double* eps0, const double* basis, int n, double* out, cudaStream_t st) {
    return ctx->adj_prec == RLB_F32 ? ic_t<float>(ctx, eps0, basis, n, out, st)
                                    : ic_t<double>(ctx, eps0, basis, n, out, st);
  }
  template <class AR>
  static rlb_status ic_t(rlb_ctx* ctx, const double* eps0, const double* basis, int n, double* out,
                         cudaStream_t st) {
    rlbk::AdjIcArgs<S, AR, NXI, NTH, NPH> a;
    a.eps0 = eps0; a.fbar = P<AR>(ctx, ctx->a_f); a.lbar = D(ctx, ctx->a_l); a.epsbar = D(ctx, ctx->a_eps);
    a.err = reinterpret_cast<int*>(ctx->scratch + ctx->err_off); a.eos = eos_view(ctx);
    a.eps_scale = rlb::kHbarc * rlb::kHbarc * rlb::kHbarc; a.Z = ctx->eosp.Z;
    a.op = make_ops<double, NXI, NTH, NPH>(ctx->lat);
    rlbk::adj_ic<S, AR, NXI, NTH, NPH><<<(unsigned)ctx->ns, NL, 0, st>>>(a);
    RLB_CUDA(cudaGetLastError(), "adj_ic launch");
    // the eta/s adjoint: per-site sums over every stage, summed over the sites
    rlbk::sum_kernel<<<1, 1024, 0, st>>>(D(ctx, ctx->a_ebar), ctx->ns, D(ctx, ctx->a_eta), 0);
    RLB_CUDA(cudaGetLastError(), "adjoint eta sum launch");
    double* proj = D(ctx, ctx->a_ebar);  // n <= ns doubles (checked by the caller)
    if (n > 0) {
      rlbk::project_kernel<<<(unsigned)n, 1024, 0, st>>>(basis, D(ctx, ctx->a_eps), ctx->ns, proj);
      RLB_CUDA(cudaGetLastError(), "projection launch");
      RLB_CUDA(cudaMemcpyAsync(out, proj, n * sizeof(double), cudaMemcpyDeviceToHost, st), "gradient download");
    }
    RLB_CUDA(cudaMemcpyAsync(out + n, D(ctx, ctx->a_eta), sizeof(double), cudaMemcpyDeviceToHost, st),
             "eta gradient download");
    RLB_CUDA(cudaStreamSynchronize(st), "adjoint ic synchronise");
    return RLB_OK;
  }
};

enum Op { OP_INIT, OP_STEP, OP_MOMENTS, OP_OBS, OP_TUNE, OP_NVAR, OP_ADJ_SEED, OP_ADJ_STEP, OP_ADJ_IC };

// arguments of the adjoint initial-condition call, passed through dispatch
struct AdjIcCall {
  const double* eps0;
  const double* basis;
  int n;
  double* out;
};

template <class S, class R, int NXI, int NTH, int NPH>
rlb_status run_op(rlb_ctx* c, Op op, int n, double* p, cudaStream_t st) {
  using Rn = Runner<S, R, NXI, NTH, NPH>;
  if (op == OP_INIT) return Rn::init(c, p, st);
  if (op == OP_STEP) return Rn::step(c, n, st);
  if (op == OP_ADJ_SEED) return Adjoint<S, R, NXI, NTH, NPH>::seed(c, p, st);
  if (op == OP_ADJ_STEP) {
    typename Adjoint<S, R, NXI, NTH, NPH>::Input in;
    if (p) {  // a device state blob: f, ln M and the moments read in place
      const char* const* b = reinterpret_cast<const char* const*>(p);
      const uint64_t* o = reinterpret_cast<const uint64_t*>(b + 1);
      in.f = reinterpret_cast<const S*>(b[0] + o[0]);
      in.lnM = reinterpret_cast<const double*>(b[0] + o[1]);
      in.mom = reinterpret_cast<const double*>(b[0] + o[3]);
    }
    return Adjoint<S, R, NXI, NTH, NPH>::step(c, st, in);
  }
  if (op == OP_ADJ_IC) {
    const AdjIcCall* a = reinterpret_cast<const AdjIcCall*>(p);
    return Adjoint<S, R, NXI, NTH, NPH>::ic(c, a->eps0, a->basis, a->n, a->out, st);
  }
  if (op == OP_TUNE) {
    int nv = 0;
    rlb_status r = Rn::autotune(c, p, &nv, st);
    if (!r && p) p[RLB_MAX_STAGE_VARIANTS] = nv;  // p: the variant times, then their count
    return r;
  }
  if (op == OP_NVAR) {
    p[0] = Stager<S, R, NXI, NTH, NPH>::kVariants;
    return RLB_OK;
  }
  if (op == OP_OBS) return observables<S, R, NXI, NTH, NPH>(c, p, st);
  return RLB_ERR_ARG;
}

template <int NXI, int NTH, int NPH>
rlb_status run_prec(rlb_ctx* c, Op op, int n, double* p, cudaStream_t st) {
  switch (c->gp.prec) {
    case RLB_F64:
      if constexpr (NXI * NTH * NPH <= 1024) return run_op<double, double, NXI, NTH, NPH>(c, op, n, p, st);
      else return fail(c, RLB_ERR_ARG, "FP64 storage supports at most 1024 nodes per site");
    case RLB_F32: return run_op<float, float, NXI, NTH, NPH>(c, op, n, p, st);
    case RLB_BF16: return run_op<__nv_bfloat16, float, NXI, NTH, NPH>(c, op, n, p, st);
  }
  return fail(c, RLB_ERR_ARG, "unknown precision");
}

rlb_status dispatch(rlb_ctx* c, Op op, int n, double* p, cudaStream_t st) {
  const int a = c->gp.n_xi, b = c->gp.n_theta, d = 2 * c->gp.n_phi_half;
  if (a == 8 && b == 8 && d == 12) return run_prec<8, 8, 12>(c, op, n, p, st);
  if (a == 16 && b == 8 && d == 16) return run_prec<16, 8, 16>(c, op, n, p, st);
  if (a == 5 && b == 5 && d == 2) return run_prec<5, 5, 2>(c, op, n, p, st);
  if (a == 6 && b == 4 && d == 6) return run_prec<6, 4, 6>(c, op, n, p, st);
  if (a == 8 && b == 8 && d == 2) return run_prec<8, 8, 2>(c, op, n, p, st);
  return fail(c, RLB_ERR_ARG, "unsupported lattice shape");
}

rlb_status set_device(rlb_ctx* ctx) {
  RLB_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
  return RLB_OK;
}

// ---------------------------------------------------------------------------
// Step variant that allocates nothing: its scratch lives in one file-scope
// device array, shared by every call in the process on a given device.
// ---------------------------------------------------------------------------
constexpr size_t kStaticScratchBytes = (size_t)24 << 20;  // 24 MiB per device
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
static void* g_static_ptr[kMaxDevices];  // device address of g_static_scratch, per device
static std::mutex g_static_mu;

// Device address of the static scratch on the current device (looked up once).
rlb_status static_scratch(rlb_ctx* ctx, char** out) {
  if (ctx->device < 0 || ctx->device >= kMaxDevices) return fail(ctx, RLB_ERR_ARG, "device id out of range");
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[ctx->device]) {
    void* p = nullptr;
    RLB_CUDA(cudaGetSymbolAddress(&p, g_static_scratch), "cudaGetSymbolAddress(static scratch)");
    g_static_ptr[ctx->device] = p;
  }
  *out = static_cast<char*>(g_static_ptr[ctx->device]);
  return RLB_OK;
}

template <class S, class R, int NXI, int NTH, int NPH>
rlb_status step_static(rlb_ctx* ctx, char* state, char* scr, int nsteps, cudaStream_t st) {
  constexpr int NL = NTH * NPH;
  // same layout as the bound scratch, rooted at the static array
  size_t sb, xb;
  rlb_ctx L;
  layout(ctx->gp, ctx_shape(ctx), (size_t)ctx->eosp.points, &sb, &xb, &L);
  S* f = reinterpret_cast<S*>(state + ctx->f_off);
  double* m = reinterpret_cast<double*>(state + ctx->lnM_off);
  S* fs = reinterpret_cast<S*>(scr + L.fs_off);
  double* ms = reinterpret_cast<double*>(scr + L.lnMs_off);
  double* mom = reinterpret_cast<double*>(scr + L.mom_off);
  double* moms = reinterpret_cast<double*>(scr + L.moms_off);
  double* Tsite = reinterpret_cast<double*>(scr + L.T_off);
  int* err = reinterpret_cast<int*>(scr + L.err_off);
  rlbk::EosView ev;
  ev.tab = reinterpret_cast<const double*>(scr + L.tab_off);
  ev.tabf = reinterpret_cast<const float*>(scr + L.tabf_off);
  ev.tabl = ev.tabf + ctx->tab.data.size();
  eos_geometry(ctx->tab, &ev);
  // contents left by earlier calls are not trusted: EOS tables, Newton starts,
  // error word and the moments of the input are rebuilt here
  RLB_CUDA(cudaMemcpyAsync(scr + L.tab_off, ctx->tab.data.data(), ctx->tab.data.size() * sizeof(double),
                           cudaMemcpyHostToDevice, st), "static EOS table upload");
  {
    const std::vector<float> tf = table_hi_lo(ctx->tab);
    RLB_CUDA(cudaMemcpyAsync(scr + L.tabf_off, tf.data(), tf.size() * sizeof(float),
                             cudaMemcpyHostToDevice, st), "static FP32 EOS table upload");
    RLB_CUDA(cudaStreamSynchronize(st), "static table upload synchronise");
  }
  {
    rlb_status rb = measure_ex2_bias(ctx, scr, L.eps_off, st);
    if (rb) return rb;
  }
  RLB_CUDA(cudaMemsetAsync(Tsite, 0, ctx->ns * sizeof(double), st), "static Newton starts reset");
  RLB_CUDA(cudaMemsetAsync(err, 0, 256, st), "static error word reset");
  rlb_status r0 = upload_tables(ctx, scr, st);
  if (r0) return r0;
  r0 = set_clock(ctx, scr, ctx->tau, st);
  if (r0) return r0;
  RLB_CUDA(cudaStreamSynchronize(st), "static table upload synchronise");
  const auto op = make_ops<R, NXI, NTH, NPH>(ctx->lat);
  {
    rlbk::MomentsArgs<S, R, NXI, NTH, NPH> a;
    a.f = f;
    a.mom = mom;
    a.momf = reinterpret_cast<float*>(mom);
    a.op = op;
    rlbk::moments_kernel<S, R, NXI, NTH, NPH><<<(unsigned)ctx->ns, NL, 0, st>>>(a);
    RLB_CUDA(cudaGetLastError(), "moments_kernel launch");
  }
  rlbk::MatchArgs ma;
  ma.Tsite = Tsite;
  ma.sc = reinterpret_cast<double*>(scr + L.sc_off);
  ma.scf = reinterpret_cast<float*>(scr + L.scf_off);
  ma.obs = nullptr;
  ma.err = err;
  ma.eos = ev;
  ma.grid = grid_map(ctx, scr);
  ma.inv2dx = 1.0 / (2.0 * ctx->gp.dx);
  ma.ns = (int)ctx->ns;
  ma.dtau = ctx->gp.dtau;
  rlbk::Clock* clock = reinterpret_cast<rlbk::Clock*>(scr + L.clock_off);
  auto run_match = [&](const double* mm, const double* lnM, rlbk::Clock* adv) -> rlb_status {
    ma.mom = mm;
    ma.momf = reinterpret_cast<const float*>(mm);
    ma.lnM = lnM;
    ma.clock = adv;
    const unsigned nb = (unsigned)((ctx->ns + kMatchThreads - 1) / kMatchThreads);
    if (ctx->gp.prec == RLB_F64) rlbk::match_kernel<false><<<nb, kMatchThreads, 0, st>>>(ma);
    else rlbk::match_kernel<true><<<nb, kMatchThreads, 0, st>>>(ma);
    RLB_CUDA(cudaGetLastError(), "match_kernel launch");
    return RLB_OK;
  };
  Stager<S, R, NXI, NTH, NPH> sg(ctx, scr, ma.sc, ma.scf, err);
  for (int s = 0; s < nsteps; ++s) {
    rlb_status r = run_match(mom, m, nullptr);
    if (r) return r;
    sg.launch(f, m, f, m, fs, ms, moms, 0, st);
    RLB_CUDA(cudaGetLastError(), "stage kernel (predictor) launch");
    r = run_match(moms, ms, clock);
    if (r) return r;
    sg.launch(fs, ms, f, m, f, m, mom, 1, st);
    RLB_CUDA(cudaGetLastError(), "stage kernel (corrector) launch");
    ctx->tau += ctx->gp.dtau;
  }
  // report numeric failures of this call (the error word is shared)
  int word = 0;
  RLB_CUDA(cudaMemcpyAsync(&word, err, sizeof(int), cudaMemcpyDeviceToHost, st), "static error word read");
  RLB_CUDA(cudaStreamSynchronize(st), "static step synchronise");
  if (word)
    return fail(ctx, (word & rlbk::ERR_TIMEOUT) ? RLB_ERR_TIMEOUT : RLB_ERR_NUMERIC,
                "device error word set in the static-scratch step");
  return RLB_OK;
}

template <int NXI, int NTH, int NPH>
rlb_status step_static_prec(rlb_ctx* c, char* state, char* scr, int n, cudaStream_t st) {
  switch (c->gp.prec) {
    case RLB_F64:
      if constexpr (NXI * NTH * NPH <= 1024) return step_static<double, double, NXI, NTH, NPH>(c, state, scr, n, st);
      else return fail(c, RLB_ERR_ARG, "FP64 storage supports at most 1024 nodes per site");
    case RLB_F32: return step_static<float, float, NXI, NTH, NPH>(c, state, scr, n, st);
    case RLB_BF16: return step_static<__nv_bfloat16, float, NXI, NTH, NPH>(c, state, scr, n, st);
  }
  return fail(c, RLB_ERR_ARG, "unknown precision");
}

}  // namespace

extern "C" {

rlb_status rlb_create(rlb_ctx** out, int cuda_device) {
  if (!out) return RLB_ERR_ARG;
  *out = nullptr;
  rlb_ctx* c = new (std::nothrow) rlb_ctx();
  if (!c) return RLB_ERR_NOMEM;
  c->device = cuda_device;
  *out = c;
  return RLB_OK;
}

void rlb_destroy(rlb_ctx* ctx) {
  if (!ctx) return;
  drop_graphs(ctx);
  if (ctx->gstream) cudaStreamDestroy(ctx->gstream);
  if (ctx->cstream) cudaStreamDestroy(ctx->cstream);
  if (ctx->mstage) cudaFree(ctx->mstage);
  for (int i = 0; i < 2; ++i) {
    if (ctx->cev_ready[i]) cudaEventDestroy(ctx->cev_ready[i]);
    if (ctx->cev_done[i]) cudaEventDestroy(ctx->cev_done[i]);
  }
  for (cudaEvent_t e : ctx->gev)
    if (e) cudaEventDestroy(e);
  for (auto& p : ctx->ev_pending) { ctx->ev_pool.push_back(p.second.first); ctx->ev_pool.push_back(p.second.second); }
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  delete ctx;
}

const char* rlb_last_error(const rlb_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

rlb_status rlb_init_eos(rlb_ctx* ctx, const rlb_eos_params* e) {
  if (!ctx || !e) return RLB_ERR_ARG;
  if (ctx->bound) return fail(ctx, RLB_ERR_STATE, "EOS must be set before binding buffers");
  rlb::EosParams p;
  p.kind = e->kind;
  p.a = e->a; p.b = e->b; p.Tc = e->Tc; p.w = e->w; p.m0 = e->m0; p.Z = e->Z;
  p.T_min = e->T_min; p.T_max = e->T_max;
  p.points = e->table_points > 0 ? e->table_points : 65536;
  std::string m = rlb::build_eos_table(p, &ctx->tab);
  if (!m.empty()) return fail(ctx, RLB_ERR_ARG, m);
  ctx->eosp = p;
  ctx->eos_ok = true;
  return RLB_OK;
}

rlb_status rlb_workspace_size(const rlb_ctx* ctx, const rlb_grid_params* g, size_t* state_bytes,
                              size_t* scratch_bytes) {
  if (!state_bytes || !scratch_bytes) return RLB_ERR_ARG;
  if (!g) {  // the configured grid or batch
    if (!ctx || !ctx->grid_ok) return RLB_ERR_ARG;
    layout(ctx->gp, ctx_shape(ctx), (size_t)ctx->eosp.points, state_bytes, scratch_bytes, nullptr);
    return RLB_OK;
  }
  if (g->nx < 1 || g->ny < 1 || g->prec < 0 || g->prec > 2) return RLB_ERR_ARG;
  size_t pts = (ctx && ctx->eos_ok) ? (size_t)ctx->eosp.points : 65536;
  layout(*g, grid_shape(*g), pts, state_bytes, scratch_bytes, nullptr);
  return RLB_OK;
}

rlb_status rlb_configure(rlb_ctx* ctx, const rlb_grid_params* g) {
  if (!ctx || !g) return RLB_ERR_ARG;
  if (!ctx->eos_ok) return fail(ctx, RLB_ERR_STATE, "rlb_init_eos must come first");
  if (ctx->bound) return fail(ctx, RLB_ERR_STATE, "grid is fixed once buffers are bound");
  if (g->nx < 1 || g->ny < 1 || !(g->dx > 0) || !(g->dtau > 0) || !(g->tau0 > 0) ||
      !(g->eta_over_s > 0))
    return fail(ctx, RLB_ERR_ARG, "invalid grid parameters");
  if (g->prec < 0 || g->prec > 2) return fail(ctx, RLB_ERR_ARG, "invalid precision");
  if (!supported_shape(g->n_xi, g->n_theta, 2 * g->n_phi_half))
    return fail(ctx, RLB_ERR_ARG, "unsupported lattice shape");
  if (g->family == RLB_RADIAL_LAGUERRE && ctx->eosp.kind != RLB_EOS_CONFORMAL)
    return fail(ctx, RLB_ERR_ARG, "the Laguerre radial family needs the conformal EOS");
  if (g->family == RLB_RADIAL_LAGUERRE && !(g->T0 > 0))
    return fail(ctx, RLB_ERR_ARG, "T0 must be positive");
  if ((size_t)g->nx * g->ny > 0x7fffffffu || g->nx > 65535)
    return fail(ctx, RLB_ERR_ARG, "grid too large (nx <= 65535, nx * ny < 2^31)");
  std::string m = rlb::build_lattice(g->family, g->n_xi, g->n_theta, g->n_phi_half, g->z0, &ctx->lat);
  if (!m.empty()) return fail(ctx, RLB_ERR_ARG, m);
  {
    // streaming stability: the second-order upwind difference with the Heun
    // stages keeps every Fourier mode bounded while the Courant numbers of the
    // two axes, (dtau/dx) |V_x| + (dtau/dx) |V_y|, stay at or below 1/2 for every
    // node (an axis of one site has no streaming)
    const rlb::Lattice& L = ctx->lat;
    const double ax = g->nx > 1 ? 1.0 : 0.0, ay = g->ny > 1 ? 1.0 : 0.0;
    double vmax = 0.0;
    for (int k = 0; k < L.nxi; ++k)
      for (int j = 0; j < L.nth; ++j)
        for (int l = 0; l < L.nph; ++l)
          vmax = std::max(vmax, L.s[k] / L.c[k] * L.sth[j] * (ax * std::fabs(L.cph[l]) + ay * std::fabs(L.sph[l])));
    const double courant = g->dtau / g->dx * vmax;
    if (courant > 0.5) {
      char buf[160];
      snprintf(buf, sizeof buf, "time step above the streaming stability limit: (dtau/dx) max(|V_x| + |V_y|) = %.3g > 0.5",
               courant);
      return fail(ctx, RLB_ERR_ARG, buf);
    }
  }
  ctx->gp = *g;
  ctx->lines_mp.clear();
  if (g->n_theta % 2 == 0) ctx->lines_mp = make_lines_mp(ctx->lat, g->dx);
  if (ctx->lines_mp.size() > kLinesBytes) return fail(ctx, RLB_ERR_ARG, "line table larger than its scratch region");
  set_events(ctx, {rlbk::EventInfo{0, g->nx, g->ny, 0, g->eta_over_s, 0.0}});
  ctx->nn = (size_t)g->n_xi * g->n_theta * 2 * g->n_phi_half;
  ctx->pop_bytes = pop_size(g->prec);
  size_t sb, xb;
  layout(*g, ctx_shape(ctx), ctx->eosp.points, &sb, &xb, ctx);
  ctx->grid_ok = true;
  ctx->tau = g->tau0;
  return RLB_OK;
}

rlb_status rlb_configure_batch(rlb_ctx* ctx, const rlb_grid_params* base, int n_events,
                               const rlb_event_desc* events) {
  if (!ctx || !base || !events || n_events < 1) return RLB_ERR_ARG;
  std::vector<rlbk::EventInfo> ev((size_t)n_events);
  size_t ns = 0, rows = 0;
  int max_nx = 0;
  for (int e = 0; e < n_events; ++e) {
    const rlb_event_desc& d = events[e];
    if (d.nx < 1 || d.ny < 1 || d.nx > 65535 || d.ny > 32767 || !(d.eta_over_s > 0))
      return fail(ctx, RLB_ERR_ARG, "invalid event (nx in [1, 65535], ny in [1, 32767], eta/s > 0)");
    ev[e] = rlbk::EventInfo{(int)ns, d.nx, d.ny, 0, d.eta_over_s, 0.0};
    ns += (size_t)d.nx * d.ny;
    rows += (size_t)d.ny;
    max_nx = std::max(max_nx, d.nx);
    if (ns > 0x7fffffffu) return fail(ctx, RLB_ERR_ARG, "batch too large (fewer than 2^31 sites)");
  }
  rlb_grid_params g = *base;  // shared lattice, precision, dx, tau0, dtau, metric
  g.nx = max_nx;
  g.ny = (int)rows;
  g.eta_over_s = events[0].eta_over_s;
  rlb_status s = rlb_configure(ctx, &g);  // validates the shared parameters, builds the lattice
  if (s) return s;
  set_events(ctx, ev);
  size_t sb, xb;
  layout(ctx->gp, ctx_shape(ctx), ctx->eosp.points, &sb, &xb, ctx);
  return RLB_OK;
}

rlb_status rlb_bind_buffers(rlb_ctx* ctx, void* state, void* scratch, void* stream) {
  if (!ctx) return RLB_ERR_ARG;
  if (!ctx->grid_ok) return fail(ctx, RLB_ERR_STATE, "rlb_configure must come first");
  if (!state || !scratch || ((uintptr_t)state & 255) || ((uintptr_t)scratch & 255))
    return fail(ctx, RLB_ERR_ARG, "buffers must be non-null and 256-byte aligned");
  rlb_status s = set_device(ctx);
  if (s) return s;
  ctx->state = static_cast<char*>(state);
  ctx->scratch = static_cast<char*>(scratch);
  drop_graphs(ctx);  // captured with the previous buffers
  ctx->scf_fresh = false;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  RLB_CUDA(cudaMemcpyAsync(ctx->scratch + ctx->tab_off, ctx->tab.data.data(),
                           ctx->tab.data.size() * sizeof(double), cudaMemcpyHostToDevice, st),
           "EOS table upload");
  {
    const std::vector<float> tf = table_hi_lo(ctx->tab);
    RLB_CUDA(cudaMemcpyAsync(ctx->scratch + ctx->tabf_off, tf.data(), tf.size() * sizeof(float),
                             cudaMemcpyHostToDevice, st),
             "FP32 EOS table upload");
    RLB_CUDA(cudaStreamSynchronize(st), "bind synchronise");
  }
  RLB_CUDA(cudaMemsetAsync(ctx->scratch + ctx->err_off, 0, 256, st), "error word reset");
  s = measure_ex2_bias(ctx, ctx->scratch, ctx->eps_off, st);  // eps0 space: free until rlb_init_grid
  if (s) return s;
  s = upload_tables(ctx, ctx->scratch, st);
  if (s) return s;
  s = set_clock(ctx, ctx->scratch, ctx->tau, st);
  if (s) return s;
  // the table copies read pageable host memory owned by ctx: wait for them
  RLB_CUDA(cudaStreamSynchronize(st), "bind synchronise");
  ctx->bound = true;
  return RLB_OK;
}

rlb_status rlb_init_grid(rlb_ctx* ctx, const double* eps0, int eps0_on_device, void* stream) {
  if (!ctx || !eps0) return RLB_ERR_ARG;
  if (!ctx->bound) return fail(ctx, RLB_ERR_STATE, "rlb_bind_buffers must come first");
  rlb_status s = set_device(ctx);
  if (s) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* dev = reinterpret_cast<double*>(ctx->scratch + ctx->eps_off);
  if (eps0_on_device) {
    RLB_CUDA(cudaMemcpyAsync(dev, eps0, ctx->ns * sizeof(double), cudaMemcpyDeviceToDevice, st),
             "eps0 copy");
  } else {
    for (size_t i = 0; i < ctx->ns; ++i)
      if (!(eps0[i] > 0.0) || !std::isfinite(eps0[i]))
        return fail(ctx, RLB_ERR_ARG, "eps0 must be positive and finite");
    RLB_CUDA(cudaMemcpyAsync(dev, eps0, ctx->ns * sizeof(double), cudaMemcpyHostToDevice, st),
             "eps0 upload");
    RLB_CUDA(cudaStreamSynchronize(st), "eps0 upload synchronise");
  }
  s = dispatch(ctx, OP_INIT, 0, dev, st);
  if (s) return s;
  ctx->tau = ctx->gp.tau0;
  s = set_clock(ctx, ctx->scratch, ctx->tau, st);
  if (s) return s;
  ctx->inited = true;
  return RLB_OK;
}

rlb_status rlb_init_batch(rlb_ctx* ctx, const double* eps0_concat, int eps0_on_device, void* stream) {
  return rlb_init_grid(ctx, eps0_concat, eps0_on_device, stream);
}

rlb_status rlb_step(rlb_ctx* ctx, int nsteps, void* stream) {
  if (!ctx || nsteps < 0) return RLB_ERR_ARG;
  if (!ctx->inited) return fail(ctx, RLB_ERR_STATE, "rlb_init_grid must come first");
  rlb_status s = set_device(ctx);
  if (s) return s;
  return dispatch(ctx, OP_STEP, nsteps, nullptr, static_cast<cudaStream_t>(stream));
}

rlb_status rlb_step_static_scratch(rlb_ctx* ctx, void* state, int nsteps, void* stream) {
  if (!ctx || !state || nsteps < 0) return RLB_ERR_ARG;
  if (!ctx->grid_ok) return fail(ctx, RLB_ERR_STATE, "rlb_configure must come first");
  ctx->scf_fresh = false;  // another state: the context's site scalars no longer describe it
  if ((uintptr_t)state & 255) return fail(ctx, RLB_ERR_ARG, "state must be 256-byte aligned");
  size_t sb, xb;
  layout(ctx->gp, ctx_shape(ctx), (size_t)ctx->eosp.points, &sb, &xb, nullptr);
  if (xb > kStaticScratchBytes) {
    char buf[200];
    snprintf(buf, sizeof buf,
             "grid needs %zu bytes of scratch; the static scratch holds %zu (use rlb_step with bound buffers)",
             xb, kStaticScratchBytes);
    return fail(ctx, RLB_ERR_ARG, buf);
  }
  rlb_status s = set_device(ctx);
  if (s) return s;
  char* scr = nullptr;
  s = static_scratch(ctx, &scr);
  if (s) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* stp = static_cast<char*>(state);
  const int a = ctx->gp.n_xi, b = ctx->gp.n_theta, d = 2 * ctx->gp.n_phi_half;
  if (a == 8 && b == 8 && d == 12) return step_static_prec<8, 8, 12>(ctx, stp, scr, nsteps, st);
  if (a == 16 && b == 8 && d == 16) return step_static_prec<16, 8, 16>(ctx, stp, scr, nsteps, st);
  if (a == 5 && b == 5 && d == 2) return step_static_prec<5, 5, 2>(ctx, stp, scr, nsteps, st);
  if (a == 6 && b == 4 && d == 6) return step_static_prec<6, 4, 6>(ctx, stp, scr, nsteps, st);
  if (a == 8 && b == 8 && d == 2) return step_static_prec<8, 8, 2>(ctx, stp, scr, nsteps, st);
  return fail(ctx, RLB_ERR_ARG, "unsupported lattice shape");
}

rlb_status rlb_alu_peaks(int cuda_device, double* tflops) {
  if (!tflops) return RLB_ERR_ARG;
  rlb_ctx tmp;  // for the error macro only
  rlb_ctx* ctx = &tmp;
  RLB_CUDA(cudaSetDevice(cuda_device), "cudaSetDevice");
  int sms = 0;
  RLB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, cuda_device), "SM count");
  cudaStream_t st;
  RLB_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "peak stream");
  cudaEvent_t e0, e1;
  RLB_CUDA(cudaEventCreate(&e0), "peak event");
  RLB_CUDA(cudaEventCreate(&e1), "peak event");
  const unsigned blocks = 8u * (unsigned)sms, threads = 256;
  const double lanes = (double)blocks * threads * rlbk::kPeakChains * rlbk::kPeakUnroll;
  // iterations sized for about 20 ms per timed launch
  const int it32 = 20000, it32x2 = 10000, it64 = 400;
  double ms[3] = {0, 0, 0};
  for (int k = 0; k < 3; ++k) {
    for (int rep = 0; rep < 2; ++rep) {  // the first launch warms up
      RLB_CUDA(cudaEventRecord(e0, st), "peak event");
      if (k == 0) rlbk::peak_ffma_kernel<<<blocks, threads, 0, st>>>(0.999999f, 1e-7f, it32);
      else if (k == 1) rlbk::peak_ffma2_kernel<<<blocks, threads, 0, st>>>(0.999999f, 1e-7f, it32x2);
      else rlbk::peak_dfma_kernel<<<blocks, threads, 0, st>>>(0.999999999, 1e-10, it64);
      RLB_CUDA(cudaGetLastError(), "peak kernel launch");
      RLB_CUDA(cudaEventRecord(e1, st), "peak event");
      RLB_CUDA(cudaEventSynchronize(e1), "peak synchronise");
      float t = 0.f;
      RLB_CUDA(cudaEventElapsedTime(&t, e0, e1), "peak time");
      ms[k] = t;
    }
  }
  tflops[0] = 2.0 * lanes * it32 / (ms[0] * 1e-3) / 1e12;
  tflops[1] = 4.0 * lanes * it32x2 / (ms[1] * 1e-3) / 1e12;
  tflops[2] = 2.0 * lanes * it64 / (ms[2] * 1e-3) / 1e12;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  return RLB_OK;
}

rlb_status rlb_wait_selftest(int cuda_device, int deliver, double limit_ms, int* expired, float* value) {
  if (!expired || !(limit_ms > 0 && limit_ms <= 2000)) return RLB_ERR_ARG;
  rlb_ctx tmp;  // for the error macro only
  rlb_ctx* ctx = &tmp;
  RLB_CUDA(cudaSetDevice(cuda_device), "cudaSetDevice");
  void* mem = nullptr;
  RLB_CUDA(cudaMalloc(&mem, 256), "self-test buffer");
  float* src = static_cast<float*>(mem);
  int* out = reinterpret_cast<int*>(static_cast<char*>(mem) + 128);
  const float v[4] = {1.25f, 0.f, 0.f, 0.f};
  const int init[2] = {-1, 0};
  cudaError_t e = cudaMemcpy(src, v, sizeof v, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(out, init, sizeof init, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    rlbk::wait_selftest_kernel<<<1, 64>>>(src, deliver, (unsigned long long)(limit_ms * 1e6), out);
    e = cudaGetLastError();
  }
  int res[2] = {-1, 0};
  if (e == cudaSuccess) e = cudaMemcpy(res, out, sizeof res, cudaMemcpyDeviceToHost);
  cudaFree(mem);
  RLB_CUDA(e, "wait self-test");
  *expired = res[0];
  if (value) std::memcpy(value, &res[1], sizeof(float));
  return RLB_OK;
}

rlb_status rlb_get_tau(const rlb_ctx* ctx, double* tau) {
  if (!ctx || !tau) return RLB_ERR_ARG;
  *tau = ctx->tau;
  return RLB_OK;
}

rlb_status rlb_check(rlb_ctx* ctx, void* stream) {
  if (!ctx) return RLB_ERR_ARG;
  if (!ctx->bound) return fail(ctx, RLB_ERR_STATE, "no buffers bound");
  rlb_status s = set_device(ctx);
  if (s) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int word = 0;
  RLB_CUDA(cudaMemcpyAsync(&word, ctx->scratch + ctx->err_off, sizeof(int), cudaMemcpyDeviceToHost, st),
           "error word read");
  RLB_CUDA(cudaStreamSynchronize(st), "synchronise");
  if (word) {
    char buf[192];
    snprintf(buf, sizeof buf,
             "device error word 0x%x (1: Landau, 2: EOS inversion, 4: non-finite, 8: index check, 16: bounded "
             "wait expired)",
             word);
    return fail(ctx, (word & rlbk::ERR_TIMEOUT) ? RLB_ERR_TIMEOUT : RLB_ERR_NUMERIC, buf);
  }
  return RLB_OK;
}

rlb_status rlb_moments(rlb_ctx* ctx, double* out, int out_on_device, void* stream) {
  if (!ctx || !out) return RLB_ERR_ARG;
  if (!ctx->inited) return fail(ctx, RLB_ERR_STATE, "rlb_init_grid must come first");
  rlb_status s = set_device(ctx);
  if (s) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const double* mom = reinterpret_cast<const double*>(ctx->scratch + ctx->mom_off);
  const double* lnM = reinterpret_cast<const double*>(ctx->state + ctx->lnM_off);
  if (out_on_device) {
    s = match(ctx, mom, lnM, out, st);
    ctx->scf_fresh = s == RLB_OK;  // the next step's first matching is this one
    return s;
  }
  // host output: stage through the predictor buffer (free between steps)
  double* dev = reinterpret_cast<double*>(ctx->scratch + ctx->fs_off);
  if (ctx->ns * 8 * sizeof(double) > ctx->ns * ctx->nn * ctx->pop_bytes)
    return fail(ctx, RLB_ERR_ARG, "lattice too small to stage host moments");
  s = match(ctx, mom, lnM, dev, st);
  if (s) return s;
  ctx->scf_fresh = true;
  RLB_CUDA(cudaMemcpyAsync(out, dev, ctx->ns * 8 * sizeof(double), cudaMemcpyDeviceToHost, st),
           "moments download");
  return rlb_check(ctx, stream);
}

rlb_status rlb_moments_async(rlb_ctx* ctx, double* host_out, void* stream) {
  if (!ctx || !host_out) return RLB_ERR_ARG;
  if (!ctx->inited) return fail(ctx, RLB_ERR_STATE, "rlb_init_grid must come first");
  cudaPointerAttributes pa;
  if (cudaPointerGetAttributes(&pa, host_out) != cudaSuccess || pa.type != cudaMemoryTypeHost) {
    cudaGetLastError();
    return fail(ctx, RLB_ERR_ARG, "rlb_moments_async writes page-locked host memory");
  }
  rlb_status s = set_device(ctx);
  if (s) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t slot_b = align256(ctx->ns * 8 * sizeof(double));
  if (!ctx->cstream) {
    // all or nothing: the context keeps the slots, stream and events only
    // once every one of them exists
    char* slots = nullptr;
    cudaStream_t cs = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaError_t e = cudaMalloc(&slots, 2 * slot_b);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventRecord(ev[2 + i], cs);
    if (e != cudaSuccess) {
      for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
      if (cs) cudaStreamDestroy(cs);
      if (slots) cudaFree(slots);
      return cuda_fail(ctx, e, "moments staging slots, copy stream and events");
    }
    ctx->mstage = slots;
    ctx->cstream = cs;
    ctx->cev_ready[0] = ev[0]; ctx->cev_ready[1] = ev[1];
    ctx->cev_done[0] = ev[2]; ctx->cev_done[1] = ev[3];
  }
  const int k = ctx->cslot;
  ctx->cslot ^= 1;
  double* dev = reinterpret_cast<double*>(ctx->mstage + (size_t)k * slot_b);
  // the slot's previous copy has left it; the matching of the current state
  // writes the observables there (the next step reuses that matching)
  RLB_CUDA(cudaStreamWaitEvent(st, ctx->cev_done[k], 0), "copy order");
  const double* mom = reinterpret_cast<const double*>(ctx->scratch + ctx->mom_off);
  const double* lnM = reinterpret_cast<const double*>(ctx->state + ctx->lnM_off);
  s = match(ctx, mom, lnM, dev, st);
  if (s) return s;
  ctx->scf_fresh = true;
  RLB_CUDA(cudaEventRecord(ctx->cev_ready[k], st), "copy order");
  RLB_CUDA(cudaStreamWaitEvent(ctx->cstream, ctx->cev_ready[k], 0), "copy order");
  RLB_CUDA(cudaMemcpyAsync(host_out, dev, ctx->ns * 8 * sizeof(double), cudaMemcpyDeviceToHost, ctx->cstream),
           "moments download");
  RLB_CUDA(cudaEventRecord(ctx->cev_done[k], ctx->cstream), "copy order");
  return RLB_OK;
}

rlb_status rlb_moments_wait(rlb_ctx* ctx) {
  if (!ctx) return RLB_ERR_ARG;
  if (!ctx->cstream) return RLB_OK;
  rlb_status s = set_device(ctx);
  if (s) return s;
  RLB_CUDA(cudaStreamSynchronize(ctx->cstream), "copy synchronise");
  return rlb_check(ctx, ctx->cstream);
}

rlb_status rlb_observables(rlb_ctx* ctx, double* eps_p, double* v2_pt, void* stream) {
  if (!ctx || !eps_p || !v2_pt) return RLB_ERR_ARG;
  if (!ctx->inited) return fail(ctx, RLB_ERR_STATE, "rlb_init_grid must come first");
  rlb_status s = set_device(ctx);
  if (s) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* dev = reinterpret_cast<double*>(ctx->scratch + ctx->eps_off);  // free between steps
  s = dispatch(ctx, OP_OBS, 0, dev, st);
  if (s) return s;
  double h[2];
  RLB_CUDA(cudaMemcpyAsync(h, dev, sizeof(h), cudaMemcpyDeviceToHost, st), "observables download");
  s = rlb_check(ctx, stream);  // synchronises the stream
  if (s) return s;
  *eps_p = h[0];
  *v2_pt = h[1];
  return RLB_OK;
}

// ---------------------------------------------------------------------------
// checkpoint blob: header, f, ln M, Newton starting temperatures, stored moments
// ---------------------------------------------------------------------------
namespace {

// Blob layout (version 2): the header in the first 256 bytes, then f, ln M,
// T and the moments, each starting at a multiple of 256 bytes (the kernels can
// read a device blob in place).
constexpr uint64_t kBlobHead = 256;
struct BlobHeader {
  char magic[8];  // "RLBSTAT1"
  uint32_t version;
  int32_t prec, nx, ny, n_xi, n_theta, n_phi_half, family, metric;
  double dx, z0, T0;
  double tau;
  uint64_t f_bytes, lnM_bytes, T_bytes, mom_bytes;
};

void blob_parts(const rlb_ctx* c, BlobHeader* h) {
  std::memset(h, 0, sizeof(*h));
  std::memcpy(h->magic, "RLBSTAT1", 8);
  h->version = 2;
  h->prec = c->gp.prec; h->nx = c->gp.nx; h->ny = c->gp.ny;
  h->n_xi = c->gp.n_xi; h->n_theta = c->gp.n_theta; h->n_phi_half = c->gp.n_phi_half;
  h->family = c->gp.family; h->metric = c->gp.metric;
  h->dx = c->gp.dx; h->z0 = c->gp.z0; h->T0 = c->gp.T0;
  h->tau = c->tau;
  h->f_bytes = (uint64_t)c->ns * c->nn * c->pop_bytes;
  h->lnM_bytes = (uint64_t)c->ns * sizeof(double);
  h->T_bytes = (uint64_t)c->ns * sizeof(double);
  h->mom_bytes = (uint64_t)c->ns * std::max(rlbk::kMom * sizeof(double), rlbk::kMom * rlbk::kMomParts * sizeof(float));
}

static_assert(sizeof(BlobHeader) <= kBlobHead, "blob header");
// byte offsets of f, ln M, T, moments in a blob, and its size
void blob_offsets(const BlobHeader& h, uint64_t (&o)[4], uint64_t* size) {
  const uint64_t n[4] = {h.f_bytes, h.lnM_bytes, h.T_bytes, h.mom_bytes};
  uint64_t off = kBlobHead;
  for (int i = 0; i < 4; ++i) {
    o[i] = off;
    off += align256(n[i]);
  }
  if (size) *size = off;
}
size_t blob_size(const BlobHeader& h) {
  uint64_t o[4], n = 0;
  blob_offsets(h, o, &n);
  return (size_t)n;
}

}  // namespace

rlb_status rlb_state_blob_size(const rlb_ctx* ctx, size_t* bytes) {
  if (!ctx || !bytes || !ctx->grid_ok) return RLB_ERR_ARG;
  BlobHeader h;
  blob_parts(ctx, &h);
  *bytes = blob_size(h);
  return RLB_OK;
}

// The blob header written on the device by the stream (it travels as a kernel
// parameter: nothing on the host has to outlive the call).
__global__ void write_header_kernel(BlobHeader h, BlobHeader* dst) { *dst = h; }

bool is_device_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice;
}

rlb_status rlb_save_state(rlb_ctx* ctx, void* host_buf, size_t bytes, void* stream) {
  if (!ctx || !host_buf) return RLB_ERR_ARG;
  if (!ctx->inited) return fail(ctx, RLB_ERR_STATE, "nothing to save: rlb_init_grid or rlb_load_state first");
  BlobHeader h;
  blob_parts(ctx, &h);
  if (bytes < blob_size(h)) {
    char buf[160];
    snprintf(buf, sizeof buf, "state blob needs %zu bytes, buffer has %zu", blob_size(h), bytes);
    return fail(ctx, RLB_ERR_ARG, buf);
  }
  rlb_status s = set_device(ctx);
  if (s) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* p = static_cast<char*>(host_buf);
  const bool dev = is_device_pointer(host_buf);
  if (dev) {  // everything enqueued on the stream: no host synchronisation
    write_header_kernel<<<1, 1, 0, st>>>(h, reinterpret_cast<BlobHeader*>(p));
    RLB_CUDA(cudaGetLastError(), "state header");
  } else {
    RLB_CUDA(cudaMemcpyAsync(p, &h, sizeof h, cudaMemcpyDefault, st), "state header");
    RLB_CUDA(cudaStreamSynchronize(st), "state header synchronise");  // h lives on this stack
  }
  uint64_t o[4];
  blob_offsets(h, o, nullptr);
  const struct { const char* src; uint64_t n; } parts[4] = {
      {ctx->state + ctx->f_off, h.f_bytes}, {ctx->state + ctx->lnM_off, h.lnM_bytes},
      {ctx->scratch + ctx->T_off, h.T_bytes}, {ctx->scratch + ctx->mom_off, h.mom_bytes}};
  for (int i = 0; i < 4; ++i)
    RLB_CUDA(cudaMemcpyAsync(p + o[i], parts[i].src, parts[i].n, cudaMemcpyDefault, st), "state copy");
  if (!dev) RLB_CUDA(cudaStreamSynchronize(st), "state download synchronise");
  return RLB_OK;
}

rlb_status rlb_load_state_async(rlb_ctx* ctx, const void* dev_buf, size_t bytes, double tau, void* stream) {
  if (!ctx || !dev_buf) return RLB_ERR_ARG;
  if (!ctx->bound) return fail(ctx, RLB_ERR_STATE, "rlb_bind_buffers must come first");
  BlobHeader want;
  blob_parts(ctx, &want);
  if (bytes < blob_size(want)) return fail(ctx, RLB_ERR_ARG, "state blob is truncated");
  if (!is_device_pointer(dev_buf)) return fail(ctx, RLB_ERR_ARG, "rlb_load_state_async takes device blobs");
  rlb_status s = set_device(ctx);
  if (s) return s;
  ctx->scf_fresh = false;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const char* p = static_cast<const char*>(dev_buf);
  uint64_t o[4];
  blob_offsets(want, o, nullptr);
  const struct { char* dst; uint64_t n; } parts[4] = {
      {ctx->state + ctx->f_off, want.f_bytes}, {ctx->state + ctx->lnM_off, want.lnM_bytes},
      {ctx->scratch + ctx->T_off, want.T_bytes}, {ctx->scratch + ctx->mom_off, want.mom_bytes}};
  for (int i = 0; i < 4; ++i)
    RLB_CUDA(cudaMemcpyAsync(parts[i].dst, p + o[i], parts[i].n, cudaMemcpyDeviceToDevice, st), "state copy");
  ctx->tau = tau;
  s = set_clock(ctx, ctx->scratch, ctx->tau, st);
  if (s) return s;
  ctx->inited = true;
  return RLB_OK;
}

rlb_status rlb_load_state(rlb_ctx* ctx, const void* host_buf, size_t bytes, void* stream) {
  if (!ctx || !host_buf) return RLB_ERR_ARG;
  if (!ctx->bound) return fail(ctx, RLB_ERR_STATE, "rlb_bind_buffers must come first");
  ctx->scf_fresh = false;
  BlobHeader want, got;
  blob_parts(ctx, &want);
  if (bytes < sizeof got) return fail(ctx, RLB_ERR_ARG, "state blob shorter than its header");
  RLB_CUDA(cudaMemcpy(&got, host_buf, sizeof got, cudaMemcpyDefault), "state header");
  if (std::memcmp(got.magic, want.magic, 8) != 0 || got.version != want.version)
    return fail(ctx, RLB_ERR_ARG, "not a state blob of this library version");
  if (got.prec != want.prec || got.nx != want.nx || got.ny != want.ny || got.n_xi != want.n_xi ||
      got.n_theta != want.n_theta || got.n_phi_half != want.n_phi_half || got.family != want.family ||
      got.metric != want.metric || got.dx != want.dx || got.z0 != want.z0 || got.T0 != want.T0 ||
      got.f_bytes != want.f_bytes || got.mom_bytes != want.mom_bytes)
    return fail(ctx, RLB_ERR_ARG, "state blob was saved with another grid, lattice or precision");
  if (bytes < blob_size(got)) return fail(ctx, RLB_ERR_ARG, "state blob is truncated");
  rlb_status s = set_device(ctx);
  if (s) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const char* p = static_cast<const char*>(host_buf);
  uint64_t o[4];
  blob_offsets(got, o, nullptr);
  const struct { char* dst; uint64_t n; } parts[4] = {
      {ctx->state + ctx->f_off, got.f_bytes}, {ctx->state + ctx->lnM_off, got.lnM_bytes},
      {ctx->scratch + ctx->T_off, got.T_bytes}, {ctx->scratch + ctx->mom_off, got.mom_bytes}};
  for (int i = 0; i < 4; ++i)
    RLB_CUDA(cudaMemcpyAsync(parts[i].dst, p + o[i], parts[i].n, cudaMemcpyDefault, st), "state copy");
  ctx->tau = got.tau;
  s = set_clock(ctx, ctx->scratch, ctx->tau, st);
  if (s) return s;
  RLB_CUDA(cudaStreamSynchronize(st), "state upload synchronise");
  ctx->inited = true;
  return RLB_OK;
}

rlb_status rlb_autotune(rlb_ctx* ctx, void* stream, int* chosen, double* variant_ms, int* n_variants) {
  if (!ctx || !chosen) return RLB_ERR_ARG;
  if (!ctx->inited) return fail(ctx, RLB_ERR_STATE, "rlb_init_grid or rlb_load_state must come first");
  rlb_status s = set_device(ctx);
  if (s) return s;
  double t[RLB_MAX_STAGE_VARIANTS + 1] = {};
  s = dispatch(ctx, OP_TUNE, 0, t, static_cast<cudaStream_t>(stream));
  if (s) return s;
  *chosen = ctx->stage_variant;
  const int nv = (int)t[RLB_MAX_STAGE_VARIANTS];
  if (n_variants) *n_variants = nv;
  if (variant_ms)
    for (int v = 0; v < nv; ++v) variant_ms[v] = t[v];
  return RLB_OK;
}

rlb_status rlb_adjoint_set_arithmetic(rlb_ctx* ctx, int prec) {
  if (!ctx) return RLB_ERR_ARG;
  if (prec != RLB_F64 && prec != RLB_F32) return fail(ctx, RLB_ERR_ARG, "adjoint arithmetic: RLB_F64 or RLB_F32");
  if (prec != ctx->adj_prec) ctx->adj = nullptr;  // the workspace layout changes: bind again
  ctx->adj_prec = prec;
  return RLB_OK;
}

rlb_status rlb_adjoint_workspace_size(rlb_ctx* ctx, size_t* bytes) {
  if (!ctx || !bytes || !ctx->grid_ok) return RLB_ERR_ARG;
  *bytes = adj_layout(ctx);
  return RLB_OK;
}

rlb_status rlb_adjoint_bind(rlb_ctx* ctx, void* workspace) {
  if (!ctx || !workspace || ((uintptr_t)workspace & 255)) return RLB_ERR_ARG;
  if (!ctx->grid_ok) return fail(ctx, RLB_ERR_STATE, "rlb_configure must come first");
  adj_layout(ctx);
  ctx->adj = static_cast<char*>(workspace);
  rlb_status s = set_device(ctx);
  if (s) return s;
  // the FP64 matchings of the adjoint start their Newton solves from zeros here:
  // results do not depend on what the memory held
  RLB_CUDA(cudaMemset(ctx->adj + ctx->a_T, 0, ctx->ns * sizeof(double)), "adjoint workspace reset");
  return RLB_OK;
}

rlb_status rlb_adjoint_seed(rlb_ctx* ctx, const double* fbar, const double* lbar, void* stream) {
  if (!ctx || !fbar || !lbar) return RLB_ERR_ARG;
  if (!ctx->inited || !ctx->adj) return fail(ctx, RLB_ERR_STATE, "state and adjoint workspace needed");
  rlb_status s = set_device(ctx);
  if (s) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t npop = ctx->ns * ctx->nn;
  if (ctx->adj_prec == RLB_F64) {
    RLB_CUDA(cudaMemcpyAsync(ctx->adj + ctx->a_f, fbar, npop * sizeof(double), cudaMemcpyDefault, st),
             "adjoint seed upload");
  } else {
    // FP64 staging in the two per-stage FP32 arrays that follow a_f (>= npop doubles)
    double* stage = reinterpret_cast<double*>(ctx->adj + ctx->a_fb);
    RLB_CUDA(cudaMemcpyAsync(stage, fbar, npop * sizeof(double), cudaMemcpyDefault, st), "adjoint seed upload");
    rlbk::convert_kernel<float><<<(unsigned)std::min<size_t>((npop + 255) / 256, 152 * 16), 256, 0, st>>>(
        reinterpret_cast<float*>(ctx->adj + ctx->a_f), stage, npop);
    RLB_CUDA(cudaGetLastError(), "adjoint seed conversion");
  }
  RLB_CUDA(cudaMemcpyAsync(ctx->adj + ctx->a_l, lbar, ctx->ns * sizeof(double), cudaMemcpyDefault, st),
           "adjoint seed upload");
  RLB_CUDA(cudaMemsetAsync(ctx->adj + ctx->a_eta, 0, sizeof(double), st), "adjoint eta reset");
  RLB_CUDA(cudaMemsetAsync(ctx->adj + ctx->a_ebar, 0, ctx->ns * sizeof(double), st), "adjoint eta reset");
  RLB_CUDA(cudaStreamSynchronize(st), "adjoint seed synchronise");
  return RLB_OK;
}

rlb_status rlb_adjoint_seed_v2(rlb_ctx* ctx, double* v2, void* stream) {
  if (!ctx || !v2) return RLB_ERR_ARG;
  if (!ctx->inited || !ctx->adj) return fail(ctx, RLB_ERR_STATE, "state and adjoint workspace needed");
  rlb_status s = set_device(ctx);
  if (s) return s;
  s = dispatch(ctx, OP_ADJ_SEED, 0, v2, static_cast<cudaStream_t>(stream));
  if (s) return s;
  return rlb_check(ctx, stream);
}

rlb_status rlb_adjoint_step(rlb_ctx* ctx, void* stream) {
  if (!ctx) return RLB_ERR_ARG;
  if (!ctx->inited || !ctx->adj) return fail(ctx, RLB_ERR_STATE, "state and adjoint workspace needed");
  rlb_status s = set_device(ctx);
  if (s) return s;
  return dispatch(ctx, OP_ADJ_STEP, 0, nullptr, static_cast<cudaStream_t>(stream));
}

rlb_status rlb_adjoint_step_from(rlb_ctx* ctx, const void* state_blob, size_t bytes, double tau, void* stream) {
  if (!ctx || !state_blob) return RLB_ERR_ARG;
  if (!ctx->inited || !ctx->adj) return fail(ctx, RLB_ERR_STATE, "state and adjoint workspace needed");
  BlobHeader h;
  blob_parts(ctx, &h);
  uint64_t o[4];
  blob_offsets(h, o, nullptr);
  if (bytes < blob_size(h)) return fail(ctx, RLB_ERR_ARG, "state blob is truncated");
  if (!is_device_pointer(state_blob)) return fail(ctx, RLB_ERR_ARG, "rlb_adjoint_step_from takes device blobs");
  rlb_status s = set_device(ctx);
  if (s) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const char* b = static_cast<const char*>(state_blob);
  // the blob's Newton starts and time; the context's own tau comes back after
  RLB_CUDA(cudaMemcpyAsync(ctx->scratch + ctx->T_off, b + o[2], h.T_bytes, cudaMemcpyDeviceToDevice, st),
           "adjoint Newton start copy");
  const double keep = ctx->tau;
  ctx->tau = tau;
  s = set_clock(ctx, ctx->scratch, tau, st);
  if (!s) {
    struct {
      const char* blob;
      uint64_t o[4];
    } call{b, {o[0], o[1], o[2], o[3]}};
    s = dispatch(ctx, OP_ADJ_STEP, 0, reinterpret_cast<double*>(&call), st);
  }
  ctx->tau = keep;
  rlb_status s2 = set_clock(ctx, ctx->scratch, keep, st);
  return s ? s : s2;
}

rlb_status rlb_adjoint_ic(rlb_ctx* ctx, const double* eps0, const double* basis, int n_basis, double* grad,
                          void* stream) {
  if (!ctx || !eps0 || !grad || n_basis < 0 || (n_basis > 0 && !basis)) return RLB_ERR_ARG;
  if (!ctx->adj) return fail(ctx, RLB_ERR_STATE, "adjoint workspace needed");
  if ((size_t)n_basis > ctx->ns) return fail(ctx, RLB_ERR_ARG, "at most one basis row per site");
  if (ctx->gp.family != RLB_RADIAL_PAPER) return fail(ctx, RLB_ERR_ARG, "initial-condition adjoint needs the dynamical mass");
  rlb_status s = set_device(ctx);
  if (s) return s;
  AdjIcCall a{eps0, basis, n_basis, grad};
  s = dispatch(ctx, OP_ADJ_IC, 0, reinterpret_cast<double*>(&a), static_cast<cudaStream_t>(stream));
  if (s) return s;
  return rlb_check(ctx, stream);
}

rlb_status rlb_set_stage_variant(rlb_ctx* ctx, int variant, int* n_variants) {
  if (!ctx) return RLB_ERR_ARG;
  if (!ctx->grid_ok) return fail(ctx, RLB_ERR_STATE, "rlb_configure must come first");
  double nv = 0.0;
  rlb_status s = dispatch(ctx, OP_NVAR, 0, &nv, nullptr);
  if (s) return s;
  if (n_variants) *n_variants = (int)nv;
  if (variant < 0) return RLB_OK;  // query only
  if (variant >= (int)nv) return fail(ctx, RLB_ERR_ARG, "no such stage-kernel variant");
  ctx->stage_variant = variant;
  drop_graphs(ctx);  // the captured step used the previous choice
  return RLB_OK;
}

rlb_status rlb_set_graphs(rlb_ctx* ctx, int enable) {
  if (!ctx) return RLB_ERR_ARG;
  ctx->graphs = enable != 0;
  return RLB_OK;
}

rlb_status rlb_set_timing(rlb_ctx* ctx, int enable) {
  if (!ctx) return RLB_ERR_ARG;
  ctx->timing = enable != 0;
  ctx->t_ms[0] = ctx->t_ms[1] = ctx->t_ms[2] = 0.0;
  ctx->t_n[0] = ctx->t_n[1] = ctx->t_n[2] = 0;
  return RLB_OK;
}

rlb_status rlb_get_timing(rlb_ctx* ctx, double* stage_ms, long* stage_launches, double* match_ms,
                          long* match_launches) {
  if (!ctx || !stage_ms || !stage_launches || !match_ms || !match_launches) return RLB_ERR_ARG;
  rlb_status s = set_device(ctx);
  if (s) return s;
  for (auto& p : ctx->ev_pending) {
    RLB_CUDA(cudaEventSynchronize(p.second.second), "timing event");
    float ms = 0.0f;
    RLB_CUDA(cudaEventElapsedTime(&ms, p.second.first, p.second.second), "timing elapsed");
    ctx->t_ms[p.first] += ms;
    ctx->t_n[p.first] += 1;
    ctx->ev_pool.push_back(p.second.first);
    ctx->ev_pool.push_back(p.second.second);
  }
  ctx->ev_pending.clear();
  *stage_ms = ctx->t_ms[K_STAGE];
  *stage_launches = ctx->t_n[K_STAGE];
  *match_ms = ctx->t_ms[K_MATCH];
  *match_launches = ctx->t_n[K_MATCH];
  return RLB_OK;
}

rlb_status rlb_state_offsets(const rlb_ctx* ctx, size_t* f_offset, size_t* lnM_offset,
                             size_t* pop_bytes) {
  if (!ctx || !f_offset || !lnM_offset || !pop_bytes) return RLB_ERR_ARG;
  if (!ctx->grid_ok) return RLB_ERR_STATE;
  *f_offset = ctx->f_off;
  *lnM_offset = ctx->lnM_off;
  *pop_bytes = ctx->pop_bytes;
  return RLB_OK;
}

rlb_status rlb_lattice(const rlb_ctx* ctx, double* c, double* s, double* wxi, double* mu,
                       double* wth, double* cph, double* sph) {
  if (!ctx) return RLB_ERR_ARG;
  if (!ctx->grid_ok) return RLB_ERR_STATE;
  const rlb::Lattice& L = ctx->lat;
  for (int k = 0; k < L.nxi; ++k) { c[k] = L.c[k]; s[k] = L.s[k]; wxi[k] = L.wxi[k]; }
  for (int j = 0; j < L.nth; ++j) { mu[j] = L.mu[j]; wth[j] = L.wth[j]; }
  for (int l = 0; l < L.nph; ++l) { cph[l] = L.cph[l]; sph[l] = L.sph[l]; }
  return RLB_OK;
}

rlb_status rlb_operators(const rlb_ctx* ctx, double* Dr, double* Dth) {
  if (!ctx || !Dr || !Dth) return RLB_ERR_ARG;
  if (!ctx->grid_ok) return RLB_ERR_STATE;
  const rlb::Lattice& L = ctx->lat;
  std::memcpy(Dr, L.Dr.data(), L.Dr.size() * sizeof(double));
  std::memcpy(Dth, L.Dth.data(), L.Dth.size() * sizeof(double));
  return RLB_OK;
}

}  // extern "C"
