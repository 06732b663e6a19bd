// rlb_host.cpp -- host construction of the momentum lattice (Sec. 4.3), the
// nodal momentum-derivative operators (Sec. 4.4) and the EOS table (Sec. 3.1)
// consumed by the GB300 kernels.
//
// Methods (chosen for accuracy at init time; none of this is on the hot path):
//   * Gauss rules by Golub-Welsch: the Jacobi matrix of the three-term
//     recurrence is diagonalised with cyclic Jacobi rotations in long double;
//     nodes are its eigenvalues, weights beta_0 times the squared first
//     eigenvector components (evaluated through the orthonormal recurrence).
//   * The recurrence of the paper's radial family (polynomials in cosh xi
//     orthogonal for e^{-z0 cosh xi} sinh^2 xi dxi) comes from a discretised
//     Stieltjes procedure in the variable u with cosh xi = 1 + u^2, where the
//     weight becomes 2 u^2 sqrt(u^2 + 2) e^{-z0 (1 + u^2)} du.
//   * Nodal operators use the Christoffel-Darboux identity
//       sum_{l<N} p_l(x_a) p_l(x_b)/||p_l||^2 = delta_ab / w_a,
//       sum_{l<N} p_l(x_a) p_l'(x_b)/||p_l||^2 = l_a'(x_b) / w_a,
//     (l_a the Lagrange basis of the nodes), which turns the Galerkin sums
//     s_1^{ml}, s_2^{ml} of Sec. 4.4 into closed nodal forms built from the
//     barycentric differentiation matrix.
//   * Modified Bessel functions K_0, K_1 from \int_0^inf e^{-x cosh t} cosh(nu t) dt
//     on 20-point Gauss-Legendre panels, K_2, K_3 by upward recurrence.
//   * EOS fields tabulated on a uniform grid in ln T for 6-point Lagrange
//     interpolation on the device.
#include "rlb_host.hpp"

#include <algorithm>
#include <cmath>
#include <thread>

namespace rlb {
namespace {

using ld = long double;

// Symmetric eigenproblem by cyclic Jacobi rotations.  A is n x n row-major and
// is destroyed; eigenvalues in ev, eigenvectors in the columns of V.
void jacobi_eigen(int n, std::vector<ld>& A, std::vector<ld>& ev, std::vector<ld>& V) {
  V.assign(n * n, 0.0L);
  for (int i = 0; i < n; ++i) V[i * n + i] = 1.0L;
  for (int sweep = 0; sweep < 100; ++sweep) {
    ld off = 0.0L, diag = 0.0L;
    for (int p = 0; p < n; ++p)
      for (int q = 0; q < n; ++q) {
        if (p == q) diag += A[p * n + p] * A[p * n + p];
        else off += A[p * n + q] * A[p * n + q];
      }
    if (off <= 1e-40L * diag) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        ld apq = A[p * n + q];
        if (apq == 0.0L) continue;
        ld theta = (A[q * n + q] - A[p * n + p]) / (2.0L * apq);
        ld t = (theta >= 0 ? 1.0L : -1.0L) / (fabsl(theta) + sqrtl(theta * theta + 1.0L));
        ld c = 1.0L / sqrtl(t * t + 1.0L), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          ld akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          ld apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          ld vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  ev.resize(n);
  for (int i = 0; i < n; ++i) ev[i] = A[i * n + i];
}

// Golub-Welsch: Gauss rule from monic recurrence coefficients alpha_k, beta_k
// (beta_0 = total mass of the weight).  Nodes ascending.
void golub_welsch(int n, const std::vector<ld>& al, const std::vector<ld>& be, std::vector<ld>& x,
                  std::vector<ld>& w) {
  std::vector<ld> J(n * n, 0.0L), ev, V;
  for (int k = 0; k < n; ++k) {
    J[k * n + k] = al[k];
    if (k + 1 < n) J[k * n + k + 1] = J[(k + 1) * n + k] = sqrtl(be[k + 1]);
  }
  jacobi_eigen(n, J, ev, V);
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](int a, int b) { return ev[a] < ev[b]; });
  x.resize(n);
  w.resize(n);
  for (int i = 0; i < n; ++i) {
    x[i] = ev[idx[i]];
    // The weight is beta_0 (first eigenvector component)^2; evaluating that
    // component through the orthonormal recurrence at the node keeps full
    // relative accuracy for the tiny weights of the outermost nodes:
    // 1/w = sum_{l<n} q_l(x)^2 with q_0 = 1/sqrt(beta_0),
    // sqrt(beta_{l+1}) q_{l+1} = (x - alpha_l) q_l - sqrt(beta_l) q_{l-1}.
    ld qm = 0.0L, q = 1.0L / sqrtl(be[0]), acc = q * q;
    for (int l = 0; l + 1 < n; ++l) {
      ld qn = ((x[i] - al[l]) * q - (l ? sqrtl(be[l]) : 0.0L) * qm) / sqrtl(be[l + 1]);
      qm = q;
      q = qn;
      acc += q * q;
    }
    w[i] = 1.0L / acc;
  }
}

void legendre_rule(int n, std::vector<ld>& x, std::vector<ld>& w) {
  std::vector<ld> al(n + 1, 0.0L), be(n + 1);
  be[0] = 2.0L;
  for (int k = 1; k <= n; ++k) be[k] = (ld)k * k / (4.0L * k * k - 1.0L);
  golub_welsch(n, al, be, x, w);
}

// Recurrence of the radial family: discretised Stieltjes in u, cosh xi = 1 + u^2.
void paper_radial_recurrence(int n, ld z0, std::vector<ld>& al, std::vector<ld>& be) {
  std::vector<ld> gx, gw;
  legendre_rule(24, gx, gw);
  const ld umax = sqrtl(1000.0L / z0) + 1.0L, hp = 0.25L;
  const int npan = (int)ceill(umax / hp);
  std::vector<ld> cc, W;
  cc.reserve(npan * 24);
  W.reserve(npan * 24);
  for (int a = 0; a < npan; ++a)
    for (int i = 0; i < 24; ++i) {
      ld u = hp * (a + 0.5L * (gx[i] + 1.0L));
      cc.push_back(1.0L + u * u);
      W.push_back(0.5L * hp * gw[i] * 2.0L * u * u * sqrtl(u * u + 2.0L) * expl(-z0 * (1.0L + u * u)));
    }
  const size_t M = cc.size();
  std::vector<ld> pm(M, 0.0L), p(M, 1.0L);
  al.assign(n + 1, 0.0L);
  be.assign(n + 1, 0.0L);
  ld prev = 1.0L;
  for (int k = 0; k <= n; ++k) {
    ld nn = 0.0L, xn = 0.0L;
    for (size_t i = 0; i < M; ++i) {
      nn += W[i] * p[i] * p[i];
      xn += W[i] * cc[i] * p[i] * p[i];
    }
    al[k] = xn / nn;
    be[k] = (k == 0) ? nn : nn / prev;
    prev = nn;
    for (size_t i = 0; i < M; ++i) {
      ld q = (cc[i] - al[k]) * p[i] - (k ? be[k] : 0.0L) * pm[i];
      pm[i] = p[i];
      p[i] = q;
    }
  }
}

// Barycentric differentiation matrix: D[i][j] = l_j'(x_i).
std::vector<ld> diff_matrix(const std::vector<ld>& x) {
  const int n = (int)x.size();
  std::vector<ld> lam(n, 1.0L), D(n * n, 0.0L);
  for (int j = 0; j < n; ++j)
    for (int m = 0; m < n; ++m)
      if (m != j) lam[j] /= (x[j] - x[m]);
  for (int i = 0; i < n; ++i) {
    ld diag = 0.0L;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      D[i * n + j] = (lam[j] / lam[i]) / (x[i] - x[j]);
      diag -= D[i * n + j];
    }
    D[i * n + i] = diag;
  }
  return D;
}

double sigma_of(const EosParams& p, double T) {
  return p.a * 0.5 * (1.0 + std::tanh((T - p.Tc) / p.w)) + p.b;
}
double sigmap_of(const EosParams& p, double T) {
  double ch = std::cosh((T - p.Tc) / p.w);
  return p.a * 0.5 / (p.w * ch * ch);
}

struct GL20 {
  double x[20], w[20];
  GL20() {
    std::vector<ld> gx, gw;
    legendre_rule(20, gx, gw);
    for (int i = 0; i < 20; ++i) { x[i] = (double)gx[i]; w[i] = (double)gw[i]; }
  }
};
const GL20& gl20() {
  static const GL20 g;
  return g;
}

// \int_0^inf F(t) e^{-x cosh t} dt on Gauss-Legendre panels of width 1/2.
template <class F>
double cosh_integral(double x, F&& fn) {
  const GL20& g = gl20();
  const double tmax = std::acosh(1.0 + 745.0 / x);
  const int npan = (int)std::ceil(tmax / 0.5);
  double sum = 0.0;
  for (int a = 0; a < npan; ++a) {
    double part = 0.0;
    for (int i = 0; i < 20; ++i) {
      double t = 0.5 * (a + 0.5 * (g.x[i] + 1.0));
      part += g.w[i] * fn(t) * std::exp(-x * std::cosh(t));
    }
    sum += 0.25 * part;
  }
  return sum;
}

// x^3 K_3(x) = tgt (decreasing in x): safeguarded Newton from a guess.
double solve_x(double tgt, double guess) {
  double lo = 1e-7, hi = 300.0, x = (guess > lo && guess < hi) ? guess : 2.0;
  for (int it = 0; it < 200; ++it) {
    double K[4];
    bessel_k(x, K);
    double F = x * x * x * K[3] - tgt;
    if (F > 0) lo = x; else hi = x;
    double xn = x + F / (x * x * x * K[2]);
    if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
    if (std::fabs(xn - x) <= 4e-16 * x) return xn;
    x = xn;
  }
  return x;
}

struct Node {
  double x, s, sp, pkin, e, D, htau, Bp;
};

Node eos_node(const EosParams& p, double T, double xguess) {
  Node o{};
  const double c2 = 2.0 * kPi * kPi, Z = p.Z;
  double J;
  if (p.kind == 2) {
    o.x = 0.0;
    o.s = 4.0 * Z * T * T * T / (kPi * kPi);
    o.sp = 3.0 * o.s / T;
    o.pkin = Z * T * T * T * T / (kPi * kPi);
    o.e = 3.0 * o.pkin;
    o.Bp = 0.0;
    J = 24.0 * std::pow(T, 5) / c2;
  } else {
    double x, K[4];
    if (p.kind == 1) {
      x = p.m0 / T;
      bessel_k(x, K);
      o.s = Z * p.m0 * p.m0 * p.m0 * K[3] / c2;
      o.sp = Z * p.m0 * p.m0 * p.m0 * (x * K[2] + 3.0 * K[3]) / (c2 * T);
      o.Bp = 0.0;
    } else {
      double sg = sigma_of(p, T);
      x = solve_x(c2 * sg / Z, xguess);
      bessel_k(x, K);
      o.s = T * T * T * sg;
      o.sp = 3.0 * T * T * sg + T * T * T * sigmap_of(p, T);
      double dxdT = -(c2 * sigmap_of(p, T) / Z) / (x * x * x * K[2]);
      double M = x * T, dMdT = x + T * dxdT;
      o.Bp = -Z * M * M * T * K[1] * dMdT / c2;
    }
    o.x = x;
    const double M = x * T;
    o.pkin = Z * M * M * T * T * K[2] / c2;
    o.e = T * o.s - o.pkin;
    double I6 = cosh_integral(x, [](double t) {
      double sh = std::sinh(t);
      return sh * sh * sh * sh * sh * sh / std::cosh(t);
    });
    J = std::pow(M, 5) * I6 / c2;
  }
  o.D = o.Bp / (T * o.sp);
  o.htau = 15.0 * T * o.s / (Z * J) * kHbarc;  // tau_R / (eta/s) in fm
  return o;
}

}  // namespace

void bessel_k(double x, double K[4]) {
  K[0] = cosh_integral(x, [](double) { return 1.0; });
  K[1] = cosh_integral(x, [](double t) { return std::cosh(t); });
  K[2] = K[0] + 2.0 / x * K[1];
  K[3] = K[1] + 4.0 / x * K[2];
}

std::string build_lattice(int family, int nxi, int nth, int nphi_half, double z0, Lattice* L) {
  if (nxi < 1 || nxi > kMaxN || nth < 1 || nth > kMaxN || nphi_half < 1 || 2 * nphi_half > kMaxN)
    return "lattice sizes out of range";
  if (family == 0 && !(z0 > 0.0)) return "z0 must be positive";
  L->nxi = nxi;
  L->nth = nth;
  L->nph = 2 * nphi_half;
  L->zexp = (family == 1) ? 1.0 : z0;
  // radial rule
  std::vector<ld> al, be, x, w;
  if (family == 1) {
    al.resize(nxi + 1);
    be.resize(nxi + 1);
    for (int k = 0; k <= nxi; ++k) {
      al[k] = 2.0L * k + 2.0L;
      be[k] = k == 0 ? 1.0L : (ld)k * (k + 1.0L);
    }
  } else {
    paper_radial_recurrence(nxi, z0, al, be);
  }
  golub_welsch(nxi, al, be, x, w);
  L->c.resize(nxi); L->s.resize(nxi); L->wxi.resize(nxi); L->ecw.resize(nxi);
  for (int k = 0; k < nxi; ++k) {
    L->c[k] = (double)x[k];
    L->s[k] = family == 1 ? (double)x[k] : (double)sqrtl((x[k] - 1.0L) * (x[k] + 1.0L));
    L->wxi[k] = (double)w[k];
    L->ecw[k] = (double)(expl((ld)L->zexp * x[k]) * w[k]);
  }
  // radial operator Dr = Galerkin(v . d/dv) in closed nodal form
  std::vector<ld> Dc = diff_matrix(x);
  L->Dr.assign(nxi * nxi, 0.0);
  for (int kp = 0; kp < nxi; ++kp)
    for (int k = 0; k < nxi; ++k) {
      ld ck = x[k], val;
      ld ratio = expl((ld)L->zexp * (x[k] - x[kp])) * w[k] / w[kp];
      if (family == 1) {
        val = -ratio * ck * Dc[k * nxi + kp];
        if (k == kp) val -= 2.0L;
      } else {
        val = -ratio * ((ck * ck - 1.0L) / ck) * Dc[k * nxi + kp];
        if (k == kp) val -= 2.0L + 1.0L / (ck * ck);
      }
      L->Dr[kp * nxi + k] = (double)val;
    }
  // polar rule and operators
  std::vector<ld> mu, wt;
  legendre_rule(nth, mu, wt);
  L->mu.resize(nth); L->sth.resize(nth); L->wth.resize(nth);
  for (int j = 0; j < nth; ++j) {
    L->mu[j] = (double)mu[j];
    L->sth[j] = (double)sqrtl((1.0L - mu[j]) * (1.0L + mu[j]));
    L->wth[j] = (double)wt[j];
  }
  std::vector<ld> Dm = diff_matrix(mu);
  L->Dth.assign(nth * nth, 0.0);
  for (int jp = 0; jp < nth; ++jp)
    for (int j = 0; j < nth; ++j) {
      ld m = mu[j];
      ld val = -(wt[j] / wt[jp]) * (m - m * m * m) * Dm[j * nth + jp];
      if (j == jp) val -= 1.0L - 3.0L * m * m;
      L->Dth[jp * nth + j] = (double)val;
    }
  // azimuths phi_l = l pi / N_phi (zeros of sin(N_phi phi))
  const int np = L->nph;
  L->cph.resize(np); L->sph.resize(np);
  for (int l = 0; l < np; ++l) {
    ld ph = (ld)l * kPi / nphi_half;
    ld cp = cosl(ph), sp = sinl(ph);
    L->cph[l] = fabsl(cp) < 1e-12L ? 0.0 : (double)cp;
    L->sph[l] = fabsl(sp) < 1e-12L ? 0.0 : (double)sp;
  }
  return "";
}

std::string build_eos_table(const EosParams& p, EosTable* out) {
  if (!(p.T_min > 0 && p.T_max > p.T_min)) return "invalid EOS temperature range";
  if (p.points < 64 || p.points > (1 << 22)) return "invalid EOS table size";
  if (!(p.Z > 0)) return "Z must be positive";
  if (p.kind == 1 && !(p.m0 > 0)) return "m0 must be positive";
  if (p.kind == 0 && !(p.w > 0)) return "w must be positive";
  if (p.kind < 0 || p.kind > 2) return "unknown EOS kind";
  const int pad = 3;
  const int n = p.points + 2 * pad;
  const double h = std::log(p.T_max / p.T_min) / (p.points - 1);
  const double y0 = std::log(p.T_min) - pad * h;
  out->y0 = y0;
  out->h = h;
  out->n = n;
  out->data.assign((size_t)n * kFields, 0.0);
  std::vector<Node> nodes(n);
  int nthr = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  std::vector<std::thread> pool;
  for (int t = 0; t < nthr; ++t)
    pool.emplace_back([&, t]() {
      int i0 = (int)((long long)n * t / nthr), i1 = (int)((long long)n * (t + 1) / nthr);
      double xg = 2.0;
      for (int i = i0; i < i1; ++i) {
        nodes[i] = eos_node(p, std::exp(y0 + i * h), xg);
        xg = nodes[i].x;
      }
    });
  for (auto& th : pool) th.join();
  // pressure p(T) = int_0^T s dT' (cumulative, 8-point Gauss-Legendre per cell in y)
  std::vector<ld> gx, gw;
  legendre_rule(8, gx, gw);
  std::vector<double> pr(n);
  const double T0 = std::exp(y0);
  auto s_of = [&](double T) { return T * T * T * sigma_of(p, T); };
  if (p.kind == 0) {
    ld acc = 0.0L;
    for (int i = 0; i < 8; ++i) {  // [0, T0]
      double T = 0.5 * T0 * ((double)gx[i] + 1.0);
      acc += 0.5L * T0 * gw[i] * s_of(T);
    }
    pr[0] = (double)acc;
    for (int q = 1; q < n; ++q) {
      double ya = y0 + (q - 1) * h;
      ld cell = 0.0L;
      for (int i = 0; i < 8; ++i) {
        double T = std::exp(ya + 0.5 * h * ((double)gx[i] + 1.0));
        cell += 0.5L * h * gw[i] * T * s_of(T);
      }
      acc += cell;
      pr[q] = (double)acc;
    }
  }
  for (int i = 0; i < n; ++i) {
    const double T = std::exp(y0 + i * h);
    const Node& o = nodes[i];
    double pres = (p.kind == 0) ? pr[i] : (p.kind == 1 ? o.pkin : o.pkin);
    double B = (p.kind == 0) ? o.pkin - pres : 0.0;
    double eps = T * o.s - pres;
    double* d = &out->data[(size_t)i * kFields];
    d[0] = o.e;
    d[1] = o.x;
    d[2] = o.D;
    d[3] = 1.0 / o.htau;
    d[4] = B / (T * T * T * T);
    d[5] = eps;
    d[6] = 0.0;
    d[7] = 0.0;
    for (int f = 0; f < 6; ++f)
      if (!std::isfinite(d[f])) return "non-finite EOS table entry";
    if (!(d[0] > 0.0 && d[5] > 0.0)) return "non-positive energy density in the EOS table";
  }
  return "";
}

}  // namespace rlb
