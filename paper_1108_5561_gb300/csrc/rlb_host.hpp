// rlb_host.hpp -- host-side construction of the momentum lattice, the nodal
// momentum-derivative operators and the equation-of-state table used by the
// GB300 kernels (Romatschke, arXiv:1108.5561, Sec. 3.1, 4.3, 4.4).
#pragma once

#include <string>
#include <vector>

namespace rlb {

constexpr double kPi = 3.14159265358979323846;
constexpr double kHbarc = 0.1973269804;  // GeV fm
constexpr int kMaxN = 32;

struct Lattice {
  int nxi = 0, nth = 0, nph = 0;
  double zexp = 1.0;  // exponent scale of the radial weight
  // radial: c = cosh xi (or x), s = sinh xi (or x), Gauss weights, e^{z c} w
  std::vector<double> c, s, wxi, ecw;
  // polar and azimuthal
  std::vector<double> mu, sth, wth, cph, sph;
  // nodal operators, row-major [out][in]
  std::vector<double> Dr, Dth;
};

struct EosParams {
  int kind = 0;  // 0 crossover, 1 constant mass, 2 conformal
  double a = 13.9, b = 0.5, Tc = 0.17, w = 0.02, m0 = 0.5, Z = 51.41035360127905;
  double T_min = 0.01, T_max = 4.0;
  int points = 65536;
};

// Table of EOS fields on a uniform grid in y = ln T; kFields doubles per node:
//   0: e(T) = eps - B, the kinetic equilibrium energy density [GeV^4]
//   1: x(T) = M(T)/T
//   2: D(T) = dB/deps
//   3: 1/h(T),  tau_R = (eta/s) h(T) [fm]  (Chapman-Enskog relation, Sec. 4.1)
//   4: B(T)/T^4
//   5: eps_EOS(T) [GeV^4]
constexpr int kFields = 8;
struct EosTable {
  double y0 = 0, h = 0;
  int n = 0;
  std::vector<double> data;  // n * kFields
};

// Returns an empty string on success, otherwise a message.
std::string build_lattice(int family, int nxi, int nth, int nphi_half, double z0, Lattice* out);
std::string build_eos_table(const EosParams& p, EosTable* out);

// Exposed for host-side unit tests.
void bessel_k(double x, double K[4]);

}  // namespace rlb
