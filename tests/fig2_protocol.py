"""The protocol of the paper's Fig. 2 (Sec. 4.5) on the GPU step: 0+1D Bjorken
flow in the Milne metric on the N_xi = N_theta = 5 lattice with
dtau = 0.2 fm/c.  Temperature evolution of the lattice Boltzmann step for
eta/s = 0.08, 0.5 and infinity (collisions off, the mass following the energy
density) against second-order viscous hydrodynamics (Eq. hydroeq with
tau_pi = 5 eta/(eps+P), lambda_1 = 5/7 eta tau_pi, the values the paper uses)
and against ideal hydrodynamics with the ideal (conformal) equation of state,
T = T0 (tau0/tau)^(1/3).  The synthetic crossover EOS replaces the lattice-QCD
one of the paper; tau0 = 0.4 fm/c, T0 = 0.4 GeV, to tau = 10 fm/c (the
crossover, T_c = 0.17 GeV, slows the cooling from T ~ 0.2 GeV on).  The hydrodynamic curves use the oracle's EOS.

    python tests/fig2_protocol.py        # prints the table (needs a GPU)
"""
import math
import os
import sys

import numpy as np
from scipy.integrate import solve_ivp

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from tests.conftest import golden  # noqa: E402

PAPER = golden("paper_values.txt")  # the run parameters and hydro coefficients of Sec. 4.5
HC = 0.1973269804
H3 = HC ** 3
TAU0, T0, DTAU, TAU1 = 0.4, 0.4, PAPER["fig2_dtau_fm"], 10.0
N_XI, N_TH, Z0 = int(PAPER["fig2_N_xi"]), int(PAPER["fig2_N_theta"]), PAPER["fig2_z0"]
ETAS = (0.08, 0.5, math.inf)


def lattice_boltzmann(etas):
    """(tau, T) of the GPU step for one eta/s."""
    import paper_1108_5561_gb300 as rlb
    from oracle.oracle import Oracle

    eps0 = Oracle(nx=1, ny=1).eos(T0)["eps"] / H3  # GeV/fm^3
    g = rlb.GridParams(nx=1, ny=1, n_xi=N_XI, n_theta=N_TH, n_phi_half=1, prec=rlb.RLB_F64,
                       eta_over_s=etas, tau0=TAU0, dtau=DTAU, z0=Z0)
    run = rlb.Run(g)
    run.init_grid(np.array([[eps0]]))
    taus, Ts = [TAU0], [run.moments()[0, 1]]
    while taus[-1] < TAU1 - 1e-9:
        run.step(1)
        taus.append(run.tau)
        Ts.append(run.moments()[0, 1])
    run.check()
    return np.array(taus), np.array(Ts)


def viscous_hydro(etas, taus):
    """T(tau) of Eq. hydroeq (Bjorken, second order) with the oracle's EOS."""
    from oracle.oracle import Oracle

    o = Oracle(nx=1, ny=1)
    eps0 = o.eos(T0)["eps"]

    def rhs(t, y):
        eps, Phi = y
        e = o.eos(o.solve_T(eps, 1))
        P, eta = e["p"], etas * e["s"]
        tp = PAPER["hydro_tau_pi_coeff"] * eta / (eps + P)
        lam = PAPER["hydro_lambda1_num"] / PAPER["hydro_lambda1_den"] * eta * tp
        return [-(eps + P) / t + Phi / t,
                -Phi / tp + 4 * eta / (3 * tp * t) - 4 * Phi / (3 * t) - lam / (2 * tp * eta ** 2) * Phi ** 2]

    sol = solve_ivp(rhs, [TAU0 / HC, taus[-1] / HC], [eps0, 0.0], t_eval=np.asarray(taus) / HC,
                    rtol=1e-10, atol=1e-14)
    return np.array([o.solve_T(e, 1) for e in sol.y[0]])


def table():
    rows = {}
    for etas in ETAS:
        taus, T = lattice_boltzmann(etas)
        rows[etas] = (taus, T, viscous_hydro(etas, taus) if math.isfinite(etas) else None)
    return rows


if __name__ == "__main__":
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    rows = table()
    taus = rows[ETAS[0]][0]
    ideal = T0 * (TAU0 / taus) ** (1.0 / 3.0)
    head = "tau[fm/c]  ideal-EOS  " + "  ".join("LB(%s) VH(%s)" % (e, e) for e in ETAS[:2]) + "  LB(inf)"
    print(head)
    for i in range(0, len(taus), 4):
        cells = ["%7.2f" % taus[i], "%9.4f" % ideal[i]]
        for e in ETAS[:2]:
            cells.append("%8.4f %8.4f" % (rows[e][1][i], rows[e][2][i]))
        cells.append("%8.4f" % rows[math.inf][1][i])
        print("  ".join(cells))
