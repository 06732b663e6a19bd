"""Pins of the oracle's equation of state against the paper's closed forms and
independent library routines (Sec. 2.1, Eq. epsp, Sec. 3.1, Sec. 4.1)."""
import math

import numpy as np
import pytest
from scipy import integrate, optimize, special

pytestmark = pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")

TS = [0.03, 0.1, 0.15, 0.165, 0.17, 0.18, 0.2, 0.3, 0.6, 1.5]


@pytest.fixture(scope="module")
def orc(oracle_mod):
    return oracle_mod.Oracle(nx=1, ny=1)


def test_bessel_matches_scipy(oracle_mod):
    # K_nu from the integral representation vs the library routine
    for x in [0.05, 0.3, 1.0, 1.8281, 3.3, 7.44, 15.0, 40.0]:
        K = oracle_mod.bessel_k(x)
        ref = [special.kv(n, x) for n in range(4)]
        assert np.allclose(K, ref, rtol=2e-14, atol=0), (x, K, ref)


def test_Z_qcd_constant(oracle_mod, paper_values):
    # Sec. 3.1: Z = pi^4/180 (4 (N_c^2 - 1) + 7 N_c N_f), N_c = N_f = 3 (fixture)
    nc, nf = paper_values["N_c"], paper_values["N_f"]
    assert oracle_mod.Z_QCD == pytest.approx(math.pi ** 4 / 180 * (4 * (nc * nc - 1) + 7 * nc * nf), rel=1e-15)
    assert oracle_mod.Z_QCD == pytest.approx(51.41035360127905, rel=1e-14)


@pytest.mark.parametrize("T", TS)
def test_mass_solves_entropy(orc, T):
    # (eps+p)/T = Z M^3 K_3(M/T)/(2 pi^2) = s(T) (Sec. 3.1), s/T^3 synthetic crossover
    p = orc.params
    e = orc.eos(T)
    sig = p["eos_a"] * 0.5 * (1 + math.tanh((T - p["eos_Tc"]) / p["eos_w"])) + p["eos_b"]
    s_ref = sig * T ** 3
    s_kin = p["Z"] * e["M"] ** 3 * special.kv(3, e["x"]) / (2 * math.pi ** 2)
    assert e["s"] == pytest.approx(s_ref, rel=1e-15)
    assert s_kin == pytest.approx(s_ref, rel=1e-13)


@pytest.mark.parametrize("T", TS)
def test_kinetic_energy_closed_form(orc, T):
    # Eq. epsp: eps - B = Z M^2 T^2 [3 K_2 + (M/T) K_1] / (2 pi^2); p + B = Z M^2 T^2 K_2/(2 pi^2)
    Z = orc.params["Z"]
    e = orc.eos(T)
    x, M = e["x"], e["M"]
    ek = Z * M * M * T * T * (3 * special.kv(2, x) + x * special.kv(1, x)) / (2 * math.pi ** 2)
    pk = Z * M * M * T * T * special.kv(2, x) / (2 * math.pi ** 2)
    assert e["e"] == pytest.approx(ek, rel=1e-13)
    assert e["pkin"] == pytest.approx(pk, rel=1e-13)
    # eps + p = T s (Eq. thermo at mu = 0) with eps = e + B, p = p_kin - B
    assert (e["e"] + e["B"]) + (e["pkin"] - e["B"]) == pytest.approx(T * e["s"], rel=1e-13)
    assert e["eps"] == pytest.approx(e["e"] + e["B"], rel=1e-12, abs=1e-18)


@pytest.mark.parametrize("T", [0.1, 0.17, 0.25, 0.6])
def test_entropy_is_dp_dT(orc, T):
    # s = dp/dT (thermodynamic consistency, Eq. thermcons) via a 4th-order difference of p(T)
    h = 1e-4
    p = [orc.eos(T + k * h)["p"] for k in (-2, -1, 1, 2)]
    dp = (p[0] - 8 * p[1] + 8 * p[2] - p[3]) / (12 * h)
    assert dp == pytest.approx(orc.eos(T)["s"], rel=1e-9)


def test_bag_function_integrates_consistency_ode(orc):
    # Sec. 3.1: dB/dT = -Z M^2 T K_1(M/T) dM/dT/(2 pi^2), integrated up from small T
    T0, T1 = 0.05, 0.4
    integral, err = integrate.quad(lambda t: orc.eos(t)["Bp"], T0, T1, epsabs=0, epsrel=1e-12,
                                   limit=200, points=[0.17])
    assert orc.eos(T1)["B"] - orc.eos(T0)["B"] == pytest.approx(integral, rel=1e-9)
    # and dB/dT against a numerical derivative of B(T)
    for T in [0.12, 0.17, 0.3]:
        h = 1e-4
        B = [orc.eos(T + k * h)["B"] for k in (-2, -1, 1, 2)]
        dB = (B[0] - 8 * B[1] + 8 * B[2] - B[3]) / (12 * h)
        assert orc.eos(T)["Bp"] == pytest.approx(dB, rel=1e-7, abs=1e-12)


def test_bag_low_temperature_closed_form(oracle_mod):
    # With s/T^3 constant, M = x* T and B(0) = 0 give B = -Z x*^3 K_1(x*) T^4/(8 pi^2)
    o = oracle_mod.Oracle(nx=1, ny=1, eos_a=0.0)
    Z, b = o.params["Z"], o.params["eos_b"]
    xs = optimize.brentq(lambda x: x ** 3 * special.kv(3, x) - 2 * math.pi ** 2 * b / Z, 0.1, 50,
                         xtol=1e-15)
    for T in [0.02, 0.1, 0.5]:
        e = o.eos(T)
        assert e["x"] == pytest.approx(xs, rel=1e-13)
        Bc = -Z * xs ** 3 * special.kv(1, xs) * T ** 4 / (8 * math.pi ** 2)
        assert e["B"] == pytest.approx(Bc, rel=1e-11)


@pytest.mark.parametrize("T", [0.12, 0.17, 0.3])
def test_dB_deps(orc, T):
    h = 1e-4
    B = [orc.eos(T + k * h)["B"] for k in (-2, -1, 1, 2)]
    E = [orc.eos(T + k * h)["eps"] for k in (-2, -1, 1, 2)]
    d = lambda v: (v[0] - 8 * v[1] + 8 * v[2] - v[3]) / (12 * h)
    assert orc.eos(T)["D"] == pytest.approx(d(B) / d(E), rel=1e-7)
    # de/dT = T s' - B'
    e = orc.eos(T)
    assert e["ep"] == pytest.approx(T * e["sp"] - e["Bp"], rel=1e-14)


def test_ideal_gas_speed_of_sound(oracle_mod):
    # Sec. 2.1: c_s^2 = (3 + (m/T) K_2/K_3)^{-1} for a constant-mass Boltzmann gas
    o = oracle_mod.Oracle(nx=1, ny=1, eos_kind=1, eos_m0=0.5)
    for T in [0.05, 0.2, 0.7]:
        e = o.eos(T)
        x = 0.5 / T
        cs2 = e["s"] / (T * e["sp"])
        assert cs2 == pytest.approx(1.0 / (3 + x * special.kv(2, x) / special.kv(3, x)), rel=1e-12)
        assert e["B"] == 0.0 and e["D"] == 0.0


def test_viscosity_integral(orc):
    # J = int d^3p/(2pi)^3 p^4/E^2 e^{-E/T}, independent quadrature in p
    for T in [0.15, 0.3]:
        e = orc.eos(T)
        M = e["M"]
        f = lambda p: p ** 6 / (p * p + M * M) * math.exp(-math.sqrt(p * p + M * M) / T)
        J, _ = integrate.quad(f, 0, 60 * T, epsabs=0, epsrel=1e-13, limit=200)
        assert e["J"] == pytest.approx(J / (2 * math.pi ** 2), rel=1e-11)


def test_massless_eta_limit(oracle_mod):
    # Sec. 4.1: massless eta = tau_R (eps + P)/5  =>  tau_R = 5 (eta/s) / T
    o = oracle_mod.Oracle(nx=1, ny=1, eos_kind=1, eos_m0=1e-5, eta_over_s=0.2)
    for T in [0.2, 0.5]:
        e = o.eos(T)
        assert e["s"] == pytest.approx(4 * o.params["Z"] * T ** 3 / math.pi ** 2, rel=1e-8)
        assert e["tauR"] == pytest.approx(5 * 0.2 / T * oracle_mod.HBARC, rel=1e-8)
    c = oracle_mod.Oracle(nx=1, ny=1, eos_kind=2, family=1, eta_over_s=0.2)
    e = c.eos(0.3)
    assert e["e"] == pytest.approx(3 * c.params["Z"] * 0.3 ** 4 / math.pi ** 2, rel=1e-15)
    assert e["tauR"] == pytest.approx(5 * 0.2 / 0.3 * oracle_mod.HBARC, rel=1e-14)


def test_constant_mass_eta(oracle_mod):
    # Sec. 4.1: constant mass: eta = (tau_R/T) int_0^T (eps + P) dT'
    o = oracle_mod.Oracle(nx=1, ny=1, eos_kind=1, eos_m0=0.5)
    Z = o.params["Z"]
    for T in [0.15, 0.4]:
        e = o.eos(T)
        eta_over_tau = Z * e["J"] / (15 * T)
        integ, _ = integrate.quad(lambda t: t * o.eos(t)["s"], 0.004, T, epsabs=0, epsrel=1e-12)
        assert eta_over_tau == pytest.approx(integ / T, rel=1e-9)


@pytest.mark.parametrize("T", [0.04, 0.16, 0.19, 0.35, 1.2])
def test_temperature_inversion(orc, T):
    e = orc.eos(T)
    assert orc.solve_T(e["e"], 0) == pytest.approx(T, rel=1e-14)
    assert orc.solve_T(e["eps"], 1) == pytest.approx(T, rel=1e-13)
