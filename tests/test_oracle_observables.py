"""Pins of the oracle's grid observables (eps_p, p_perp-weighted v2).

The paper defines no observables; these are the usual heavy-ion definitions
built on its moments (Eq. emtnew) and momentum weights (Sec. 4.3).  The pins use
exact properties of the azimuthal rule (phi_l = l pi / N_phi, 2 N_phi nodes):
sum_l cos 2phi_l = 0 and the mean of cos^2 2phi_l is 1/2, so a population
f_eq (1 + a cos 2 phi) has v2 = a/2 exactly, eps_p = a/2 exactly when B = 0,
and eps_p = (a/2) p_kin / (p_kin - B) up to the quadrature error of p_kin.
"""
import math

import numpy as np
import pytest


def _phi(o):
    nd = o.nodes()
    phi = np.arctan2(nd["sph"], nd["cph"])
    nth, nxi = len(nd["mu"]), len(nd["c"])
    return np.repeat(phi, nth * nxi)  # node order: k fastest, then j, then l


def _modulated(o, eps, a):
    f, lnM = o.init_state(eps)
    phi = _phi(o)
    return f * (1.0 + np.asarray(a)[:, None] * np.cos(2.0 * phi)[None, :]), lnM


def test_isotropic_equilibrium_has_no_anisotropy(oracle_mod):
    o = oracle_mod.Oracle(nx=3, ny=2)
    f, lnM = o.init_state(np.full(6, 7.0))
    ep, v2 = o.observables(f, lnM)
    assert abs(ep) < 1e-14 and abs(v2) < 1e-14


@pytest.mark.parametrize("a", [0.05, -0.2])
def test_v2_of_a_cos2phi_modulation(oracle_mod, a):
    o = oracle_mod.Oracle(nx=2, ny=2)
    f, lnM = _modulated(o, np.array([3.0, 5.0, 9.0, 20.0]), np.full(4, a))
    _, v2 = o.observables(f, lnM)
    assert v2 == pytest.approx(a / 2, rel=1e-13)


def test_conformal_eps_p_is_a_half(oracle_mod):
    # B = 0: T^xx - T^yy = (a/2)(T^xx + T^yy) node by node in phi
    o = oracle_mod.Oracle(nx=2, ny=1, eos_kind=2, family=1, T0=0.5)
    f, lnM = _modulated(o, np.array([4.0, 11.0]), np.array([0.1, 0.1]))
    ep, v2 = o.observables(f, lnM)
    assert ep == pytest.approx(0.05, rel=1e-12)
    assert v2 == pytest.approx(0.05, rel=1e-12)


def test_crossover_eps_p_carries_the_bag_term(oracle_mod):
    # eps_p = (a/2) p_kin(T) / (p_kin(T) - B(T)) for one site at rest; the lattice
    # p_kin differs from the continuum one by the radial quadrature error
    o = oracle_mod.Oracle(nx=1, ny=1)
    a = 0.1
    for eps in [2.0, 10.0]:
        f, lnM = _modulated(o, np.array([eps]), np.array([a]))
        ep, _ = o.observables(f, lnM)
        T = o.moments(f, lnM)[0, 1]
        e = o.eos(T)
        pkin, B = e["pkin"], e["B"]
        want = 0.5 * a * pkin / (pkin - B)
        assert ep == pytest.approx(want, rel=2e-3)
        assert abs(B) / pkin > 0.01  # the bag term matters at these temperatures


def test_sums_run_over_sites_not_site_ratios(oracle_mod):
    # two sites at the same temperature with different modulations: the grid v2
    # is the plain mean (equal denominators), a per-site average would agree too;
    # with different temperatures the site with the larger p_perp-weighted density
    # dominates
    o = oracle_mod.Oracle(nx=2, ny=1)
    f, lnM = _modulated(o, np.array([6.0, 6.0]), np.array([0.1, 0.3]))
    assert o.observables(f, lnM)[1] == pytest.approx(0.1, rel=1e-12)
    f, lnM = _modulated(o, np.array([1.0, 30.0]), np.array([0.1, 0.3]))
    v2 = o.observables(f, lnM)[1]
    assert 0.1 < v2 < 0.15 and v2 > 0.1 + 0.9 * (0.15 - 0.1)  # near the hot site's 0.15


def test_flow_in_x_gives_positive_eps_p(oracle_mod):
    # a population boosted along x (equilibrium at u^x > 0): T^xx > T^yy
    o = oracle_mod.Oracle(nx=1, ny=1)
    f, lnM = o.init_state(np.array([8.0]))
    nd = o.nodes()
    nth, nxi = len(nd["mu"]), len(nd["c"])
    vx = (nd["s"][None, None, :] * np.sqrt(1 - nd["mu"] ** 2)[None, :, None] * nd["cph"][:, None, None]).reshape(-1)
    fb = f * np.exp(0.3 * vx)[None, :]  # a boost-like tilt towards +x
    ep, v2 = o.observables(fb, lnM)
    assert ep > 0.01 and v2 > 0.0
