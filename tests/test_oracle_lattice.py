"""Pins of the oracle's momentum lattice (Sec. 4.3) and momentum-derivative
operators (Sec. 4.4) against closed forms, library rules, and the exact
integration-by-parts identities the Galerkin construction must satisfy."""
import math

import numpy as np
import pytest
from scipy import special

mp = pytest.importorskip("mpmath")


def radial_moment(z0, j):
    # mu_j = int_1^inf c^j e^{-z0 c} sqrt(c^2 - 1) dc  (= int dxi e^{-z0 cosh} sinh^2 cosh^j)
    mp.mp.dps = 40
    return float(mp.quad(lambda c: c ** j * mp.e ** (-z0 * c) * mp.sqrt(c * c - 1),
                         [1, 2, 5, 15, 40, 120, mp.inf]))


@pytest.mark.parametrize("z0", [0.5, 1.0, 1.8281, 3.0])
@pytest.mark.parametrize("N", [1, 3, 5, 8, 16])
def test_radial_weight_sum(oracle_mod, z0, N):
    # Sec. 4.3: sum_k w_k^xi R_0(xi_k) = K_1(z0)/z0
    o = oracle_mod.Oracle(nx=1, ny=1, n_xi=N, z0=z0)
    assert o.nodes()["wxi"].sum() == pytest.approx(special.kv(1, z0) / z0, rel=2e-14)


@pytest.mark.parametrize("z0", [0.7, 1.0, 2.5])
def test_radial_first_node_is_root_of_R1(oracle_mod, z0):
    # Sec. 4.3: R_1 = cosh xi - K_2(z0)/K_1(z0): the one-point rule sits at its root
    o = oracle_mod.Oracle(nx=1, ny=1, n_xi=1, z0=z0)
    assert o.nodes()["c"][0] == pytest.approx(special.kv(2, z0) / special.kv(1, z0), rel=1e-14)


@pytest.mark.parametrize("z0,N", [(1.0, 5), (1.0, 8), (1.8281, 8), (1.0, 16)])
def test_radial_gauss_exactness(oracle_mod, z0, N):
    # exact for e^{-z0 cosh} sinh^2 cosh^j, j <= 2N - 1 (Sec. 4.3)
    o = oracle_mod.Oracle(nx=1, ny=1, n_xi=N, z0=z0)
    nd = o.nodes()
    for j in range(0, 2 * N):
        got = float(np.sum(nd["wxi"] * nd["c"] ** j))
        assert got == pytest.approx(radial_moment(z0, j), rel=5e-13), j
    assert np.allclose(nd["s"], np.sqrt(nd["c"] ** 2 - 1), rtol=1e-15)
    assert np.all(np.diff(nd["c"]) > 0) and nd["c"][0] > 1


def test_laguerre_family_matches_library(oracle_mod):
    # conformal limit: Gauss rule for x e^{-x} (generalised Laguerre, alpha = 1)
    o = oracle_mod.Oracle(nx=1, ny=1, eos_kind=2, family=1, n_xi=8)
    x, w = special.roots_genlaguerre(8, 1.0)
    nd = o.nodes()
    assert np.allclose(nd["c"], x, rtol=1e-13)
    assert np.allclose(nd["wxi"], w, rtol=1e-12)


@pytest.mark.parametrize("Nt", [2, 5, 8, 12])
def test_gauss_legendre(oracle_mod, Nt):
    # Sec. 4.3: roots of L_N, w = 2/((1-x^2) L_N'(x)^2)
    o = oracle_mod.Oracle(nx=1, ny=1, n_theta=Nt)
    x, w = np.polynomial.legendre.leggauss(Nt)
    nd = o.nodes()
    assert np.allclose(nd["mu"], x, atol=1e-15, rtol=0)
    assert np.allclose(nd["wth"], w, atol=1e-15, rtol=0)


@pytest.mark.parametrize("Nphi", [2, 3, 6, 8])
def test_azimuthal_rule(oracle_mod, Nphi):
    # Sec. 4.3: phi_l = l pi / N_phi integrates (sin)^a (cos)^b exactly for a + b < 2 N_phi
    o = oracle_mod.Oracle(nx=1, ny=1, n_phi_half=Nphi)
    nd = o.nodes()
    L = 2 * Nphi
    phi = np.arange(L) * math.pi / Nphi
    assert np.allclose(nd["cph"], np.where(abs(np.cos(phi)) < 1e-12, 0, np.cos(phi)), atol=1e-15)
    for a in range(0, 2 * Nphi):
        for b in range(0, 2 * Nphi - a):
            num = np.mean(np.sin(phi) ** a * np.cos(phi) ** b)
            ex = 0.0
            if a % 2 == 0 and b % 2 == 0:
                ex = special.beta((a + 1) / 2, (b + 1) / 2) / math.pi
            assert num == pytest.approx(ex, abs=1e-14), (a, b)


def test_full_lattice_integrates_moments(oracle_mod):
    # sum_n w_n f(P_n) = int dOmega/4pi int dxi sinh^2 xi f  for f = e^{-z0 c} q(c, v)
    o = oracle_mod.Oracle(nx=1, ny=1)
    nd = o.nodes()
    w = o.weights().reshape(12, 8, 8)
    c = nd["c"][None, None, :]
    s = nd["s"][None, None, :]
    st = nd["sth"][None, :, None]
    mu = nd["mu"][None, :, None]
    cp = nd["cph"][:, None, None]
    sp = nd["sph"][:, None, None]
    vx, vy, vz = s * st * cp, s * st * sp, s * mu
    f = np.exp(-1.0 * c)
    # energy-like c^2 f: int = mu_2 ; vx^2 f: (1/3) int s^2 ; vx^2 vy^2 f: (1/15) int s^4
    assert np.sum(w * c ** 2 * f) == pytest.approx(radial_moment(1.0, 2), rel=1e-13)
    s2 = radial_moment(1.0, 2) - radial_moment(1.0, 0)
    s4 = radial_moment(1.0, 4) - 2 * radial_moment(1.0, 2) + radial_moment(1.0, 0)
    assert np.sum(w * vx ** 2 * f) == pytest.approx(s2 / 3, rel=1e-13)
    assert np.sum(w * vz ** 2 * f) == pytest.approx(s2 / 3, rel=1e-13)
    assert np.sum(w * vx ** 2 * vy ** 2 * f) == pytest.approx(s4 / 15, rel=1e-13)
    assert abs(np.sum(w * vx * c * f)) < 1e-15


def _grid(o):
    nd = o.nodes()
    p = o.params
    L, Nt, N = 2 * p["n_phi_half"], p["n_theta"], p["n_xi"]
    c = np.broadcast_to(nd["c"][None, None, :], (L, Nt, N))
    s = np.broadcast_to(nd["s"][None, None, :], (L, Nt, N))
    mu = np.broadcast_to(nd["mu"][None, :, None], (L, Nt, N))
    return c, s, mu, o.weights().reshape(L, Nt, N)


def _apply(o, f):
    ops = o.operators()
    S2 = np.einsum("ab,ljb->lja", ops["Dr"], f)
    Dth = np.einsum("ab,lbk->lak", ops["Dth"], f)
    c, s, mu, w = _grid(o)
    S1 = mu ** 2 * S2 + Dth
    return S1, S2


@pytest.mark.parametrize("fam", [0, 1])
def test_galerkin_integration_by_parts(oracle_mod, fam):
    # Exact discrete identities sum_n w psi (S f) = - sum_n w f (S^dagger psi) for the test
    # functions psi the Galerkin space contains (continuum: int d^3v/c psi v.d_v f = ...).
    kw = dict(nx=1, ny=1) if fam == 0 else dict(nx=1, ny=1, eos_kind=2, family=1)
    o = oracle_mod.Oracle(**kw)
    rng = np.random.default_rng(5)
    c, s, mu, w = _grid(o)
    f = np.exp(-1.0 * c) * (1 + 0.3 * rng.standard_normal(c.shape))
    S1, S2 = _apply(o, f)
    tot = lambda a: float(np.sum(w * a))
    scale = tot(c ** 2 * np.abs(f))
    if fam == 0:
        cases = [
            (1.0, S2, (2 + 1 / c ** 2)),                       # psi = 1,   v.d_v
            (c, S2, 3 * c),                                     # psi = c
            (c ** 2, S2, 4 * c ** 2 - 1),                       # psi = c^2  (energy)
            (1.0, S1, 1 - mu ** 2 * s ** 2 / c ** 2),           # psi = 1,   v_z d_vz
            (c ** 2, S1, c ** 2 + s ** 2 * mu ** 2),            # psi = c^2
            (s ** 2 * mu ** 2, S1, 3 * s ** 2 * mu ** 2 - s ** 4 * mu ** 4 / c ** 2),
        ]
    else:
        cases = [
            (1.0, S2, 2.0 + 0 * c),
            (c ** 2, S2, 4 * c ** 2),
            (c ** 2, S1, c ** 2 + c ** 2 * mu ** 2),
        ]
    for psi, Sf, adj in cases:
        lhs = tot(psi * Sf)
        rhs = -tot(adj * f)
        assert lhs == pytest.approx(rhs, abs=1e-13 * scale)


def _landau_case(rng):
    # T = Lambda diag(eps, p1, p2, p3) Lambda^T (anisotropic, boosted in x-y)
    eps = 2.0 + rng.random()
    p = eps * np.array([0.2, 0.35, 0.1]) * (0.5 + rng.random(3))
    vx, vy = 0.6 * (rng.random(2) - 0.5)
    ut = 1 / math.sqrt(1 - vx * vx - vy * vy)
    u = np.array([ut, ut * vx, ut * vy, 0.0])
    g = np.diag([1.0, -1, -1, -1])
    # orthonormal spatial triad orthogonal to u (Gram-Schmidt in Minkowski metric)
    basis = [u]
    for e in np.eye(4)[1:]:
        v = e.copy()
        for b in basis:
            v = v - (b @ g @ v) / (b @ g @ b) * b
        v /= math.sqrt(-(v @ g @ v))
        basis.append(v)
    Tmn = eps * np.outer(u, u) + sum(pi * np.outer(b, b) for pi, b in zip(p, basis[1:]))
    return Tmn, u, eps


def test_landau_matching(oracle_mod):
    rng = np.random.default_rng(11)
    for _ in range(20):
        Tmn, u, eps = _landau_case(rng)
        u2, e2 = oracle_mod.landau(Tmn)
        assert e2 == pytest.approx(eps, rel=1e-13)
        assert np.allclose(u2, u, rtol=0, atol=1e-13)
        # the library eigen solver on T^mu_nu agrees
        w, V = np.linalg.eig(Tmn @ np.diag([1.0, -1, -1, -1]))
        assert np.max(w.real) == pytest.approx(eps, rel=1e-12)
