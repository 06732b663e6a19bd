"""Two facts the FP32 matching kernel relies on, checked against the oracle.

1. Landau matching (Eq. sanity): for a kinetic T^{mu nu} built from
   non-negative populations on the momentum lattice (a positive sum of p^mu
   p^nu / p^0 terms), the energy u_mu u_nu T^{mu nu} in any frame is at least
   the Landau energy density eps (eps is its minimum over timelike unit u).
   The kernel starts its Newton iteration for the largest root of the cubic
   from the energy in the frame moving with T^{0i} / T^{00}, which must
   therefore lie at or above the root.
2. EOS inversion (Sec. 3.1, 4.4): the kernel stops its FP32 Newton iteration
   on e(y) = eps_kin, y = ln T, at a step below 5e-4 and leaves the rest to one
   double-FP32 Newton step; the error after the stop is C dy^2 with
   C = e''/(2 e'), which must stay below 8 over the tabulated range for that
   step to reach ~3e-11."""
import numpy as np
import pytest


def _energy_in_flux_frame(T):
    """u_mu u_nu T^{mu nu} for u along (T^{00}, T^{0x}, T^{0y}) (3x3 block)."""
    b = T[0, 1:] / T[0, 0]
    bb = float(b @ b)
    assert bb < 1.0
    return (T[0, 0] - 2.0 * float(b @ T[0, 1:]) + float(b @ T[1:, 1:] @ b)) / (1.0 - bb)


def _landau_eps(oracle_mod, T3):
    T4 = np.zeros((4, 4))
    T4[:3, :3] = T3
    T4[3, 3] = 0.3 * T3[0, 0]  # the Y component, decoupled from the (tau, x, y) block
    _, eps = oracle_mod.landau(T4)
    return eps


def test_energy_in_the_flux_frame_bounds_the_landau_energy(oracle_mod):
    orc = oracle_mod.Oracle(nx=1, ny=1)
    nd = orc.nodes()
    w = orc.weights()
    nph = 2 * orc.params["n_phi_half"]
    # node momenta (per unit mass) in node order [phi][theta][xi]
    sh, ch = nd["s"], nd["c"]
    st, mu = nd["sth"], nd["mu"]
    cp, sp = nd["cph"], nd["sph"]
    px = np.einsum("l,j,k->ljk", cp, st, sh).reshape(-1)
    py = np.einsum("l,j,k->ljk", sp, st, sh).reshape(-1)
    pz = np.einsum("l,j,k->ljk", np.ones(nph), mu, sh).reshape(-1)
    E = np.einsum("l,j,k->ljk", np.ones(nph), np.ones_like(mu), ch).reshape(-1)
    rng = np.random.default_rng(1108)
    worst = np.inf
    for trial in range(400):
        # a boosted equilibrium on the lattice with random positive distortions
        v = rng.uniform(0.0, 0.9)
        a = rng.uniform(0.0, 2.0 * np.pi)
        g = 1.0 / np.sqrt(1.0 - v * v)
        ut, ux, uy = g, g * v * np.cos(a), g * v * np.sin(a)
        z = rng.uniform(1.0, 7.0)
        f = np.exp(-z * (ut * E - ux * px - uy * py)) * rng.uniform(0.5, 1.5, E.size)
        P = [E, px, py]
        T3 = np.array([[np.sum(w * f * P[m] * P[n] / E) for n in range(3)] for m in range(3)])
        eps = _landau_eps(oracle_mod, T3)
        e_flux = _energy_in_flux_frame(T3)
        worst = min(worst, e_flux / eps - 1.0)
        assert e_flux >= eps * (1.0 - 1e-12), (trial, e_flux, eps)
    assert worst > -1e-12


def test_eos_newton_constant_is_small(oracle_mod):
    orc = oracle_mod.Oracle(nx=1, ny=1)
    ys = np.linspace(np.log(0.03), np.log(1.5), 4001)
    e = np.array([orc.eos(np.exp(y))["e"] for y in ys])
    h = ys[1] - ys[0]
    d1 = np.gradient(e, h)
    d2 = np.gradient(d1, h)
    assert np.all(d1 > 0.0)
    C = d2 / (2.0 * d1)
    assert C.max() < 8.0, (C.max(), np.exp(ys[C.argmax()]))
    # the error left by the FP32 stop rule, then after one exact Newton step
    err_stop = C.max() * 5e-4 ** 2
    assert err_stop < 2.1e-6 and C.max() * err_stop ** 2 < 4e-11
