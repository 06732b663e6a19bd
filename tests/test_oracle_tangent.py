"""The oracle in complex arithmetic (complex-step derivatives, the tangent
oracle that gives the adjoint's reference gradient): its real part is the FP64
oracle, and its derivatives of the final p_perp-weighted v2 with respect to a
hotspot amplitude and to eta/s agree with central differences of the FP64
oracle to their O(h^2) truncation error."""
import numpy as np
import pytest

from paper_1108_5561_gb300.inputs import hotspot_basis, hotspots

N, STEPS = 8, 20


def _case():
    eps0, amps, cen = hotspots(N, N, n=4, seed=5, spread=0.25, mean_amp=15.0)
    return eps0, hotspot_basis(N, N, cen).reshape(4, N, N)


def _v2(oracle_mod, eps0, eta):
    o = oracle_mod.Oracle(nx=N, ny=N, dx=0.1, eta_over_s=eta)
    f, lnM = o.init_state(eps0)
    o.step(f, lnM, 0.4, 0.0036, STEPS)
    return o.observables(f, lnM)[1]


def test_tangent_oracle_real_part_is_the_oracle(oracle_mod):
    eps0, basis = _case()
    o = oracle_mod.TangentOracle(nx=N, ny=N, dx=0.1, eta_over_s=0.16)
    f, lnM = o.init_state(eps0 + 0j)
    o.step(f, lnM, 0.4, 0.0036, STEPS)
    r = oracle_mod.Oracle(nx=N, ny=N, dx=0.1, eta_over_s=0.16)
    fr, lnMr = r.init_state(eps0)
    r.step(fr, lnMr, 0.4, 0.0036, STEPS)
    # the same arithmetic up to rounding (the complex build ends its Newton
    # solves with one more step, and complex exponentials round their own way)
    assert np.array_equal(f.imag, np.zeros_like(fr))
    assert np.abs(f.real - fr).max() < 1e-13 * np.abs(fr).max()
    mo, mr = o.moments(f, lnM).real, r.moments(fr, lnMr)
    assert np.abs(mo - mr).max() < 1e-13 * np.abs(mr).max()


@pytest.mark.parametrize("which", ["amplitude", "eta"])
def test_complex_step_matches_central_differences(oracle_mod, which):
    eps0, basis = _case()
    d_eps = basis[0] if which == "amplitude" else 0 * eps0
    d_eta = 0.0 if which == "amplitude" else 1.0
    v2, d = oracle_mod.v2_directional_derivative(eps0, d_eps, d_eta, STEPS, 0.4, 0.0036, nx=N, ny=N, dx=0.1,
                                                  eta_over_s=0.16)
    assert v2 == pytest.approx(_v2(oracle_mod, eps0, 0.16), rel=1e-13)
    fd = []
    for h in (2e-2, 1e-2):
        s = h * (1.0 if which == "amplitude" else 0.16)
        plus = _v2(oracle_mod, eps0 + s * d_eps, 0.16 + s * d_eta)
        minus = _v2(oracle_mod, eps0 - s * d_eps, 0.16 - s * d_eta)
        fd.append((plus - minus) / (2 * s))
    e1, e2 = abs(fd[0] - d), abs(fd[1] - d)
    print(which, "complex step %.10e, central differences %.10e %.10e" % (d, fd[0], fd[1]))
    # the finite-difference error falls as h^2 towards the complex-step value
    assert e2 < 1e-4 * abs(d)
    assert e2 < 0.35 * e1 or e2 < 1e-9 * abs(d)
