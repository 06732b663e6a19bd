"""GPU grid observables (rlb_observables: eps_p and p_perp-weighted v2) against
the FP64 oracle on the same seeded states, and against the exact value v2 = a/2
for an equilibrium modulated by (1 + a cos 2 phi).  The observables are ratios
of grid sums bounded by 1; tolerances are absolute: 1e-12 (FP64), 1e-5 (FP32)."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1108_5561_gb300 as rlb  # noqa: E402
from paper_1108_5561_gb300.inputs import hotspots  # noqa: E402

NT = os.cpu_count() or 1


def _pair(oracle_mod, g, eps0, steps):
    run = rlb.Run(g)
    run.init_grid(eps0)
    run.step(steps)
    og = run.observables()
    o = oracle_mod.Oracle(nx=g.nx, ny=g.ny, n_xi=g.n_xi, n_theta=g.n_theta, n_phi_half=g.n_phi_half,
                          eta_over_s=g.eta_over_s, dx=g.dx)
    f, lnM = o.init_state(eps0, NT)
    o.step(f, lnM, g.tau0, g.dtau, steps, NT)
    return og, o.observables(f, lnM, NT)


def test_fp64_observables_match_oracle(oracle_mod):
    g = rlb.GridParams(nx=12, ny=10, dx=0.2, prec=rlb.RLB_F64, eta_over_s=0.12, tau0=0.4, dtau=0.02)
    eps0, _, _ = hotspots(12, 10, dx=0.2, n=8, seed=21, spread=0.6, floor=0.005)
    (ep_g, v2_g), (ep_o, v2_o) = _pair(oracle_mod, g, eps0, 25)
    print("fp64 observables", ep_g, ep_o, v2_g, v2_o)
    assert abs(ep_o) > 1e-3 and abs(v2_o) > 1e-4  # the state is anisotropic
    assert abs(ep_g - ep_o) < 1e-12 and abs(v2_g - v2_o) < 1e-12


def test_fp32_observables_match_oracle(oracle_mod):
    g = rlb.GridParams(nx=24, ny=24, dx=0.1, prec=rlb.RLB_F32, eta_over_s=0.16, tau0=0.4, dtau=0.0036)
    eps0, _, _ = hotspots(24, 24, n=12, seed=1108, spread=0.6)
    (ep_g, v2_g), (ep_o, v2_o) = _pair(oracle_mod, g, eps0, 60)
    print("fp32 observables", ep_g, ep_o, v2_g, v2_o)
    assert abs(ep_g - ep_o) < 1e-5 and abs(v2_g - v2_o) < 1e-5


@pytest.mark.parametrize("prec,tol", [(rlb.RLB_F64, 1e-13), (rlb.RLB_F32, 1e-6)])
def test_v2_of_modulated_equilibrium_is_exact(prec, tol):
    g = rlb.GridParams(nx=5, ny=4, prec=prec)
    run = rlb.Run(g)
    run.init_grid(np.full((4, 5), 6.0))
    lat = run.lattice()
    phi = np.arctan2(lat["sph"], lat["cph"])
    mod = np.repeat(1.0 + 0.2 * np.cos(2 * phi), g.n_theta * g.n_xi)  # node order: k, then j, then l
    pops = run.populations()
    pops.mul_(torch.as_tensor(mod, dtype=pops.dtype, device=pops.device)[None, :])
    ep, v2 = run.observables()
    assert abs(v2 - 0.1) < tol
    assert ep > 0.05  # x pressure above y pressure
