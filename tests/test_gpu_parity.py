"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on
the same seeded inputs.  Tolerances: 1e-12 relative for the FP64 path, 1e-5 for
FP32 populations (FP32 Landau/EOS), BF16 reported with a loose bound.

Norms (per site, maximum over the grid): eps and T relative; u the relative
error of the 4-vector, max_mu |du^mu| / max_mu |u^mu| (u^tau >= 1); u^tau
relative; uperp, a stricter FP64 check, |du_perp| / max(max |u_perp|, 1e-3)."""
import math
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1108_5561_gb300 as rlb  # noqa: E402
from paper_1108_5561_gb300.inputs import hotspots, smooth_gaussian  # noqa: E402

NT = os.cpu_count() or 1


def errors(mg, mo):
    d = {}
    for name, col in (("eps", 0), ("T", 1)):
        den = np.maximum(np.abs(mo[:, col]), 1e-6 * np.abs(mo[:, col]).max())
        d[name] = float(np.max(np.abs(mg[:, col] - mo[:, col]) / den))
    d["ut"] = float(np.max(np.abs(mg[:, 2] / mo[:, 2] - 1)))
    d["u"] = float(np.max(np.abs(mg[:, 2:5] - mo[:, 2:5]).max(axis=1) / np.abs(mo[:, 2:5]).max(axis=1)))
    d["uperp"] = float(np.max(np.abs(mg[:, 3:5] - mo[:, 3:5])) /
                       max(np.max(np.abs(mo[:, 3:5])), 1e-3))
    d["M"] = float(np.max(np.abs(mg[:, 5] / mo[:, 5] - 1)))
    return d


def run_pair(oracle_mod, g, eps0, steps, eos=None, okw=None):
    run = rlb.Run(g, eos)
    run.init_grid(eps0)
    run.step(steps)
    mg = run.moments()
    run.check()
    kw = dict(nx=g.nx, ny=g.ny, n_xi=g.n_xi, n_theta=g.n_theta, n_phi_half=g.n_phi_half,
              eta_over_s=g.eta_over_s, metric=g.metric, z0=g.z0, dx=g.dx, family=g.family, T0=g.T0)
    kw.update(okw or {})
    o = oracle_mod.Oracle(**kw)
    f, lnM = o.init_state(eps0, NT)
    o.step(f, lnM, g.tau0, g.dtau, steps, NT)
    return run, mg, o.moments(f, lnM, NT), (o, f, lnM)


def test_initial_state_matches_oracle(oracle_mod):
    g = rlb.GridParams(nx=9, ny=6, prec=rlb.RLB_F64)
    eps0, _, _ = hotspots(9, 6, dx=0.2, n=10, seed=3, spread=0.6, floor=0.005)
    run, mg, mo, (o, f, lnM) = run_pair(oracle_mod, g, eps0, 0)
    fg = run.populations().cpu().numpy()
    assert np.allclose(fg, f, rtol=1e-13, atol=0)
    assert np.allclose(run.lnM().cpu().numpy(), lnM, rtol=0, atol=1e-14)
    e = errors(mg, mo)
    assert e["eps"] < 1e-13 and e["T"] < 1e-13 and e["M"] < 1e-13, e
    assert e["uperp"] < 1e-12, e  # u_perp is rounding noise at rest


def test_fp64_config1_parity(oracle_mod):
    # 32x32, dx = 0.2 fm, 8 x 8 x 12 lattice, eta/s = 0.08, eps0 = 30 exp(-r^2/8), tau 0.4 -> 4
    g = rlb.GridParams(nx=32, ny=32, prec=rlb.RLB_F64, eta_over_s=0.08, tau0=0.4, dtau=0.018)
    eps0 = smooth_gaussian(32, 32)
    run, mg, mo, _ = run_pair(oracle_mod, g, eps0, 200)
    assert run.tau == pytest.approx(4.0, rel=1e-12)
    e = errors(mg, mo)
    print("config-1 errors", e)
    assert e["eps"] < 1e-12 and e["T"] < 1e-12 and e["ut"] < 1e-12 and e["uperp"] < 1e-12, e
    assert np.max(np.abs(mo[:, 3])) > 1e-2  # transverse flow developed


def test_fp64_ragged_grid_hotspots(oracle_mod):
    g = rlb.GridParams(nx=7, ny=5, n_xi=6, n_theta=4, n_phi_half=3, prec=rlb.RLB_F64,
                       eta_over_s=0.12, dtau=0.02)
    eps0, _, _ = hotspots(7, 5, dx=0.2, n=8, seed=11, spread=0.5, floor=0.005)
    _, mg, mo, _ = run_pair(oracle_mod, g, eps0, 15)
    e = errors(mg, mo)
    assert max(e.values()) < 1e-12, e


def test_fp64_minkowski_and_free_streaming(oracle_mod):
    g = rlb.GridParams(nx=6, ny=7, n_xi=6, n_theta=4, n_phi_half=3, prec=rlb.RLB_F64,
                       metric=rlb.RLB_MINKOWSKI, eta_over_s=math.inf, dtau=0.05, tau0=1.0)
    eps0, _, _ = hotspots(6, 7, dx=0.2, n=5, seed=5, spread=0.5, floor=0.005)
    _, mg, mo, _ = run_pair(oracle_mod, g, eps0, 10)
    e = errors(mg, mo)
    assert max(e.values()) < 1e-12, e


def test_fp64_minkowski_mass_gradients_with_collisions(oracle_mod):
    # Minkowski, crossover EOS, collisions on, one Gaussian bump: the mass-gradient
    # force and node motion act (grad ln M up to ~0.6/fm).  The GPU state matches
    # the oracle, and so does the change of sum_x (T^{tau tau}_kin + B) that the
    # lattice makes (a spatial discretisation error, see the oracle tests)
    from paper_1108_5561_gb300.inputs import coords
    n, dx = 12, 0.1
    X, Y = coords(n, n, dx)
    eps0 = 10.0 + 25.0 * np.exp(-((X - 0.13) ** 2 + (Y + 0.07) ** 2) / (2 * 0.25 ** 2))
    g = rlb.GridParams(nx=n, ny=n, dx=dx, prec=rlb.RLB_F64, metric=rlb.RLB_MINKOWSKI, eta_over_s=0.03,
                       tau0=1.0, dtau=0.005)
    run, mg, mo, (o, f, lnM) = run_pair(oracle_mod, g, eps0, 40)
    e = errors(mg, mo)
    assert max(e.values()) < 1e-12, e

    def energy(ff, lm, T):
        nd, w = o.nodes(), o.weights()
        c = np.tile(nd["c"], 12 * 8)
        M4 = np.exp(4 * lm)[:, None] / (2 * math.pi ** 2)
        return float(np.sum(M4 * ff * w * c * c) + sum(o.eos(t)["B"] for t in T))
    f0, lnM0 = o.init_state(eps0, NT)
    E0 = energy(f0, lnM0, o.moments(f0, lnM0, NT)[:, 1])
    dE_gpu = energy(run.populations().cpu().numpy(), run.lnM().cpu().numpy(), mg[:, 1]) / E0 - 1
    dE_orc = energy(f, lnM, mo[:, 1]) / E0 - 1
    print("energy change: GPU %.6e oracle %.6e" % (dE_gpu, dE_orc))
    assert abs(dE_orc) > 1e-5 and abs(dE_gpu - dE_orc) < 1e-12


def test_fp64_0p1d_paper_lattice(oracle_mod):
    # N_xi = N_theta = 5, dtau = 0.2 fm/c (Sec. 4.5), single site
    g = rlb.GridParams(nx=1, ny=1, n_xi=5, n_theta=5, n_phi_half=1, prec=rlb.RLB_F64,
                       eta_over_s=0.5, tau0=1.0, dtau=0.2)
    _, mg, mo, _ = run_pair(oracle_mod, g, np.array([[25.0]]), 15)
    e = errors(mg, mo)
    assert e["eps"] < 1e-12 and e["T"] < 1e-12, e


def test_static_equilibrium_on_gpu():
    # Minkowski, u = 0, z0 = M(T_s)/T_s: the populations stay at f_eq
    Ts, xs = 0.25, None
    from oracle.oracle import Oracle  # only for z0 of the reference temperature
    xs = Oracle(nx=1, ny=1).eos(Ts)
    g = rlb.GridParams(nx=4, ny=3, metric=rlb.RLB_MINKOWSKI, z0=xs["x"], prec=rlb.RLB_F64,
                       eta_over_s=0.1, tau0=0.5, dtau=0.05)
    run = rlb.Run(g)
    run.init_grid(np.full((3, 4), xs["eps"] / rlb.HBARC ** 3))
    f0 = run.populations().cpu().numpy().copy()
    run.step(100)
    run.check()
    f1 = run.populations().cpu().numpy()
    big = f0 > 1e-30
    assert np.max(np.abs(f1[big] / f0[big] - 1)) < 1e-11


def test_fp32_static_equilibrium_keeps_its_energy():
    # Minkowski, u = 0, uniform T_s, z0 = M(T_s)/T_s: the lattice moments of
    # f_eq are exact, so the populations must stay at f_eq.  With FP32
    # populations a factor common to every f_eq (a rounded log2 Z, a biased
    # 2^x or square root) shows up as a shift of the energy density, constant
    # after a few relaxation times (tau_R = 0.4 fm/c here; 2000 steps = 100 fm/c).
    Ts = 0.25
    from oracle.oracle import Oracle  # only for z0 of the reference temperature
    xs = Oracle(nx=1, ny=1).eos(Ts)
    g = rlb.GridParams(nx=4, ny=4, metric=rlb.RLB_MINKOWSKI, z0=xs["x"], prec=rlb.RLB_F32,
                       eta_over_s=0.1, tau0=0.5, dtau=0.05)
    run = rlb.Run(g)
    run.init_grid(np.full((4, 4), xs["eps"] / rlb.HBARC ** 3))
    e0 = run.moments()[:, 0].mean()
    run.step(500)
    e1 = run.moments()[:, 0].mean()
    run.step(1500)
    m = run.moments()
    run.check()
    shift, drift = e1 / e0 - 1, m[:, 0].mean() / e1 - 1
    print("FP32 static equilibrium: energy shift %.2e, drift over the last 1500 steps %.2e" % (shift, drift))
    assert abs(shift) < 5e-8 and abs(drift) < 2e-8
    assert np.abs(m[:, 3:5]).max() < 1e-7


def test_conformal_free_streaming_closed_form():
    g = rlb.GridParams(nx=1, ny=1, n_xi=8, n_theta=8, n_phi_half=1, family=rlb.RLB_RADIAL_LAGUERRE,
                       T0=0.5, prec=rlb.RLB_F64, eta_over_s=math.inf, tau0=0.4, dtau=0.004)
    run = rlb.Run(g, rlb.EosParams(kind=rlb.RLB_EOS_CONFORMAL))
    run.init_grid(np.array([[10.0]]))
    e0 = run.moments()[0, 0]
    run.step(300)
    r = run.tau / 0.4
    ex = 0.5 * (1 / r ** 2 + math.atan(math.sqrt(r * r - 1)) / math.sqrt(r * r - 1))
    assert run.moments()[0, 0] / e0 == pytest.approx(ex, rel=3e-4)


def test_fp32_hotspots_parity(oracle_mod):
    # config-2 physics (eta/s = 0.16, dtau = 0.0036, dx = 0.1 fm) on a 24x24 grid, 150 steps
    g = rlb.GridParams(nx=24, ny=24, dx=0.1, prec=rlb.RLB_F32, eta_over_s=0.16, tau0=0.4,
                       dtau=0.0036)
    eps0, _, _ = hotspots(24, 24, n=12, seed=1108, spread=0.6)
    _, mg, mo, _ = run_pair(oracle_mod, g, eps0, 150)
    e = errors(mg, mo)
    print("fp32 errors", e)
    assert np.abs(mo[:, 3:5]).max() > 1e-2  # developed transverse flow
    assert e["eps"] < 1e-5 and e["T"] < 1e-5 and e["u"] < 1e-5 and e["uperp"] < 1e-5, e


def test_fp32_config2_window_full_run(oracle_mod):
    # The 256x256 hotspot workload at its stated length: the central 32x32
    # window of its initial condition (40 hotspots, seed 1108; the densest part
    # of the grid), periodic, FP32 populations, eta/s = 0.16, 1000 steps of
    # dtau = 0.0036 fm/c from tau = 0.4 fm/c, against the FP64 oracle.  uperp is
    # |du_perp| / max |u_perp|: the flow is developed (max |u_perp| 0.33 at step
    # 150, 0.11 at the end).
    n = 256
    full, _, _ = hotspots(n, n, n=40, seed=1108)
    eps0 = full[112:144, 112:144].copy()
    g = rlb.GridParams(nx=32, ny=32, dx=0.1, prec=rlb.RLB_F32, eta_over_s=0.16, tau0=0.4, dtau=0.0036)
    run, mg, mo, _ = run_pair(oracle_mod, g, eps0, 1000)
    assert run.tau == pytest.approx(4.0, rel=1e-12)
    e = errors(mg, mo)
    print("config-2 window, 1000 steps", e)
    assert np.abs(mo[:, 3:5]).max() > 0.05
    assert e["eps"] < 1e-5 and e["T"] < 1e-5 and e["u"] < 1e-5 and e["uperp"] < 1e-5, e


def test_fp32_full_size_sampled(oracle_mod):
    # the benchmark workload: 256x256, 768 nodes, FP32, one step in the timed launch
    # configuration; checked at sampled sites (including the periodic edges) against
    # the oracle on 11x11 windows (the step's stencil reaches 4 sites).
    n = 256
    g = rlb.GridParams(nx=n, ny=n, dx=0.1, prec=rlb.RLB_F32, eta_over_s=0.16, tau0=0.4, dtau=0.0036)
    eps0, _, _ = hotspots(n, n, n=40, seed=1108)
    run = rlb.Run(g)
    run.init_grid(eps0)
    run.step(1)
    mg = run.moments()
    run.check()
    rng = np.random.default_rng(0)
    hot = np.argsort(eps0.reshape(-1))[-3:]
    picks = [0, n - 1, n * (n - 1), n * n - 1] + list(hot) + list(rng.integers(0, n * n, 5))
    r = 5
    o = oracle_mod.Oracle(nx=2 * r + 1, ny=2 * r + 1, dx=0.1, eta_over_s=0.16)
    rows = []
    for s in picks:
        x, y = s % n, s // n
        win = eps0[np.ix_([(y + d) % n for d in range(-r, r + 1)],
                          [(x + d) % n for d in range(-r, r + 1)])]
        f, lnM = o.init_state(win, NT)
        o.step(f, lnM, 0.4, 0.0036, 1, NT)
        rows.append(o.moments(f, lnM, NT)[r * (2 * r + 1) + r])
    mo = np.array(rows)
    worst = errors(mg[picks], mo)
    assert np.abs(mo[:, 3:5]).max() > 1e-4  # the step built transverse flow
    print("full-size sampled errors", worst)
    assert worst["eps"] < 1e-5 and worst["T"] < 1e-5 and worst["u"] < 1e-5, worst


def test_bf16_error_is_reported(oracle_mod):
    g = rlb.GridParams(nx=12, ny=12, dx=0.1, prec=rlb.RLB_BF16, eta_over_s=0.16, tau0=0.4,
                       dtau=0.0036)
    eps0, _, _ = hotspots(12, 12, n=6, seed=2, spread=0.3)
    _, mg, mo, _ = run_pair(oracle_mod, g, eps0, 50)
    e = errors(mg, mo)
    print("bf16 errors", e)  # reported, no fixed tolerance: a sanity bound only
    assert e["eps"] < 0.2 and e["T"] < 0.05, e


def test_out_of_table_temperature_sets_error_word():
    g = rlb.GridParams(nx=2, ny=2, prec=rlb.RLB_F32)
    run = rlb.Run(g)
    run.init_grid(np.full((2, 2), 1e9))  # far above the tabulated temperature range
    with pytest.raises(rlb.RLBError) as ei:
        run.check()
    assert ei.value.status == -3


def test_bad_eps0_is_rejected_on_host():
    run = rlb.Run(rlb.GridParams(nx=2, ny=2, prec=rlb.RLB_F32))
    with pytest.raises(rlb.RLBError) as ei:
        run.init_grid(np.array([[1.0, -1.0], [1.0, 1.0]]))
    assert ei.value.status == -1
