"""Size limits of the launch configuration.  A single grid runs on a (ny, nx)
CTA grid (ny, ceil(nx / 2) for the two-site variants), so nx is bounded by the
65,535 CTAs of the second launch dimension; a batch packs (x, y) of a site into
16 + 15 bits.  The longest allowed row is run for one step and checked at
sampled sites (both periodic ends, the interior) against the FP64 oracle on
11 x 11 windows, with the one-site and the two-site kernels; sizes beyond the
limits are rejected on the host."""
import ctypes
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1108_5561_gb300 as rlb  # noqa: E402

NT = os.cpu_count() or 1
NX_MAX = 65535


def _ripple(nx, ny):
    # smooth, non-periodic-looking structure along the whole row (including the
    # periodic seam between x = nx - 1 and x = 0), GeV/fm^3
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    return (10.0 + 2.0 * np.sin(2 * np.pi * x / 5.3 + 0.7) + 1.5 * np.cos(2 * np.pi * x / 17.1)
            + 0.8 * np.sin(2 * np.pi * (x + 3 * y) / 9.7))


def _sampled(oracle_mod, mg, eps0, picks, nx, ny):
    r = 5
    o = oracle_mod.Oracle(nx=2 * r + 1, ny=2 * r + 1, dx=0.1, eta_over_s=0.16)
    rows = []
    for s in picks:
        x, y = s % nx, s // nx
        win = eps0[np.ix_([(y + d) % ny for d in range(-r, r + 1)],
                          [(x + d) % nx for d in range(-r, r + 1)])]
        f, lnM = o.init_state(win, NT)
        o.step(f, lnM, 0.4, 0.0036, 1, NT)
        rows.append(o.moments(f, lnM, NT)[r * (2 * r + 1) + r])
    mo = np.array(rows)
    g = mg[picks]
    rel = lambda c: float(np.max(np.abs(g[:, c] - mo[:, c]) / np.abs(mo[:, c])))  # noqa: E731
    du = float(np.max(np.abs(g[:, 2:5] - mo[:, 2:5]).max(axis=1) / np.abs(mo[:, 2:5]).max(axis=1)))
    assert np.abs(mo[:, 3]).max() > 1e-4  # the step built transverse flow at the samples
    return {"eps": rel(0), "T": rel(1), "u": du}


@pytest.mark.parametrize("variant", [0, 3, 5, 6])
def test_longest_row_one_step_sampled(oracle_mod, variant):
    nx, ny = NX_MAX, 2
    g = rlb.GridParams(nx=nx, ny=ny, dx=0.1, prec=rlb.RLB_F32, eta_over_s=0.16, tau0=0.4, dtau=0.0036)
    eps0 = _ripple(nx, ny)
    run = rlb.Run(g)
    run.set_stage_variant(variant)
    run.init_grid(eps0)
    run.step(1)
    mg = run.moments()
    run.check()
    picks = [0, 1, nx - 2, nx - 1, nx, 2 * nx - 1, nx // 2, nx + 12345, 40000]
    e = _sampled(oracle_mod, mg, eps0, picks, nx, ny)
    print("longest row, variant", variant, e)
    assert e["eps"] < 1e-5 and e["T"] < 1e-5 and e["u"] < 1e-5, e


def test_streaming_stability_limit():
    # (dtau/dx) max(|V_x| + |V_y|) <= 1/2; max |V| < 1, so dtau = 0.3 dx passes and
    # dtau = 0.8 dx fails; a 1 x 1 grid has no streaming and takes any step
    rlb.Run(rlb.GridParams(nx=4, ny=4, dx=0.1, dtau=0.03, prec=rlb.RLB_F32))
    with pytest.raises(rlb.RLBError) as ei:
        rlb.Run(rlb.GridParams(nx=4, ny=4, dx=0.1, dtau=0.08, prec=rlb.RLB_F32))
    assert "stability" in str(ei.value)
    rlb.Run(rlb.GridParams(nx=1, ny=1, dx=0.1, dtau=0.2, prec=rlb.RLB_F32))


def test_sizes_beyond_the_limits_are_rejected():
    with pytest.raises(rlb.RLBError):
        rlb.Run(rlb.GridParams(nx=NX_MAX + 1, ny=1, prec=rlb.RLB_F32))
    g = rlb.GridParams(dx=0.1, prec=rlb.RLB_F32)
    with pytest.raises(rlb.RLBError):
        rlb.Run(g, events=[rlb.Event(NX_MAX + 1, 1, 0.1)])
    with pytest.raises(rlb.RLBError):
        rlb.Run(g, events=[rlb.Event(4, 32768, 0.1)])
    run = rlb.Run(rlb.GridParams(nx=4, ny=4, prec=rlb.RLB_F32))
    assert run.lib.rlb_configure_batch(run._h, ctypes.byref(run._gs), 0, None) == -1  # no events
