"""rlb_moments matches the current state; the next rlb_step starts from that
matching instead of repeating it.  Stepping with per-step observables (host or
device output, graphs on or off, one or several steps per call) must give the
same states bit for bit as stepping without them."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1108_5561_gb300 as rlb  # noqa: E402
from paper_1108_5561_gb300._lib import RLB_ERR_ARG  # noqa: E402
from paper_1108_5561_gb300.inputs import hotspots  # noqa: E402


@pytest.mark.parametrize("prec", [rlb.RLB_F64, rlb.RLB_F32])
@pytest.mark.parametrize("graphs", [True, False])
def test_per_step_moments_do_not_change_the_run(prec, graphs):
    g = rlb.GridParams(nx=11, ny=9, dx=0.1, prec=prec, eta_over_s=0.12, tau0=0.4, dtau=0.0036)
    eps, _, _ = hotspots(11, 9, n=4, seed=21, spread=0.4)
    a = rlb.Run(g)
    a.set_graphs(graphs)
    a.init_grid(eps)
    a.step(9)
    b = rlb.Run(g)
    b.set_graphs(graphs)
    b.init_grid(eps)
    for i in range(6):
        b.step(1)
        b.moments(host=(i % 2 == 0))
    b.step(3)  # one call: the first step reuses the matching, the others do not
    torch.cuda.synchronize()
    a.check()
    b.check()
    assert torch.equal(a.populations(), b.populations())
    assert torch.equal(a.lnM(), b.lnM())
    assert a.tau == b.tau
    assert np.array_equal(a.moments(), b.moments())


@pytest.mark.parametrize("prec", [rlb.RLB_F64, rlb.RLB_F32])
@pytest.mark.parametrize("graphs", [True, False])
def test_async_moments_equal_synchronous_moments(prec, graphs):
    """rlb_moments_async (two staging slots, downloads overlapping the next
    steps) delivers, for every step, the same observables as rlb_moments, and
    the run it is interleaved with gives the same states bit for bit."""
    g = rlb.GridParams(nx=13, ny=10, dx=0.1, prec=prec, eta_over_s=0.12, tau0=0.4, dtau=0.0036)
    eps, _, _ = hotspots(13, 10, n=4, seed=22, spread=0.4)
    a = rlb.Run(g)
    a.set_graphs(graphs)
    a.init_grid(eps)
    want = []
    for _ in range(5):
        a.step(1)
        want.append(a.moments())
    b = rlb.Run(g)
    b.set_graphs(graphs)
    b.init_grid(eps)
    outs = [torch.empty((b.ns, 8), dtype=torch.float64).pin_memory() for _ in range(5)]
    for k in range(5):
        b.step(1)
        b.moments_async(outs[k])
    b.moments_wait()
    torch.cuda.synchronize()
    for k in range(5):
        assert np.array_equal(outs[k].numpy().reshape(want[k].shape), want[k]), k
    assert torch.equal(a.populations(), b.populations())
    assert a.tau == b.tau


def test_async_moments_reject_pageable_memory():
    g = rlb.GridParams(nx=6, ny=5, dx=0.1, prec=rlb.RLB_F32, tau0=0.4, dtau=0.0036)
    eps, _, _ = hotspots(6, 5, n=2, seed=3, spread=0.4)
    r = rlb.Run(g)
    r.init_grid(eps)
    host = np.zeros((r.ns, 8))
    rc = r.lib.rlb_moments_async(r._h, host.ctypes.data, None)
    assert rc == RLB_ERR_ARG
    r.moments_wait()  # nothing enqueued: returns at once
