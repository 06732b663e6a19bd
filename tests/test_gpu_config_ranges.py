"""The stated time ranges of the workloads: tau from 0.4 to 4 fm/c in the
stated number of steps at dx = 0.1 fm (a batch of events with dtau = 0.018
(200 steps), the adjoint workload's 128 x 128 grid with dtau = 0.012 (300
steps)), within the streaming stability limit; the runs complete without a
device error and keep a physical state (temperatures above the floor, flow
below the speed of light).  The per-step cost does not depend on dtau: the
benchmarks time these steps."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1108_5561_gb300 as rlb  # noqa: E402
from paper_1108_5561_gb300.inputs import batch_events, hotspots  # noqa: E402


def _physical(m):
    assert np.all(np.isfinite(m))
    assert m[:, 1].min() > 0.1 and m[:, 1].max() < 0.5  # T in GeV
    assert np.abs(m[:, 3:5]).max() < 0.9


def test_batch_events_over_the_stated_range():
    evs = batch_events(512, seed=1108)[:24]
    events = [rlb.Event(n, n, eta) for n, eta in evs]
    eps = np.concatenate([hotspots(n, n, n=40, seed=1108 + i)[0].reshape(-1) for i, (n, _) in enumerate(evs)])
    r = rlb.Run(rlb.GridParams(dx=0.1, prec=rlb.RLB_F32, tau0=0.4, dtau=3.6 / 200), events=events)
    r.init_grid(eps)
    r.step(200)
    r.check()
    assert abs(r.tau - 4.0) < 1e-9
    _physical(r.moments())


def test_adjoint_workload_over_the_stated_range():
    r = rlb.Run(rlb.GridParams(nx=128, ny=128, dx=0.1, prec=rlb.RLB_F32, eta_over_s=0.08, tau0=0.4,
                               dtau=3.6 / 300))
    r.init_grid(hotspots(128, 128, n=40, seed=1108)[0])
    r.step(300)
    r.check()
    assert abs(r.tau - 4.0) < 1e-9
    _physical(r.moments())
