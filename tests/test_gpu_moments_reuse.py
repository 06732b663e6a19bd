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
