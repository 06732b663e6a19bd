"""Batched events (rlb_configure_batch / rlb_init_batch): every event of a
batch evolves exactly as the same event run alone (bit for bit: same kernels,
same arithmetic, only the site indexing differs), with its own grid size and
eta/s."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1108_5561_gb300 as rlb  # noqa: E402
from paper_1108_5561_gb300.inputs import hotspots  # noqa: E402

EVENTS = [rlb.Event(7, 5, 0.08), rlb.Event(12, 9, 0.2), rlb.Event(4, 11, 0.3), rlb.Event(1, 3, 0.16)]


def _eps(e, i):
    eps, _, _ = hotspots(e.nx, e.ny, n=4, seed=100 + i, spread=0.4)
    return eps


@pytest.mark.parametrize("prec", [rlb.RLB_F64, rlb.RLB_F32, rlb.RLB_BF16])
def test_batch_equals_single_runs(prec):
    g = rlb.GridParams(dx=0.1, prec=prec, tau0=0.4, dtau=0.0036)
    batch = rlb.Run(g, events=EVENTS)
    batch.init_grid(np.concatenate([_eps(e, i).reshape(-1) for i, e in enumerate(EVENTS)]))
    batch.step(12)
    batch.check()
    pb, mb = batch.populations(), batch.moments()
    for i, e in enumerate(EVENTS):
        gi = rlb.GridParams(nx=e.nx, ny=e.ny, dx=0.1, prec=prec, tau0=0.4, dtau=0.0036,
                            eta_over_s=e.eta_over_s)
        one = rlb.Run(gi)
        one.init_grid(_eps(e, i))
        one.step(12)
        o, n = batch.event_offsets[i], e.nx * e.ny
        assert torch.equal(pb[o:o + n], one.populations()), i
        assert np.array_equal(mb[o:o + n], one.moments()), i
        assert one.tau == batch.tau


def test_batch_rejects_bad_events():
    g = rlb.GridParams(prec=rlb.RLB_F32)
    with pytest.raises(rlb.RLBError):
        rlb.Run(g, events=[rlb.Event(0, 4, 0.1)])
    with pytest.raises(rlb.RLBError):
        rlb.Run(g, events=[rlb.Event(4, 4, -1.0)])
