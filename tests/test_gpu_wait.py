"""The bounded wait of the halo-staged stage kernel (variant 6), tested
without a GPU fault: the staging mbarrier with its copy delivered completes;
with the copy withheld the wait runs out after its limit, the kernel reports
it, and the context stays usable (a step runs afterwards)."""
import time

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1108_5561_gb300 as rlb  # noqa: E402
from paper_1108_5561_gb300.inputs import hotspots  # noqa: E402


def test_delivered_copy_completes_the_wait():
    expired, value = rlb.wait_selftest(0, deliver=True, limit_ms=200.0)
    assert not expired and value == 1.25


def test_withheld_copy_expires_and_the_device_stays_usable():
    t0 = time.perf_counter()
    expired, _ = rlb.wait_selftest(0, deliver=False, limit_ms=20.0)
    dt = time.perf_counter() - t0
    assert expired
    assert dt < 5.0
    g = rlb.GridParams(nx=8, ny=6, dx=0.1, prec=rlb.RLB_F32, eta_over_s=0.16, tau0=0.4, dtau=0.0036)
    r = rlb.Run(g)
    r.set_stage_variant(6)
    r.init_grid(hotspots(8, 6, n=3, seed=1, spread=0.3)[0])
    r.step(2)
    r.check()


def test_wait_limit_is_bounded_by_the_api():
    with pytest.raises(rlb.RLBError):
        rlb.wait_selftest(0, deliver=False, limit_ms=5000.0)
