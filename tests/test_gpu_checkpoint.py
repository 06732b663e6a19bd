"""Checkpoint and restart through rlb_save_state / rlb_load_state: a run
restarted from a blob continues bit for bit like the uninterrupted run; blobs of
another grid or truncated blobs are rejected on the host."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1108_5561_gb300 as rlb  # noqa: E402
from paper_1108_5561_gb300.inputs import hotspots  # noqa: E402


@pytest.mark.parametrize("prec", [rlb.RLB_F64, rlb.RLB_F32, rlb.RLB_BF16])
def test_restart_is_bit_identical(prec):
    g = rlb.GridParams(nx=16, ny=12, dx=0.1, prec=prec, eta_over_s=0.16, tau0=0.4, dtau=0.0036)
    eps0, _, _ = hotspots(16, 12, n=6, seed=9, spread=0.5)
    a = rlb.Run(g)
    a.init_grid(eps0)
    a.step(5)
    blob = a.save_state()
    a.step(7)
    b = rlb.Run(g)
    b.load_state(blob)
    assert b.tau == pytest.approx(0.4 + 5 * 0.0036, abs=1e-15)
    b.step(7)
    torch.cuda.synchronize()
    assert torch.equal(a.populations(), b.populations())
    assert torch.equal(a.lnM(), b.lnM())
    assert a.tau == b.tau
    assert np.array_equal(a.moments(), b.moments())


def test_foreign_and_truncated_blobs_are_rejected():
    g = rlb.GridParams(nx=6, ny=5, prec=rlb.RLB_F32)
    a = rlb.Run(g)
    a.init_grid(np.full((5, 6), 4.0))
    blob = a.save_state()
    other = rlb.Run(rlb.GridParams(nx=5, ny=6, prec=rlb.RLB_F32))
    with pytest.raises(rlb.RLBError, match="another grid"):
        other.load_state(blob)
    with pytest.raises(rlb.RLBError, match="truncated"):
        a.load_state(blob[: len(blob) // 2])
    with pytest.raises(rlb.RLBError, match="not a state blob"):
        a.load_state(b"x" * len(blob))
