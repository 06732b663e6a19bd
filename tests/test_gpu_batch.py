"""Batched events (rlb_configure_batch / rlb_init_batch): every event of an
uneven batch matches the FP64 oracle run on that event alone with its own grid
and eta/s, and evolves exactly as the same event run alone on the GPU (bit for
bit: same kernels, same arithmetic, only the site indexing differs)."""
import os

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


ORACLE_EVENTS = [rlb.Event(7, 5, 0.04), rlb.Event(12, 9, 0.3), rlb.Event(1, 3, 0.16)]


@pytest.mark.parametrize("prec,tol", [(rlb.RLB_F64, 1e-12), (rlb.RLB_F32, 1e-5)])
def test_batch_events_match_the_oracle(oracle_mod, prec, tol):
    # per event: eps, T relative per site, u as the 4-vector, u_perp against the
    # event's own max |u_perp|
    steps, nt = 20, os.cpu_count() or 1
    g = rlb.GridParams(dx=0.1, prec=prec, tau0=0.4, dtau=0.0036)
    batch = rlb.Run(g, events=ORACLE_EVENTS)
    eps = [hotspots(e.nx, e.ny, n=4, seed=300 + i, spread=0.3)[0] for i, e in enumerate(ORACLE_EVENTS)]
    batch.init_grid(np.concatenate([x.reshape(-1) for x in eps]))
    batch.step(steps)
    batch.check()
    mb = batch.moments()
    for i, e in enumerate(ORACLE_EVENTS):
        o = oracle_mod.Oracle(nx=e.nx, ny=e.ny, dx=0.1, eta_over_s=e.eta_over_s)
        f, lnM = o.init_state(eps[i], nt)
        o.step(f, lnM, 0.4, 0.0036, steps, nt)
        mo = o.moments(f, lnM, nt)
        mg = mb[batch.event_offsets[i]:batch.event_offsets[i] + e.nx * e.ny]
        err = [float(np.max(np.abs(mg[:, c] / mo[:, c] - 1))) for c in (0, 1)]
        err.append(float(np.max(np.abs(mg[:, 2:5] - mo[:, 2:5]).max(axis=1) / np.abs(mo[:, 2:5]).max(axis=1))))
        if e.nx > 1:
            err.append(float(np.abs(mg[:, 3:5] - mo[:, 3:5]).max() / np.abs(mo[:, 3:5]).max()))
        print("event", i, e, ["%.1e" % x for x in err])
        assert max(err) < tol, (i, err)


def test_batch_rejects_bad_events():
    g = rlb.GridParams(prec=rlb.RLB_F32)
    with pytest.raises(rlb.RLBError):
        rlb.Run(g, events=[rlb.Event(0, 4, 0.1)])
    with pytest.raises(rlb.RLBError):
        rlb.Run(g, events=[rlb.Event(4, 4, -1.0)])


@pytest.mark.parametrize("prec", [rlb.RLB_F64, rlb.RLB_F32])
def test_graph_replay_equals_plain_launches(prec):
    g = rlb.GridParams(dx=0.1, prec=prec, tau0=0.4, dtau=0.0036)
    eps = np.concatenate([_eps(e, i).reshape(-1) for i, e in enumerate(EVENTS)])
    runs = []
    for graphs in (True, False):
        r = rlb.Run(g, events=EVENTS)
        r.set_graphs(graphs)
        r.init_grid(eps)
        r.step(5)
        r.step(4)
        runs.append(r)
    torch.cuda.synchronize()
    assert torch.equal(runs[0].populations(), runs[1].populations())
    assert torch.equal(runs[0].lnM(), runs[1].lnM())
    assert runs[0].tau == runs[1].tau


def test_autotune_keeps_state_and_picks_a_variant():
    g = rlb.GridParams(dx=0.1, prec=rlb.RLB_F32, tau0=0.4, dtau=0.0036)
    eps = np.concatenate([_eps(e, i).reshape(-1) for i, e in enumerate(EVENTS)])
    r = rlb.Run(g, events=EVENTS)
    r.init_grid(eps)
    r.step(3)
    before = r.populations().clone()
    tau = r.tau
    chosen, ms = r.autotune()
    assert len(ms) == r.set_stage_variant(-1) == 7 and 0 <= chosen < 6
    # variant 6 (the staged halo) takes one grid only: on a batch it is not timed (-1)
    assert all(t > 0 for t in ms[:6]) and ms[6] == -1.0
    assert ms[chosen] == min(ms[:6])
    assert torch.equal(before, r.populations()) and r.tau == tau
    r.step(3)  # steps with the chosen variant stay within FP32 parity of the default one
    ref = rlb.Run(g, events=EVENTS)
    ref.init_grid(eps)
    ref.step(6)
    d = np.abs(r.moments()[:, 0] / ref.moments()[:, 0] - 1).max()
    assert d < 1e-5, d
