"""The library built with device-side range checks (RLB_CHECKS, loaded with
RLB_CHECKED=1): every site index and grid coordinate the kernels derive is
checked, and every stored population for finiteness, on the paths the
benchmarks and the tests use (one- and two-site packed kernels on odd grids and
an odd-sized batch, the generic FP64 kernel, the BF16 2048-node lattice, the
FP64 and FP32 adjoints).  No check may fire, and the results must equal those
of the release library."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
import paper_1108_5561_gb300 as rlb
from paper_1108_5561_gb300 import adjoint as ADJ
from paper_1108_5561_gb300.inputs import hotspots, hotspot_basis

out = {}
def record(name, run):
    run.check()
    f = run.populations().double()
    out[name] = [float(f.sum()), float(f.abs().sum()), float(run.lnM().sum())]

for v in range(7):
    g = rlb.GridParams(nx=23, ny=17, dx=0.1, prec=rlb.RLB_F32, eta_over_s=0.16, tau0=0.4, dtau=0.0036)
    r = rlb.Run(g)
    r.set_stage_variant(v)
    r.init_grid(hotspots(23, 17, n=6, seed=3, spread=0.5)[0])
    r.step(6)
    record("fp32 variant %d" % v, r)
events = [rlb.Event(7, 5, 0.08), rlb.Event(12, 9, 0.2), rlb.Event(4, 3, 0.3)]
for v in (0, 3, 5, 6):
    g = rlb.GridParams(dx=0.1, prec=rlb.RLB_F32, tau0=0.4, dtau=0.0036)
    r = rlb.Run(g, events=events)
    r.set_stage_variant(v)
    r.init_grid(np.concatenate([hotspots(e.nx, e.ny, n=3, seed=7 + i, spread=0.4)[0].reshape(-1)
                                for i, e in enumerate(events)]))
    r.step(5)
    record("batch variant %d" % v, r)
g = rlb.GridParams(nx=9, ny=6, dx=0.2, prec=rlb.RLB_F64, eta_over_s=0.1, tau0=0.4, dtau=0.018)
r = rlb.Run(g)
r.init_grid(hotspots(9, 6, dx=0.2, n=4, seed=9, spread=0.6)[0])
r.step(5)
record("fp64", r)
g = rlb.GridParams(nx=9, ny=7, dx=0.1, prec=rlb.RLB_BF16, eta_over_s=0.16, tau0=0.4, dtau=0.0036,
                   n_xi=16, n_phi_half=8)
r = rlb.Run(g)
r.init_grid(hotspots(9, 7, n=3, seed=2, spread=0.4)[0])
r.step(3)
record("bf16 lattice16", r)
_, amps, cen = hotspots(8, 7, dx=0.1, n=3, seed=5, spread=0.25, mean_amp=15.0)
basis = hotspot_basis(8, 7, cen, dx=0.1)
for arith in (rlb.RLB_F64, rlb.RLB_F32):
    g = rlb.GridParams(nx=8, ny=7, dx=0.1, prec=rlb.RLB_F32, eta_over_s=0.16, tau0=0.4, dtau=0.0036)
    r = rlb.Run(g)
    e0 = torch.as_tensor(10.0 + amps @ basis, dtype=torch.float64, device="cuda")
    v2, gA, geta = ADJ.v2_gradient(r, e0, torch.as_tensor(basis, device="cuda"), 4, 2, arithmetic=arith)
    r.check()
    out["adjoint %d" % arith] = [float(v2)] + [float(x) for x in gA] + [float(geta)]
print(json.dumps(out))
"""


def _run(checked: bool):
    env = dict(os.environ, RLB_CHECKED="1" if checked else "0")
    p = subprocess.run([sys.executable, "-c", CASES, ROOT], env=env, capture_output=True, text=True,
                       timeout=600)
    assert p.returncode == 0, p.stderr[-3000:]
    return json.loads(p.stdout.strip().splitlines()[-1])


def test_checked_build_fires_no_check_and_changes_nothing():
    from paper_1108_5561_gb300 import build as B
    assert os.path.exists(B.LIB_CHECKED), "build() makes the checked library too"
    checked, release = _run(True), _run(False)
    assert checked.keys() == release.keys()
    for k in release:
        a, b = np.array(checked[k]), np.array(release[k])
        # the same arithmetic; the compiler may fuse a few scalar multiply-adds
        # differently around the extra checks: FP32-level agreement
        assert np.allclose(a, b, rtol=1e-5, atol=0), (k, a, b)
