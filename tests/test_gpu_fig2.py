"""Fig. 2 protocol (Sec. 4.5) on the GPU: 0+1D Bjorken flow, N_xi = N_theta = 5,
dtau = 0.2 fm/c, synthetic crossover EOS.  The lattice Boltzmann temperature
follows second-order viscous hydrodynamics within a few percent for eta/s = 0.08
and 0.5 (the paper: "reasonably well"; the hydrodynamic transport coefficients
are the massless-gas ones, so exact agreement is not expected), and the less
the collisions, the slower the cooling (the longitudinal pressure drops with
growing eta/s; free streaming keeps the warmest medium)."""
import math
import os
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import fig2_protocol as F  # noqa: E402


def test_fig2_protocol(oracle_mod):
    rows = F.table()
    for etas, tol in ((0.08, 0.03), (0.5, 0.05)):
        taus, T_lb, T_vh = rows[etas]
        dev = np.abs(T_lb / T_vh - 1)
        print("eta/s", etas, "max |LB/VH - 1|", dev.max(), "at tau", taus[np.argmax(dev)])
        assert dev.max() < tol, (etas, dev.max())
        assert T_lb[-1] < 0.18 < T_lb[0]  # the run reaches the crossover (the EOS slows the cooling there)
    t_fs = rows[math.inf][1]
    assert np.all(np.diff(t_fs) < 0)
    assert t_fs[-1] > rows[0.5][1][-1] > rows[0.08][1][-1]
