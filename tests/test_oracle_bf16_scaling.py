"""Scaled BF16 storage g = f e^{z0 cosh xi_k} / Z changes nothing for BF16.

BF16 keeps FP32's 8 exponent bits: every population of the hotspot workload
(and its scaled form) is a normal BF16 number, so the relative rounding error
of a stored value is at most 2^-9 whatever the scale, and the moments built
from the stored values inherit errors of the same size.  Checked on an FP64
oracle state of the precision-sweep lattice (16 x 8 x 16): round the
populations to BF16 directly and through the scaled form, and compare the
errors of eps, T and u.  (A scale would matter for a format with a narrow
exponent range, such as FP16.)"""
import numpy as np

from oracle.oracle import Oracle
from paper_1108_5561_gb300.inputs import hotspots


def _bf16(x):
    """Round FP64 values to BF16 (through FP32, nearest even), back to FP64."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def test_bf16_rounding_is_scale_free_on_the_sweep_lattice():
    o = Oracle(nx=8, ny=8, dx=0.1, n_xi=16, n_theta=8, n_phi_half=8, eta_over_s=0.16)
    eps0, _, _ = hotspots(8, 8, n=4, seed=3, spread=0.3)
    f, lnM = o.init_state(eps0)
    o.step(f, lnM, 0.4, 0.0072, 5)
    ref = o.moments(f, lnM)
    c = o.nodes()["c"]
    z0, Z = o.params["z0"], o.params["Z"]
    scale = np.tile(np.exp(z0 * c) / Z, f.shape[1] // c.size)  # node order: k fastest
    plain = _bf16(f)
    scaled = _bf16(f * scale) / scale
    for v in (plain, scaled):
        big = np.abs(f) > 0
        assert np.max(np.abs(v[big] / f[big] - 1)) <= 2.0 ** -8
    assert np.all(np.abs(f[f != 0]) > 1.2e-38) and np.all(np.abs((f * scale)[f != 0]) > 1.2e-38)  # all normal

    def errs(g):
        m = o.moments(g, lnM)
        e = np.abs(m[:, 0] / ref[:, 0] - 1).max()
        t = np.abs(m[:, 1] / ref[:, 1] - 1).max()
        u = (np.abs(m[:, 2:5] - ref[:, 2:5]).max(axis=1) / np.abs(ref[:, 2:5]).max(axis=1)).max()
        return np.array([e, t, u])

    ep, es = errs(plain), errs(scaled)
    assert np.all(ep < 1e-2) and np.all(es < 1e-2)
    # the same size: the scaled form is not more accurate
    assert np.all(es > 0.3 * ep) and np.all(ep > 0.3 * es), (ep, es)
