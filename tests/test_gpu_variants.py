"""Stage-kernel variants (rlb_set_stage_variant).  The packed FP32 kernel with
one or two sites per CTA, with or without its register cap, does the same
per-site arithmetic up to the compiler's fusing of scalar multiply-adds (which
may differ between the instantiations), so the variants agree to FP32
rounding; so do the generic kernel and the mirror-paired kernel (other
operation order: the polar operator on even and odd parts, E_eq from a
reciprocal square root).  Odd row lengths and odd site counts exercise the CTA
whose second site is missing (it repeats the first and stores nothing).  The
halo-staged variant runs the mirror-paired arithmetic on lines read from shared
memory, so on grids it takes (one grid, even nx) it equals variant 5 bit for
bit; elsewhere it runs variant 5."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1108_5561_gb300 as rlb  # noqa: E402
from paper_1108_5561_gb300.inputs import hotspots  # noqa: E402

PACKED = [0, 1, 3, 4]  # one site (capped, uncapped), two sites (capped, uncapped)
GENERIC = 2
MIRROR = [5, 6]  # mirror-paired polar lines (8 x 8 x 12 lattice; 5 the default there), 6 with the staged halo


def _grid(nx, ny, prec=rlb.RLB_F32, **lat):
    return rlb.GridParams(nx=nx, ny=ny, dx=0.1, prec=prec, eta_over_s=0.12, tau0=0.4, dtau=0.0036,
                          n_phi_half=lat.get("n_phi_half", 6), n_xi=lat.get("n_xi", 8))


def _evolve(g, variant, eps, events=None, steps=8):
    r = rlb.Run(g, events=events)
    n = r.set_stage_variant(variant)
    mp = g.n_xi == 8 and g.n_theta == 8 and g.n_phi_half == 6
    assert n == ((7 if g.prec == rlb.RLB_F32 else 6) if mp else 5)
    r.init_grid(eps)
    r.step(steps)
    r.check()
    return r


def _same(a, b, tol=2e-6):
    fa, fb = a.populations().double(), b.populations().double()
    assert float((fa - fb).abs().max() / fa.abs().max()) < tol
    assert float((a.lnM() - b.lnM()).abs().max()) < tol
    ma, mb = a.moments(), b.moments()
    assert np.abs(ma - mb).max() / np.abs(ma).max() < tol


@pytest.mark.parametrize("nx,ny", [(23, 17), (24, 16), (1, 5), (2, 3)])
def test_packed_variants_agree(nx, ny):
    g = _grid(nx, ny)
    eps, _, _ = hotspots(nx, ny, n=4, seed=31 + nx, spread=0.4)
    ref = _evolve(g, 0, eps)
    for v in PACKED[1:]:
        _same(ref, _evolve(g, v, eps))


def test_packed_variants_agree_on_a_batch_with_an_odd_site_count():
    events = [rlb.Event(7, 5, 0.08), rlb.Event(12, 9, 0.2), rlb.Event(4, 3, 0.3)]
    assert sum(e.nx * e.ny for e in events) % 2 == 1
    g = rlb.GridParams(dx=0.1, prec=rlb.RLB_F32, tau0=0.4, dtau=0.0036)
    eps = np.concatenate([hotspots(e.nx, e.ny, n=3, seed=7 + i, spread=0.4)[0].reshape(-1)
                          for i, e in enumerate(events)])
    ref = _evolve(g, 0, eps, events=events)
    for v in PACKED[1:]:
        _same(ref, _evolve(g, v, eps, events=events))


def test_generic_variant_within_fp32_rounding():
    g = _grid(17, 12)
    eps, _, _ = hotspots(17, 12, n=4, seed=5, spread=0.4)
    _same(_evolve(g, 0, eps), _evolve(g, GENERIC, eps), tol=1e-5)


def test_bf16_lattice16_packed_variants_agree():
    g = _grid(9, 7, prec=rlb.RLB_BF16, n_xi=16, n_phi_half=8)
    eps, _, _ = hotspots(9, 7, n=3, seed=2, spread=0.4)
    ref = _evolve(g, 0, eps, steps=4)
    for v in PACKED[1:]:
        _same(ref, _evolve(g, v, eps, steps=4), tol=2e-2)  # BF16 storage: one rounding step apart


@pytest.mark.parametrize("variant", MIRROR)
@pytest.mark.parametrize("nx,ny", [(23, 17), (24, 16), (1, 5), (2, 3), (3, 1)])
def test_mirror_paired_variants_within_fp32_rounding(nx, ny, variant):
    g = _grid(nx, ny)
    eps, _, _ = hotspots(nx, ny, n=4, seed=31 + nx, spread=0.4)
    _same(_evolve(g, 0, eps), _evolve(g, variant, eps), tol=1e-5)


def test_mirror_paired_variant_on_a_grid_larger_than_one_wave():
    # more CTAs than fit on the GPU at once: the L2 prefetch of the CTA one wave
    # ahead reaches real sites, and the last wave's prefetches fall off the end
    g = _grid(160, 150)
    eps, _, _ = hotspots(160, 150, n=20, seed=9, spread=2.0)
    _same(_evolve(g, 0, eps, steps=3), _evolve(g, MIRROR[0], eps, steps=3), tol=1e-5)


@pytest.mark.parametrize("variant", MIRROR)
def test_mirror_paired_variants_on_a_batch_with_an_odd_site_count(variant):
    events = [rlb.Event(7, 5, 0.08), rlb.Event(12, 9, 0.2), rlb.Event(4, 3, 0.3)]
    g = rlb.GridParams(dx=0.1, prec=rlb.RLB_F32, tau0=0.4, dtau=0.0036)
    eps = np.concatenate([hotspots(e.nx, e.ny, n=3, seed=7 + i, spread=0.4)[0].reshape(-1)
                          for i, e in enumerate(events)])
    _same(_evolve(g, 0, eps, events=events), _evolve(g, variant, eps, events=events), tol=1e-5)


@pytest.mark.parametrize("variant", MIRROR)
def test_mirror_paired_variants_bf16_and_minkowski(variant):
    if variant == 5:  # the staged variant takes FP32 storage only
        g = _grid(9, 7, prec=rlb.RLB_BF16)
        eps, _, _ = hotspots(9, 7, n=3, seed=2, spread=0.4)
        _same(_evolve(g, 0, eps, steps=4), _evolve(g, variant, eps, steps=4), tol=2e-2)
    g = rlb.GridParams(nx=6, ny=5, dx=0.1, prec=rlb.RLB_F32, metric=rlb.RLB_MINKOWSKI, eta_over_s=0.12,
                       tau0=1.0, dtau=0.0036)
    eps, _, _ = hotspots(6, 5, n=3, seed=4, spread=0.3)
    _same(_evolve(g, 0, eps), _evolve(g, variant, eps), tol=1e-5)


@pytest.mark.parametrize("nx,ny", [(24, 16), (2, 3), (2, 1), (4, 5), (160, 150)])
def test_staged_halo_equals_mirror_paired_bit_for_bit(nx, ny):
    g = _grid(nx, ny)
    eps, _, _ = hotspots(nx, ny, n=max(4, nx * ny // 1200), seed=17 + nx, spread=0.4 + nx / 80)
    a, b = _evolve(g, 5, eps, steps=4), _evolve(g, 6, eps, steps=4)
    assert torch.equal(a.populations(), b.populations())
    assert torch.equal(a.lnM(), b.lnM())
    assert np.array_equal(a.moments(), b.moments())


def test_staged_halo_minkowski_bit_for_bit():
    g = rlb.GridParams(nx=6, ny=5, dx=0.1, prec=rlb.RLB_F32, metric=rlb.RLB_MINKOWSKI, eta_over_s=0.12,
                       tau0=1.0, dtau=0.0036)
    eps, _, _ = hotspots(6, 5, n=3, seed=4, spread=0.3)
    a, b = _evolve(g, 5, eps), _evolve(g, 6, eps)
    assert torch.equal(a.populations(), b.populations())


def test_set_stage_variant_rejects_unknown_numbers():
    r = rlb.Run(_grid(4, 4))
    assert r.set_stage_variant(-1) == 7
    with pytest.raises(rlb.RLBError):
        r.set_stage_variant(7)
    r = rlb.Run(_grid(4, 4, prec=rlb.RLB_BF16))
    assert r.set_stage_variant(-1) == 6
    with pytest.raises(rlb.RLBError):
        r.set_stage_variant(6)
    r = rlb.Run(_grid(4, 4, n_xi=16, n_phi_half=8))
    assert r.set_stage_variant(-1) == 5
