"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports every
symbol the header declares, and its host-side lattice and operator
construction (Golub-Welsch + Christoffel-Darboux) agrees with the oracle's
independent construction (Stieltjes + bisection, modal Galerkin sums).
No kernel is launched here."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "rlb.h")).read()
    return sorted(set(re.findall(r"^\s*(?:rlb_status|void|const char\*)\s+(rlb_\w+)\s*\(", txt, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1108_5561_gb300 import _lib
    return _lib.load()


def test_exports_every_header_symbol(lib):
    from paper_1108_5561_gb300 import _lib
    syms = header_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(lib, s), s
    assert sorted(_lib.EXPORTS) == syms


def _host_ctx(lib, grid, eos=None):
    from paper_1108_5561_gb300 import EosParams
    h = ctypes.c_void_p()
    assert lib.rlb_create(ctypes.byref(h), 0) == 0
    es = (eos or EosParams(table_points=256)).c_struct()
    assert lib.rlb_init_eos(h, ctypes.byref(es)) == 0, lib.rlb_last_error(h)
    gs = grid.c_struct()
    assert lib.rlb_configure(h, ctypes.byref(gs)) == 0, lib.rlb_last_error(h)
    return h


@pytest.mark.parametrize("shape,z0,fam", [((8, 8, 6), 1.0, 0), ((16, 8, 8), 1.0, 0),
                                          ((5, 5, 1), 1.0, 0), ((6, 4, 3), 1.8281, 0),
                                          ((8, 8, 6), 1.0, 1)])
def test_lattice_and_operators_match_oracle(lib, oracle_mod, shape, z0, fam):
    from paper_1108_5561_gb300 import EosParams, GridParams
    nxi, nth, nph = shape
    eos = EosParams(kind=2 if fam else 0, table_points=256)
    g = GridParams(nx=1, ny=1, n_xi=nxi, n_theta=nth, n_phi_half=nph, z0=z0, family=fam)
    h = _host_ctx(lib, g, eos)
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    c, s, w = np.zeros(nxi), np.zeros(nxi), np.zeros(nxi)
    mu, wt = np.zeros(nth), np.zeros(nth)
    cp, sp = np.zeros(2 * nph), np.zeros(2 * nph)
    assert lib.rlb_lattice(h, dp(c), dp(s), dp(w), dp(mu), dp(wt), dp(cp), dp(sp)) == 0
    Dr, Dth = np.zeros((nxi, nxi)), np.zeros((nth, nth))
    assert lib.rlb_operators(h, dp(Dr), dp(Dth)) == 0
    lib.rlb_destroy(h)
    o = oracle_mod.Oracle(nx=1, ny=1, n_xi=nxi, n_theta=nth, n_phi_half=nph, z0=z0, family=fam,
                          eos_kind=2 if fam else 0)
    nd, ops = o.nodes(), o.operators()
    assert np.allclose(c, nd["c"], rtol=1e-14, atol=0)
    assert np.allclose(s, nd["s"], rtol=1e-13, atol=0)
    assert np.allclose(w, nd["wxi"], rtol=1e-12, atol=0)
    assert np.allclose(mu, nd["mu"], rtol=0, atol=2e-16)
    assert np.allclose(wt, nd["wth"], rtol=1e-14, atol=0)
    assert np.array_equal(cp, nd["cph"]) or np.allclose(cp, nd["cph"], atol=1e-16)
    assert np.allclose(sp, nd["sph"], atol=1e-16)
    scale = lambda A: max(np.abs(A).max(), 1.0)
    assert np.allclose(Dr, ops["Dr"], rtol=0, atol=1e-12 * scale(Dr))
    assert np.allclose(Dth, ops["Dth"], rtol=0, atol=1e-13 * scale(Dth))


def test_invalid_arguments_are_rejected(lib):
    from paper_1108_5561_gb300 import EosParams, GridParams
    h = ctypes.c_void_p()
    assert lib.rlb_create(ctypes.byref(h), 0) == 0
    gs = GridParams().c_struct()
    assert lib.rlb_configure(h, ctypes.byref(gs)) == -5  # EOS first
    bad = EosParams(T_min=1.0, T_max=0.5).c_struct()
    assert lib.rlb_init_eos(h, ctypes.byref(bad)) == -1
    es = EosParams(table_points=256).c_struct()
    assert lib.rlb_init_eos(h, ctypes.byref(es)) == 0
    gs = GridParams(n_xi=7).c_struct()
    assert lib.rlb_configure(h, ctypes.byref(gs)) == -1
    assert b"unsupported" in lib.rlb_last_error(h)
    gs = GridParams(family=1).c_struct()  # Laguerre family needs the conformal EOS
    assert lib.rlb_configure(h, ctypes.byref(gs)) == -1
    gs = GridParams().c_struct()
    assert lib.rlb_configure(h, ctypes.byref(gs)) == 0
    assert lib.rlb_step(h, 1, None) == -5  # before init_grid
    lib.rlb_destroy(h)


def test_later_entry_points_check_their_arguments_on_the_host(lib):
    # argument and state checks that return before any device call
    from paper_1108_5561_gb300 import EosParams, GridParams
    buf = np.zeros(64)
    ptr = buf.ctypes.data_as(ctypes.c_void_p)
    assert lib.rlb_moments_async(None, ptr, None) == -1
    assert lib.rlb_moments_wait(None) == -1
    assert lib.rlb_load_state_async(None, ptr, 64, ctypes.c_double(0.4), None) == -1
    assert lib.rlb_adjoint_step_from(None, ptr, 64, ctypes.c_double(0.4), None) == -1
    expired = ctypes.c_int()
    assert lib.rlb_wait_selftest(0, 1, ctypes.c_double(0.0), ctypes.byref(expired), None) == -1
    assert lib.rlb_wait_selftest(0, 1, ctypes.c_double(5000.0), ctypes.byref(expired), None) == -1
    h = ctypes.c_void_p()
    assert lib.rlb_create(ctypes.byref(h), 0) == 0
    es = EosParams(table_points=256).c_struct()
    assert lib.rlb_init_eos(h, ctypes.byref(es)) == 0
    gs = GridParams().c_struct()
    assert lib.rlb_configure(h, ctypes.byref(gs)) == 0
    assert lib.rlb_moments_async(h, None, None) == -1
    assert lib.rlb_moments_async(h, ptr, None) == -5  # before init_grid
    assert b"init_grid" in lib.rlb_last_error(h)
    assert lib.rlb_moments_wait(h) == 0  # nothing enqueued
    assert lib.rlb_load_state_async(h, ptr, 64, ctypes.c_double(0.4), None) == -5  # no bound buffers
    assert lib.rlb_adjoint_step_from(h, ptr, 64, ctypes.c_double(0.4), None) == -5
    lib.rlb_destroy(h)
