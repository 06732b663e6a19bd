"""The allocation-free step variant (rlb_step_static_scratch) against the
regular step (rlb_step with caller-bound buffers): the same initial state,
advanced by two calls in a row through each entry point, must agree within the
FP64 parity tolerance.  Collected last on purpose: if it fails, every other
test has already run."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1108_5561_gb300 as rlb  # noqa: E402
from paper_1108_5561_gb300 import _lib  # noqa: E402
from paper_1108_5561_gb300.inputs import hotspots  # noqa: E402


def _bare_ctx(lib, g, eos):
    """A context with EOS and grid configured but no device buffers bound."""
    h = ctypes.c_void_p()
    assert lib.rlb_create(ctypes.byref(h), 0) == 0
    es, gs = eos.c_struct(), g.c_struct()
    assert lib.rlb_init_eos(h, ctypes.byref(es)) == 0, lib.rlb_last_error(h)
    assert lib.rlb_configure(h, ctypes.byref(gs)) == 0, lib.rlb_last_error(h)
    return h


@pytest.mark.parametrize("prec,tol", [(rlb.RLB_F64, 1e-12), (rlb.RLB_F32, 1e-5)])
def test_static_scratch_step_matches_bound_step(prec, tol):
    lib = _lib.load()
    g = rlb.GridParams(nx=12, ny=10, dx=0.1, prec=prec, eta_over_s=0.16, tau0=0.4, dtau=0.0036)
    eos = rlb.EosParams()
    eps0, _, _ = hotspots(12, 10, n=6, seed=21, spread=0.3)
    ref = rlb.Run(g, eos)
    ref.init_grid(eps0)
    torch.cuda.synchronize()
    state = ref.state.clone()  # the caller's own state buffer, same layout
    h = _bare_ctx(lib, g, eos)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    try:
        for _ in range(2):  # two calls in a row through each entry point
            ref.step(3)
            rc = lib.rlb_step_static_scratch(h, ctypes.c_void_p(state.data_ptr()), 3, stream)
            assert rc == 0, lib.rlb_last_error(h)
            torch.cuda.synchronize()
            ref.check()
            fo, mo = ref._f_off, ref._m_off
            nbytes = ref.ns * ref.nn * ref.pop_bytes
            dt = ref.populations().dtype
            fa = ref.populations().double().cpu().numpy()
            fb = state[fo:fo + nbytes].view(dt).double().cpu().numpy().reshape(fa.shape)
            la = ref.lnM().cpu().numpy()
            lb = state[mo:mo + 8 * ref.ns].view(torch.float64).cpu().numpy()
            big = np.abs(fa) > 1e-8 * np.abs(fa).max()
            assert np.max(np.abs(fb[big] / fa[big] - 1)) < tol
            assert np.max(np.abs(lb - la)) < tol
        t = ctypes.c_double()
        assert lib.rlb_get_tau(h, ctypes.byref(t)) == 0
        assert t.value == pytest.approx(ref.tau, rel=1e-14)
    finally:
        lib.rlb_destroy(h)


def test_static_scratch_rejects_oversized_grid():
    lib = _lib.load()
    g = rlb.GridParams(nx=256, ny=256, dx=0.1, prec=rlb.RLB_F32)
    h = _bare_ctx(lib, g, rlb.EosParams())
    try:
        buf = torch.empty(256, dtype=torch.uint8, device="cuda")
        rc = lib.rlb_step_static_scratch(h, ctypes.c_void_p(buf.data_ptr()), 1, None)
        assert rc == _lib.RLB_ERR_ARG
        assert b"static scratch" in lib.rlb_last_error(h)
    finally:
        lib.rlb_destroy(h)
