"""Thin Python front end of the C ABI (include/rlb.h).

Every computation happens in the CUDA library; this module only marshals
arguments.  PyTorch provides the device memory (the library borrows it) and the
CUDA stream.  There is no CPU fallback: constructing a run without a CUDA
device or without the compiled library raises.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass, field

import numpy as np

from . import _lib as L

HBARC = 0.1973269804  # GeV fm
Z_QCD = math.pi ** 4 / 180.0 * (4 * (3 * 3 - 1) + 7 * 3 * 3)  # Sec. 3.1, N_c = N_f = 3


@dataclass
class EosParams:
    """Equation of state (Sec. 3.1); kind: 0 crossover s/T^3, 1 constant mass, 2 conformal."""
    kind: int = L.RLB_EOS_CROSSOVER
    a: float = 13.9
    b: float = 0.5
    Tc: float = 0.17
    w: float = 0.02
    m0: float = 0.5
    Z: float = Z_QCD
    T_min: float = 0.01
    T_max: float = 4.0
    table_points: int = 0

    def c_struct(self):
        return L.EosParamsC(self.kind, self.table_points, self.a, self.b, self.Tc, self.w,
                            self.m0, self.Z, self.T_min, self.T_max)


@dataclass
class GridParams:
    nx: int = 32
    ny: int = 32
    dx: float = 0.2
    metric: int = L.RLB_MILNE
    n_xi: int = 8
    n_theta: int = 8
    n_phi_half: int = 6
    family: int = L.RLB_RADIAL_PAPER
    z0: float = 1.0
    T0: float = 0.3
    prec: int = L.RLB_F64
    eta_over_s: float = 0.08
    tau0: float = 0.4
    dtau: float = 0.018

    @property
    def nodes(self) -> int:
        return self.n_xi * self.n_theta * 2 * self.n_phi_half

    def c_struct(self):
        return L.GridParamsC(self.nx, self.ny, self.metric, self.n_xi, self.n_theta,
                             self.n_phi_half, self.family, self.prec, self.dx, self.z0, self.T0,
                             self.eta_over_s, self.tau0, self.dtau)


_TORCH_DT = {L.RLB_F64: "float64", L.RLB_F32: "float32", L.RLB_BF16: "bfloat16"}


@dataclass
class Event:
    """One event of a batch: its own periodic nx x ny grid and eta/s."""
    nx: int
    ny: int
    eta_over_s: float


def alu_peaks(device: int = 0) -> dict:
    """Measured FP32 (FFMA), packed FP32 (FFMA2) and FP64 multiply-add rates of
    the device in TFLOP/s (rlb_alu_peaks)."""
    out = np.zeros(3)
    lib = L.load()
    rc = lib.rlb_alu_peaks(int(device), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != 0:
        raise L.RLBError(rc, "rlb_alu_peaks")
    return {"fp32_ffma_tflops": float(out[0]), "fp32_ffma2_tflops": float(out[1]),
            "fp64_dfma_tflops": float(out[2])}


def wait_selftest(device: int = 0, deliver: bool = True, limit_ms: float = 50.0):
    """The staging wait of stage variant 6 on its own (rlb_wait_selftest):
    (expired, value); value is 1.25 when the copy was delivered."""
    lib = L.load()
    e, v = ctypes.c_int(-1), ctypes.c_float(0.0)
    rc = lib.rlb_wait_selftest(int(device), int(bool(deliver)), float(limit_ms), ctypes.byref(e), ctypes.byref(v))
    if rc != 0:
        raise L.RLBError(rc, "rlb_wait_selftest")
    return bool(e.value), float(v.value)


class Run:
    """One simulation on one GPU: EOS table, grid (or batch of events), device
    buffers, state.  With `events`, the grid's lattice, precision, dx, tau0,
    dtau and metric are shared by all events and its nx, ny, eta/s are unused."""

    def __init__(self, grid: GridParams, eos: EosParams | None = None, device: int = 0,
                 events: list[Event] | None = None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("the lattice Boltzmann step runs on a CUDA device; none is available")
        self.torch = torch
        self.grid = grid
        self.eos = eos or EosParams()
        self.device = torch.device("cuda", device)
        self.lib = L.load()
        h = ctypes.c_void_p()
        self._chk(self.lib.rlb_create(ctypes.byref(h), device), "rlb_create", h0=True)
        self._h = h
        gs, es = grid.c_struct(), self.eos.c_struct()
        self._gs = gs
        self._chk(self.lib.rlb_init_eos(self._h, ctypes.byref(es)), "rlb_init_eos")
        self.events = list(events) if events else None
        if self.events:
            arr = (L.EventDescC * len(self.events))(*[L.EventDescC(e.nx, e.ny, e.eta_over_s)
                                                       for e in self.events])
            self._chk(self.lib.rlb_configure_batch(self._h, ctypes.byref(gs), len(self.events), arr),
                      "rlb_configure_batch")
        else:
            self._chk(self.lib.rlb_configure(self._h, ctypes.byref(gs)), "rlb_configure")
        sb, xb = ctypes.c_size_t(), ctypes.c_size_t()
        self._chk(self.lib.rlb_workspace_size(self._h, None, ctypes.byref(sb), ctypes.byref(xb)),
                  "rlb_workspace_size")
        self.state = torch.empty(sb.value, dtype=torch.uint8, device=self.device)
        self.scratch = torch.empty(xb.value, dtype=torch.uint8, device=self.device)
        self._chk(self.lib.rlb_bind_buffers(self._h, ctypes.c_void_p(self.state.data_ptr()),
                                            ctypes.c_void_p(self.scratch.data_ptr()), self._stream()),
                  "rlb_bind_buffers")
        fo, mo, pb = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
        self._chk(self.lib.rlb_state_offsets(self._h, ctypes.byref(fo), ctypes.byref(mo),
                                             ctypes.byref(pb)), "rlb_state_offsets")
        self._f_off, self._m_off, self.pop_bytes = fo.value, mo.value, pb.value
        self.ns = sum(e.nx * e.ny for e in self.events) if self.events else grid.nx * grid.ny
        self.nn = grid.nodes
        # first site of every event (batch) or [0]
        offs = [0]
        for e in (self.events or []):
            offs.append(offs[-1] + e.nx * e.ny)
        self.event_offsets = offs[:-1] if self.events else [0]

    # -- helpers --------------------------------------------------------------
    def _stream(self):
        return ctypes.c_void_p(self.torch.cuda.current_stream(self.device).cuda_stream)

    def _chk(self, rc, what, h0=False):
        if rc != 0:
            msg = what
            if not h0 and getattr(self, "_h", None) is not None:
                msg += ": " + self.lib.rlb_last_error(self._h).decode()
            raise L.RLBError(rc, msg)

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self.lib.rlb_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- API ------------------------------------------------------------------
    def init_grid(self, eps0):
        """Local equilibrium at rest with energy density eps0 [GeV/fm^3], shape (ny, nx)."""
        torch = self.torch
        if isinstance(eps0, torch.Tensor) and eps0.is_cuda:
            e = eps0.to(torch.float64).contiguous().reshape(-1)
            assert e.numel() == self.ns
            ptr = ctypes.cast(ctypes.c_void_p(e.data_ptr()), ctypes.POINTER(ctypes.c_double))
            self._chk(self.lib.rlb_init_grid(self._h, ptr, 1, self._stream()), "rlb_init_grid")
            self._keep = e
        else:
            e = np.ascontiguousarray(np.asarray(eps0, dtype=np.float64).reshape(-1))
            assert e.size == self.ns
            ptr = e.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            self._chk(self.lib.rlb_init_grid(self._h, ptr, 0, self._stream()), "rlb_init_grid")

    def step(self, nsteps: int = 1):
        self._chk(self.lib.rlb_step(self._h, int(nsteps), self._stream()), "rlb_step")

    @property
    def tau(self) -> float:
        t = ctypes.c_double()
        self._chk(self.lib.rlb_get_tau(self._h, ctypes.byref(t)), "rlb_get_tau")
        return t.value

    def check(self):
        self._chk(self.lib.rlb_check(self._h, self._stream()), "rlb_check")

    def moments_async(self, out):
        """Per-site observables into `out`, a page-locked host float64 tensor
        (sites x 8), downloaded while the next steps run (rlb_moments_async);
        read it after moments_wait()."""
        torch = self.torch
        assert isinstance(out, torch.Tensor) and out.dtype == torch.float64 and out.is_pinned()
        assert out.numel() == self.ns * 8 and out.is_contiguous()
        self._chk(self.lib.rlb_moments_async(self._h, ctypes.c_void_p(out.data_ptr()), self._stream()),
                  "rlb_moments_async")

    def moments_wait(self):
        self._chk(self.lib.rlb_moments_wait(self._h), "rlb_moments_wait")

    def moments(self, out=None, host: bool = True):
        """Per-site (eps, T, u^tau, u^x, u^y, M, P_L, M(T)); numpy (host) or a device tensor."""
        torch = self.torch
        if host:
            arr = np.empty((self.ns, 8)) if out is None else out
            ptr = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            self._chk(self.lib.rlb_moments(self._h, ptr, 0, self._stream()), "rlb_moments")
            return arr
        t = torch.empty((self.ns, 8), dtype=torch.float64, device=self.device) if out is None else out
        ptr = ctypes.cast(ctypes.c_void_p(t.data_ptr()), ctypes.POINTER(ctypes.c_double))
        self._chk(self.lib.rlb_moments(self._h, ptr, 1, self._stream()), "rlb_moments")
        return t

    def observables(self):
        """(eps_p, v2 weighted by p_perp) of the current state (synchronises)."""
        a, b = ctypes.c_double(), ctypes.c_double()
        self._chk(self.lib.rlb_observables(self._h, ctypes.byref(a), ctypes.byref(b), self._stream()),
                  "rlb_observables")
        return a.value, b.value

    def state_blob_size(self) -> int:
        n = ctypes.c_size_t()
        self._chk(self.lib.rlb_state_blob_size(self._h, ctypes.byref(n)), "rlb_state_blob_size")
        return n.value

    def save_state(self, device: bool = False):
        """Checkpoint blob of the current state: host bytes, or a CUDA uint8 tensor
        (filled in stream order; it carries the tau it was saved at, so that
        load_state restores it without reading its header back)."""
        n = ctypes.c_size_t(self.state_blob_size())
        if device:
            t = self.torch.empty(n.value, dtype=self.torch.uint8, device=self.device)
            self._chk(self.lib.rlb_save_state(self._h, ctypes.c_void_p(t.data_ptr()), n, self._stream()),
                      "rlb_save_state")
            t._rlb_saved = (self._h.value, self.tau)
            return t
        buf = ctypes.create_string_buffer(n.value)
        self._chk(self.lib.rlb_save_state(self._h, buf, n, self._stream()), "rlb_save_state")
        return buf.raw

    def load_state(self, blob):
        """Replace the state (and tau) by a blob from save_state of the same grid."""
        if isinstance(blob, self.torch.Tensor):
            saved = getattr(blob, "_rlb_saved", None)
            if saved is not None and saved[0] == self._h.value and blob.is_cuda:  # written by this context
                self._chk(self.lib.rlb_load_state_async(self._h, ctypes.c_void_p(blob.data_ptr()), blob.numel(),
                                                        ctypes.c_double(saved[1]), self._stream()),
                          "rlb_load_state_async")
                return
            self._chk(self.lib.rlb_load_state(self._h, ctypes.c_void_p(blob.data_ptr()), blob.numel(),
                                              self._stream()), "rlb_load_state")
            return
        buf = ctypes.create_string_buffer(blob, len(blob))
        self._chk(self.lib.rlb_load_state(self._h, buf, len(blob), self._stream()), "rlb_load_state")

    def populations(self):
        """Device view (ns, nodes) of f in the storage precision (aliases the state buffer)."""
        torch = self.torch
        dt = getattr(torch, _TORCH_DT[self.grid.prec])
        nbytes = self.ns * self.nn * self.pop_bytes
        return self.state[self._f_off:self._f_off + nbytes].view(dt).view(self.ns, self.nn)

    def lnM(self):
        return self.state[self._m_off:self._m_off + 8 * self.ns].view(self.torch.float64)

    def autotune(self):
        """Time the stage-kernel variants on the current state and keep the fastest.
        Returns (chosen variant, [ms per launch of each variant])."""
        c, n = ctypes.c_int(), ctypes.c_int()
        ms = np.zeros(8)  # RLB_MAX_STAGE_VARIANTS
        self._chk(self.lib.rlb_autotune(self._h, self._stream(), ctypes.byref(c),
                                        ms.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        ctypes.byref(n)), "rlb_autotune")
        return c.value, [float(x) for x in ms[:n.value]]

    def set_stage_variant(self, variant: int) -> int:
        """Use stage-kernel variant `variant` (rlb_autotune's numbering) from now
        on; variant < 0 only asks.  Returns the number of variants."""
        n = ctypes.c_int()
        self._chk(self.lib.rlb_set_stage_variant(self._h, int(variant), ctypes.byref(n)),
                  "rlb_set_stage_variant")
        return n.value

    def set_graphs(self, enable: bool = True):
        self._chk(self.lib.rlb_set_graphs(self._h, int(enable)), "rlb_set_graphs")

    def set_timing(self, enable: bool = True):
        self._chk(self.lib.rlb_set_timing(self._h, int(enable)), "rlb_set_timing")

    def timing(self):
        """(stage ms, stage launches, match ms, match launches) since timing was enabled."""
        a, b, c, d = ctypes.c_double(), ctypes.c_long(), ctypes.c_double(), ctypes.c_long()
        self._chk(self.lib.rlb_get_timing(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                          ctypes.byref(d)), "rlb_get_timing")
        return a.value, b.value, c.value, d.value

    def lattice(self):
        g = self.grid
        n1, n2, n3 = g.n_xi, g.n_theta, 2 * g.n_phi_half
        arrs = [np.zeros(n1), np.zeros(n1), np.zeros(n1), np.zeros(n2), np.zeros(n2),
                np.zeros(n3), np.zeros(n3)]
        self._chk(self.lib.rlb_lattice(self._h, *[a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
                                                   for a in arrs]), "rlb_lattice")
        return dict(zip(["c", "s", "wxi", "mu", "wth", "cph", "sph"], arrs))
