"""ctypes binding of the FP64 CPU oracle (``oracle/rlb_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The product path never imports it.

The oracle computes, in plain FP64 with sequential sums, one Heun time step of
the relativistic lattice Boltzmann scheme with a quasiparticle equation of
state (Romatschke, arXiv:1108.5561, Sec. 3-4).  State layout (shared by
definition with the public C header, not by code): populations ``f[site][node]``
with ``site = y*nx + x`` and ``node = (l*n_theta + j)*n_xi + k``
(k radial, j polar, l azimuthal), plus one ``ln M`` per site.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rlb_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
# the same source in complex arithmetic (complex-step derivatives, TangentOracle)
_LIB_CS = os.path.join(_HERE, "_build", "liboracle_cs.so")

HBARC = 0.1973269804  # GeV fm
Z_QCD = math.pi ** 4 / 180.0 * (4 * (3 * 3 - 1) + 7 * 3 * 3)  # Sec. 3.1, N_c = N_f = 3


class OracleParams(ctypes.Structure):
    _fields_ = [
        ("eos_kind", ctypes.c_int),
        ("family", ctypes.c_int),
        ("metric", ctypes.c_int),
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("n_xi", ctypes.c_int),
        ("n_theta", ctypes.c_int),
        ("n_phi_half", ctypes.c_int),
        ("pad_", ctypes.c_int),
        ("eos_a", ctypes.c_double),
        ("eos_b", ctypes.c_double),
        ("eos_Tc", ctypes.c_double),
        ("eos_w", ctypes.c_double),
        ("eos_m0", ctypes.c_double),
        ("Z", ctypes.c_double),
        ("z0", ctypes.c_double),
        ("T0", ctypes.c_double),
        ("dx", ctypes.c_double),
        ("eta_over_s", ctypes.c_double),
        ("eta_over_s_im", ctypes.c_double),
    ]


DEFAULTS = dict(
    eos_kind=0, family=0, metric=1, nx=32, ny=32, n_xi=8, n_theta=8, n_phi_half=6,
    eos_a=13.9, eos_b=0.5, eos_Tc=0.17, eos_w=0.02, eos_m0=0.5, Z=Z_QCD,
    z0=1.0, T0=0.3, dx=0.2, eta_over_s=0.08, eta_over_s_im=0.0,
)


def build(force: bool = False) -> str:
    """Compile the oracle shared libraries with gcc (-O2, OpenMP): the FP64
    oracle and the same source in complex arithmetic (-DOR_COMPLEX_STEP;
    -fcx-limited-range: plain complex products and quotients, the operands
    are finite)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    for lib, extra in ((_LIB, []), (_LIB_CS, ["-DOR_COMPLEX_STEP", "-fcx-limited-range"])):
        if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
            tmp = lib + ".tmp%d" % os.getpid()
            cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", *extra, "-o", tmp, _SRC, "-lm"]
            subprocess.check_call(cmd)
            os.replace(tmp, lib)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        d = ctypes.c_double
        dp = P(ctypes.c_double)
        ip = P(ctypes.c_int)
        vp = ctypes.c_void_p
        lib.or_create.argtypes = [P(OracleParams), P(vp)]
        lib.or_destroy.argtypes = [vp]
        lib.or_destroy.restype = None
        lib.or_num_nodes.argtypes = [vp]
        lib.or_nodes.argtypes = [vp] + [dp] * 9
        lib.or_operators.argtypes = [vp, dp, dp, dp, dp]
        lib.or_eos.argtypes = [vp, d, dp]
        lib.or_solve_T.argtypes = [vp, d, ctypes.c_int, dp]
        lib.or_landau.argtypes = [dp, dp, dp]
        lib.or_bessel.argtypes = [d, dp]
        lib.or_step.argtypes = [vp, dp, dp, d, d, ctypes.c_int, ctypes.c_int]
        lib.or_rhs.argtypes = [vp, dp, dp, d, dp, dp, ctypes.c_int]
        lib.or_moments.argtypes = [vp, dp, dp, dp, ctypes.c_int]
        lib.or_observables.argtypes = [vp, dp, dp, dp, ctypes.c_int]
        lib.or_init_state.argtypes = [vp, dp, dp, dp, ctypes.c_int]
        lib.or_step_sites.argtypes = [vp, dp, dp, d, d, ip, ctypes.c_int, dp, dp, ctypes.c_int]
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc, what):
    if rc != 0:
        raise RuntimeError("oracle %s failed with status %d" % (what, rc))


def bessel_k(x: float) -> np.ndarray:
    """K_0..K_3 at x from the oracle's integral representation."""
    out = np.zeros(4)
    _check(_load().or_bessel(float(x), _dp(out)), "bessel")
    return out


def landau(Tmunu: np.ndarray):
    """Timelike eigenvector u^mu and eigenvalue eps of T^mu_nu (4x4, upper indices)."""
    T = np.ascontiguousarray(Tmunu, dtype=np.float64).reshape(16)
    u = np.zeros(4)
    e = ctypes.c_double()
    _check(_load().or_landau(_dp(T), _dp(u), ctypes.byref(e)), "landau")
    return u, e.value


EOS_FIELDS = ["x", "M", "s", "sp", "pkin", "e", "ep", "Bp", "D", "J", "tauR", "p", "B", "eps",
              "K1", "K2"]


class Oracle:
    """One oracle context (parameters, momentum lattice, operators)."""

    def __init__(self, **kw):
        p = dict(DEFAULTS)
        unknown = set(kw) - set(p)
        if unknown:
            raise TypeError("unknown oracle parameters: %s" % sorted(unknown))
        p.update(kw)
        self.params = p
        self._p = OracleParams(**{k: p[k] for k in p})
        self._lib = _load()
        h = ctypes.c_void_p()
        _check(self._lib.or_create(ctypes.byref(self._p), ctypes.byref(h)), "create")
        self._h = h
        self.nn = self._lib.or_num_nodes(self._h)
        self.ns = p["nx"] * p["ny"]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.or_destroy(h)
            self._h = None

    # -- lattice and operators ------------------------------------------------
    def nodes(self):
        p = self.params
        nxi, nth, nph = p["n_xi"], p["n_theta"], 2 * p["n_phi_half"]
        arrs = [np.zeros(nxi) for _ in range(4)] + [np.zeros(nth) for _ in range(3)] + \
               [np.zeros(nph) for _ in range(2)]
        _check(self._lib.or_nodes(self._h, *[_dp(a) for a in arrs]), "nodes")
        names = ["c", "s", "wxi", "ecw", "mu", "sth", "wth", "cph", "sph"]
        return dict(zip(names, arrs))

    def operators(self):
        p = self.params
        nxi, nth, nph = p["n_xi"], p["n_theta"], 2 * p["n_phi_half"]
        Dr, Dth, Dmu, Dph = np.zeros((nxi, nxi)), np.zeros((nth, nth)), np.zeros((nth, nth)), \
            np.zeros((nph, nph))
        _check(self._lib.or_operators(self._h, _dp(Dr), _dp(Dth), _dp(Dmu), _dp(Dph)), "ops")
        return dict(Dr=Dr, Dth=Dth, Dmu=Dmu, Dph=Dph)

    def weights(self):
        """w_n = e^{z0 c_k} w^xi_k w^theta_j / (4 N_phi) in node order (Sec. 4.3)."""
        nd = self.nodes()
        p = self.params
        nph = 2 * p["n_phi_half"]
        w = np.einsum("j,k->jk", nd["wth"], nd["ecw"]) / (2.0 * nph)
        return np.broadcast_to(w, (nph,) + w.shape).reshape(-1).copy()

    # -- equation of state ----------------------------------------------------
    def eos(self, T: float) -> dict:
        out = np.zeros(16)
        _check(self._lib.or_eos(self._h, float(T), _dp(out)), "eos")
        return dict(zip(EOS_FIELDS, out))

    def solve_T(self, target: float, which: int = 0) -> float:
        T = ctypes.c_double()
        _check(self._lib.or_solve_T(self._h, float(target), int(which), ctypes.byref(T)), "solve_T")
        return T.value

    # -- state ----------------------------------------------------------------
    def init_state(self, eps0, nthreads: int = 0):
        eps0 = np.ascontiguousarray(eps0, dtype=np.float64).reshape(self.ns)
        f = np.zeros((self.ns, self.nn))
        lnM = np.zeros(self.ns)
        _check(self._lib.or_init_state(self._h, _dp(eps0), _dp(f), _dp(lnM), _nt(nthreads)), "init")
        return f, lnM

    def step(self, f, lnM, tau, dtau, nsteps=1, nthreads: int = 0):
        """Advance (f, lnM) in place by nsteps Heun steps starting at tau."""
        assert f.dtype == np.float64 and f.flags.c_contiguous and f.shape == (self.ns, self.nn)
        assert lnM.dtype == np.float64 and lnM.flags.c_contiguous and lnM.shape == (self.ns,)
        _check(self._lib.or_step(self._h, _dp(f), _dp(lnM), float(tau), float(dtau), int(nsteps),
                                 _nt(nthreads)), "step")
        return f, lnM

    def rhs(self, f, lnM, tau, nthreads: int = 0):
        f = np.ascontiguousarray(f, dtype=np.float64)
        lnM = np.ascontiguousarray(lnM, dtype=np.float64)
        r = np.zeros_like(f)
        g = np.zeros(self.ns)
        _check(self._lib.or_rhs(self._h, _dp(f), _dp(lnM), float(tau), _dp(r), _dp(g),
                                _nt(nthreads)), "rhs")
        return r, g

    def moments(self, f, lnM, nthreads: int = 0):
        """Per site: eps [GeV/fm^3], T, u^tau, u^x, u^y, M, P_L [GeV/fm^3], M(T)."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        lnM = np.ascontiguousarray(lnM, dtype=np.float64)
        out = np.zeros((self.ns, 8))
        _check(self._lib.or_moments(self._h, _dp(f), _dp(lnM), _dp(out), _nt(nthreads)), "moments")
        return out

    def observables(self, f, lnM, nthreads: int = 0):
        """(eps_p, v2 weighted by p_perp) of the whole grid."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        lnM = np.ascontiguousarray(lnM, dtype=np.float64)
        out = np.zeros(2)
        _check(self._lib.or_observables(self._h, _dp(f), _dp(lnM), _dp(out), _nt(nthreads)), "observables")
        return float(out[0]), float(out[1])

    def step_sites(self, f, lnM, tau, dtau, sites, nthreads: int = 0):
        """One Heun step evaluated only at `sites` of a (possibly huge) grid."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        lnM = np.ascontiguousarray(lnM, dtype=np.float64)
        sites = np.ascontiguousarray(sites, dtype=np.int32)
        fo = np.zeros((len(sites), self.nn))
        mo = np.zeros(len(sites))
        _check(self._lib.or_step_sites(self._h, _dp(f), _dp(lnM), float(tau), float(dtau),
                                       sites.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                       len(sites), _dp(fo), _dp(mo), _nt(nthreads)), "step_sites")
        return fo, mo


def _nt(n):
    return int(n) if n and n > 0 else (os.cpu_count() or 1)


_lib_cs = None


def _load_cs():
    global _lib_cs
    if _lib_cs is None:
        build()
        lib = ctypes.CDLL(_LIB_CS)
        vp, d, i = ctypes.c_void_p, ctypes.c_double, ctypes.c_int
        lib.or_create.argtypes = [ctypes.POINTER(OracleParams), ctypes.POINTER(vp)]
        lib.or_destroy.argtypes = [vp]
        lib.or_destroy.restype = None
        lib.or_num_nodes.argtypes = [vp]
        lib.or_init_state.argtypes = [vp, vp, vp, vp, i]
        lib.or_step.argtypes = [vp, vp, vp, d, d, i, i]
        lib.or_moments.argtypes = [vp, vp, vp, vp, i]
        lib.or_observables.argtypes = [vp, vp, vp, vp, i]
        _lib_cs = lib
    return _lib_cs


class TangentOracle:
    """The oracle's algorithm in complex arithmetic (the complex-step build of
    rlb_oracle.c): inputs with imaginary parts h d carry, through every step,
    imaginary parts that are h times the derivatives along d (forward-mode
    differentiation, exact to rounding for h far below the real parts; no
    subtraction as in finite differences).  eta_over_s_im is the imaginary
    part of eta/s.  Arrays are complex128."""

    def __init__(self, **kw):
        p = dict(DEFAULTS)
        unknown = set(kw) - set(p)
        if unknown:
            raise TypeError("unknown oracle parameters: %s" % sorted(unknown))
        p.update(kw)
        self.params = p
        self._p = OracleParams(**{k: p[k] for k in p})
        self._lib = _load_cs()
        h = ctypes.c_void_p()
        _check(self._lib.or_create(ctypes.byref(self._p), ctypes.byref(h)), "create")
        self._h = h
        self.nn = self._lib.or_num_nodes(self._h)
        self.ns = p["nx"] * p["ny"]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.or_destroy(h)
            self._h = None

    def init_state(self, eps0, nthreads: int = 0):
        eps0 = np.ascontiguousarray(eps0, dtype=np.complex128).reshape(self.ns)
        f = np.zeros((self.ns, self.nn), dtype=np.complex128)
        lnM = np.zeros(self.ns, dtype=np.complex128)
        _check(self._lib.or_init_state(self._h, eps0.ctypes.data, f.ctypes.data, lnM.ctypes.data,
                                       _nt(nthreads)), "init")
        return f, lnM

    def step(self, f, lnM, tau, dtau, nsteps=1, nthreads: int = 0):
        assert f.dtype == np.complex128 and f.flags.c_contiguous and lnM.dtype == np.complex128
        _check(self._lib.or_step(self._h, f.ctypes.data, lnM.ctypes.data, float(tau), float(dtau),
                                 int(nsteps), _nt(nthreads)), "step")
        return f, lnM

    def moments(self, f, lnM, nthreads: int = 0):
        out = np.zeros((self.ns, 8), dtype=np.complex128)
        _check(self._lib.or_moments(self._h, f.ctypes.data, lnM.ctypes.data, out.ctypes.data,
                                    _nt(nthreads)), "moments")
        return out

    def observables(self, f, lnM, nthreads: int = 0):
        out = np.zeros(2, dtype=np.complex128)
        _check(self._lib.or_observables(self._h, f.ctypes.data, lnM.ctypes.data, out.ctypes.data,
                                        _nt(nthreads)), "observables")
        return complex(out[0]), complex(out[1])


def v2_directional_derivative(eps0, d_eps0, d_eta, steps, tau0, dtau, h=1e-30, nthreads: int = 0, **kw):
    """(v2, dv2 along (d_eps0, d_eta)) of the oracle run eps0 -> steps Heun
    steps -> p_perp-weighted v2, by one complex-step run: eps0 + i h d_eps0,
    eta/s + i h d_eta."""
    eta = kw.pop("eta_over_s", DEFAULTS["eta_over_s"])
    o = TangentOracle(eta_over_s=eta, eta_over_s_im=h * d_eta, **kw)
    f, lnM = o.init_state(np.asarray(eps0, dtype=np.float64) + 1j * h * np.asarray(d_eps0, dtype=np.float64),
                          nthreads)
    o.step(f, lnM, tau0, dtau, steps, nthreads)
    v2 = o.observables(f, lnM, nthreads)[1]
    return v2.real, v2.imag / h


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
