"""Gradient of the final-state elliptic flow (v2 weighted by p_perp, see
rlb_observables) with respect to eta/s and to the amplitudes of the initial
hotspots, through the whole time evolution.  The adjoint of every time step
runs in the CUDA library (rlb_adjoint_step: the discrete adjoint of the
predictor-corrector; per-node work in FP64 or FP32 arithmetic, per-site
matching adjoint in FP64); this module only orders the calls, keeps step
checkpoints and wraps the result as a torch.autograd.Function.

Checkpointing: the forward run stores the state every `every` steps; the
backward sweep reruns each segment from its checkpoint, storing the state of
every step of the segment (device blobs), and reverses the steps one by one,
each reading its input state from its blob in place.  With every = 1 nothing
is recomputed (one blob per step: 52 MB per step on a 128 x 128 grid of 768
FP32 populations, 15.6 GB for 300 steps).  State blobs hold the
moments and Newton starting values too, so recomputed steps are bit-exact
copies of the forward ones.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib as L


class Adjoint:
    """Adjoint workspace of a Run (device memory from torch); `arithmetic` is
    RLB_F64 (default) or RLB_F32 for the per-node adjoint work."""

    def __init__(self, run, arithmetic: int = L.RLB_F64):
        self.run, self.lib, torch = run, run.lib, run.torch
        run._chk(self.lib.rlb_adjoint_set_arithmetic(run._h, int(arithmetic)), "rlb_adjoint_set_arithmetic")
        n = ctypes.c_size_t()
        run._chk(self.lib.rlb_adjoint_workspace_size(run._h, ctypes.byref(n)), "rlb_adjoint_workspace_size")
        self.ws = torch.empty(n.value, dtype=torch.uint8, device=run.device)
        run._chk(self.lib.rlb_adjoint_bind(run._h, ctypes.c_void_p(self.ws.data_ptr())), "rlb_adjoint_bind")

    def seed_v2(self) -> float:
        """v2 of the current state; the adjoint buffers become dv2/d(f, ln M)."""
        v = ctypes.c_double()
        self.run._chk(self.lib.rlb_adjoint_seed_v2(self.run._h, ctypes.byref(v), self.run._stream()),
                      "rlb_adjoint_seed_v2")
        return v.value

    def seed(self, fbar, lbar):
        """A general objective: the adjoint buffers become (dJ/df, dJ/d ln M) of
        the current state, given as FP64 tensors (sites x nodes, sites; host or
        device)."""
        torch = self.run.torch
        fb = torch.as_tensor(fbar, dtype=torch.float64).contiguous()
        lb = torch.as_tensor(lbar, dtype=torch.float64).contiguous()
        if fb.numel() != self.run.ns * self.run.nn or lb.numel() != self.run.ns:
            raise ValueError("seed shapes: (sites, nodes) and (sites,)")
        self.run._chk(self.lib.rlb_adjoint_seed(self.run._h, ctypes.c_void_p(fb.data_ptr()),
                                                ctypes.c_void_p(lb.data_ptr()), self.run._stream()),
                      "rlb_adjoint_seed")

    def step(self, blob=None):
        """Reverse one step.  Its input state: the run's state, or a device blob
        from run.save_state(device=True) of this run, read in place (the run's
        state is left as it is)."""
        saved = getattr(blob, "_rlb_saved", None) if blob is not None else None
        if saved is not None and saved[0] == self.run._h.value and blob.is_cuda:
            self.run._chk(self.lib.rlb_adjoint_step_from(self.run._h, ctypes.c_void_p(blob.data_ptr()), blob.numel(),
                                                         ctypes.c_double(saved[1]), self.run._stream()),
                          "rlb_adjoint_step_from")
            return
        if blob is not None:
            self.run.load_state(blob)
        self.run._chk(self.lib.rlb_adjoint_step(self.run._h, self.run._stream()), "rlb_adjoint_step")

    def ic(self, eps0, basis):
        """(dJ/dA_i for the rows of `basis` (n x sites, device FP64), dJ/d(eta/s))
        from the adjoint buffers of the initial state built from eps0 (device)."""
        n = 0 if basis is None else basis.shape[0]
        out = np.zeros(n + 1)
        dp = ctypes.POINTER(ctypes.c_double)
        bp = None if basis is None else ctypes.cast(ctypes.c_void_p(basis.data_ptr()), dp)
        ep = ctypes.cast(ctypes.c_void_p(eps0.data_ptr()), dp)
        self.run._chk(self.lib.rlb_adjoint_ic(self.run._h, ep, bp, n, out.ctypes.data_as(dp), self.run._stream()),
                      "rlb_adjoint_ic")
        return out[:n], float(out[n])


def forward_with_checkpoints(run, eps0, steps: int, every: int):
    """Initial state from eps0 (device FP64 tensor), then `steps` steps; returns
    the checkpoints {step: blob}."""
    cks = {}
    run.init_grid(eps0)
    for s in range(steps):
        if s % every == 0:
            cks[s] = run.save_state(device=True)
        run.step(1)
    return cks


def reverse_sweep(run, adj: Adjoint, cks, steps: int, every: int):
    """Adjoint of the `steps` steps (the adjoint buffers hold the seed).  A
    segment of one step needs no recompute: its adjoint reads the checkpoint
    in place, so the run's state is not restored for it."""
    for start in reversed(range(0, steps, every)):
        end = min(start + every, steps)
        if end - start > 1:
            run.load_state(cks[start])
        states = [cks[start]]
        for _ in range(start, end - 1):
            run.step(1)
            states.append(run.save_state(device=True))
        for s in reversed(range(start, end)):
            adj.step(states[s - start])  # the step's input state read in place


def v2_gradient(run, eps0, basis, steps: int, every: int = 32, arithmetic: int = L.RLB_F64):
    """v2 after `steps` steps from eps0 and its gradient: (v2, dv2/dA over the
    rows of basis, dv2/d(eta/s))."""
    cks = forward_with_checkpoints(run, eps0, steps, every)
    adj = Adjoint(run, arithmetic)
    v2 = adj.seed_v2()
    reverse_sweep(run, adj, cks, steps, every)
    gA, geta = adj.ic(eps0, basis)
    return v2, gA, geta


def elliptic_flow_function(arithmetic: int = L.RLB_F64):
    """torch.autograd.Function: v2(amplitudes, eta) = final p_perp-weighted v2
    of the run started from eps0 = floor + amplitudes @ basis (adjoint in
    `arithmetic`, RLB_F64 or RLB_F32)."""
    import torch

    class EllipticFlow(torch.autograd.Function):
        @staticmethod
        def forward(ctx, amps, eta, run, basis, floor, steps, every):
            if abs(float(eta) - run.grid.eta_over_s) > 1e-12 * run.grid.eta_over_s:
                raise ValueError("eta must be the run's eta/s")
            eps0 = (floor + amps.to(device=basis.device, dtype=torch.float64) @ basis).contiguous()
            cks = forward_with_checkpoints(run, eps0, steps, every)
            adj = Adjoint(run, arithmetic)
            v2 = adj.seed_v2()
            ctx.run, ctx.adj, ctx.cks, ctx.eps0, ctx.basis = run, adj, cks, eps0, basis
            ctx.steps, ctx.every = steps, every
            return torch.tensor(v2, dtype=torch.float64)

        @staticmethod
        def backward(ctx, gout):
            reverse_sweep(ctx.run, ctx.adj, ctx.cks, ctx.steps, ctx.every)
            gA, geta = ctx.adj.ic(ctx.eps0, ctx.basis)
            g = float(gout)
            return (torch.as_tensor(gA * g, dtype=torch.float64), torch.tensor(geta * g, dtype=torch.float64),
                    None, None, None, None, None)

    return EllipticFlow
