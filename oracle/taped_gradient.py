"""Oracle (forward-mode) gradient of the adjoint test case, written to
tests/golden/adjoint_taped_32x32.json.

TEST INFRASTRUCTURE ONLY: calls nothing but oracle/ and the seeded input
generator.  The case: 32 x 32 grid, dx = 0.1 fm, 8 x 8 x 12 lattice, eta/s
0.08, 40 hotspots (0.4 fm, Exp(mean 15 GeV/fm^3) amplitudes, centres N(0,
0.8 fm), seed 1108) on 10 GeV/fm^3, 50 Heun steps of 0.0036 fm/c from 0.4
fm/c; the objective is the final p_perp-weighted v2 of the grid.  Each of the
41 derivatives (40 amplitudes, eta/s) is one run of the oracle's own algorithm
in complex arithmetic (oracle/rlb_oracle.c built with -DOR_COMPLEX_STEP): the
input gets an imaginary part h = 1e-30 along the parameter and dv2 = Im(v2)/h.

    python oracle/taped_gradient.py [--threads N]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

from oracle import oracle as om  # noqa: E402
from paper_1108_5561_gb300.inputs import hotspot_basis, hotspots  # noqa: E402

CASE = dict(nx=32, ny=32, dx=0.1, eta_over_s=0.08, n_hot=40, seed=1108, spread=0.8, mean_amp=15.0,
            floor=10.0, steps=50, tau0=0.4, dtau=0.0036, h=1e-30)
OUT = os.path.join(os.path.dirname(HERE), "tests", "golden", "adjoint_taped_32x32.json")


def case_inputs():
    c = CASE
    _, amps, cen = hotspots(c["nx"], c["ny"], dx=c["dx"], n=c["n_hot"], seed=c["seed"], spread=c["spread"],
                            mean_amp=c["mean_amp"], floor=c["floor"])
    basis = hotspot_basis(c["nx"], c["ny"], cen, dx=c["dx"])
    eps0 = c["floor"] + amps @ basis
    return eps0.reshape(c["ny"], c["nx"]), amps, basis


def derivative(eps0, d_eps0, d_eta, threads):
    c = CASE
    return om.v2_directional_derivative(eps0, d_eps0, d_eta, c["steps"], c["tau0"], c["dtau"], h=c["h"],
                                        nthreads=threads, nx=c["nx"], ny=c["ny"], dx=c["dx"],
                                        eta_over_s=c["eta_over_s"])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=0)
    args = ap.parse_args()
    eps0, amps, basis = case_inputs()
    t0 = time.time()
    v2, deta = derivative(eps0, np.zeros_like(eps0), 1.0, args.threads)
    dA = []
    for i in range(len(amps)):
        _, d = derivative(eps0, basis[i].reshape(eps0.shape), 0.0, args.threads)
        dA.append(d)
        print("amplitude %2d: %.12e (%.0f s)" % (i, d, time.time() - t0), flush=True)
    rec = {"case": CASE, "v2": v2, "dv2_deta_over_s": deta, "dv2_dA": dA, "amplitudes": list(map(float, amps)),
           "method": "complex-step forward derivatives of the FP64 oracle (rlb_oracle.c, -DOR_COMPLEX_STEP)"}
    with open(OUT, "w") as fh:
        json.dump(rec, fh, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
