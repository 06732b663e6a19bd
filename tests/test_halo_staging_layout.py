"""Host-side check of the halo staging of stage variant 6 (the copies and line
offsets of stage_kernel_mpt, restated here): on small and odd-sized periodic
grids every copy stays inside the population array and the staging buffer,
no two copies overlap, the bytes equal the mbarrier's expected count, every
address is 16-byte aligned, and every thread's staged line (own, upwind x and
y neighbours, corrector base) is the line the unstaged kernel reads from
global memory.  Azimuths phi_l = l pi / N_phi' (the lattice's nodes)."""
import math

import numpy as np
import pytest

NXI, NTH, NPH = 8, 8, 12
H = NTH // 2
TS = H * NPH
CH = NTH * NXI
NN = CH * NPH


def _nodes():
    c = [math.cos(l * math.pi / (NPH // 2)) for l in range(NPH)]
    s = [math.sin(l * math.pi / (NPH // 2)) for l in range(NPH)]
    return [0.0 if abs(v) < 1e-12 else v for v in c], [0.0 if abs(v) < 1e-12 else v for v in s]


CPH, SPH = _nodes()


def _runs():
    start = [[0, 0] for _ in range(4)]
    count = [[0, 0] for _ in range(4)]
    n = [0] * 4
    for c in range(4):
        r = 0
        for l in range(NPH):
            v = CPH[l] if c < 2 else SPH[l]
            if not ((v > 0) if c % 2 == 0 else not v > 0):
                continue
            n[c] += 1
            pv = (CPH[l - 1] if c < 2 else SPH[l - 1]) if l > 0 else 0.0
            if not (l > 0 and ((pv > 0) if c % 2 == 0 else not pv > 0)):
                assert r < 2
                start[c][r] = l
                r += 1
            count[c][r - 1] += 1
    return start, count, n


START, COUNT, N = _runs()
OWN, XP1 = 0, 2 * NPH
XP2 = XP1 + N[0]
XM2 = XP2 + N[0]
XM3 = XM2 + N[1]
YP = XM3 + N[1]
YM = YP + 4 * N[2]
BASE = YM + 4 * N[3]


def _copy(c, x0, y, nx, ny):
    if c in (0, 25):
        return (OWN if c == 0 else BASE), y * nx + x0, 0, 2 * NPH, c != 0
    g, r = (c - 1) >> 1, (c - 1) & 1
    if g < 4:
        cls, dx, dy, d = (0 if g < 2 else 1), [-1, -2, 2, 3][g], 0, [XP1, XP2, XM2, XM3][g]
    else:
        h = g - 4
        s, rr = h & 1, ((h >> 1) & 1) + 1
        cls = 2 if h < 4 else 3
        dx, dy = s, (-rr if cls == 2 else rr)
        d = (YP if cls == 2 else YM) + (2 * (rr - 1) + s) * N[cls]
    xs, ys = (x0 + dx) % nx, (y + dy) % ny
    return d + (COUNT[cls][0] if r == 1 else 0), ys * nx + xs, START[cls][r], COUNT[cls][r], False


def test_azimuth_classes_are_two_runs_at_most():
    assert BASE == 8 * NPH
    for c in range(4):
        assert sum(COUNT[c]) == N[c]
    assert N[0] + N[1] == NPH and N[2] + N[3] == NPH


@pytest.mark.parametrize("nx,ny", [(2, 1), (2, 2), (4, 1), (4, 3), (6, 5), (8, 7), (16, 16), (10, 2)])
def test_staged_lines_are_the_global_lines(nx, ny):
    ns = nx * ny
    f = np.arange(ns * NN, dtype=np.int64)
    fb = -1 - f
    for y in range(ny):
        for x0 in range(0, nx, 2):
            for mode in (0, 1):
                stg = np.full(10 * NN, -(10 ** 12), dtype=np.int64)
                used = np.zeros(10 * NN, dtype=bool)
                total = 0
                for c in range(26):
                    dst, site, l0, cnt, from_base = _copy(c, x0, y, nx, ny)
                    if cnt == 0 or (from_base and mode == 0):
                        continue
                    assert 0 <= site < ns
                    if c in (0, 25):
                        assert cnt == 2 * NPH and site % nx + 1 < nx
                    else:
                        assert l0 + cnt <= NPH
                    s0, d0 = site * NN + l0 * CH, dst * CH
                    assert s0 + cnt * CH <= ns * NN and d0 + cnt * CH <= 10 * NN
                    assert (s0 * 4) % 16 == 0 and (d0 * 4) % 16 == 0
                    assert not used[d0:d0 + cnt * CH].any()
                    used[d0:d0 + cnt * CH] = True
                    stg[d0:d0 + cnt * CH] = (fb if from_base else f)[s0:s0 + cnt * CH]
                    total += cnt * CH * 4
                assert total == (10 if mode == 1 else 8) * NN * 4
                for t in range(2 * TS):
                    sl = t // TS
                    q = t - sl * TS
                    l, jp = q // H, q % H
                    cp, sp = CPH[l], SPH[l]
                    hx = sum((CPH[m] > 0) == (cp > 0) for m in range(l))
                    hy = sum((SPH[m] > 0) == (sp > 0) for m in range(l))
                    if cp > 0:
                        c1, c2 = (XP1 + hx, XP2 + hx) if sl == 0 else (OWN + l, XP1 + hx)
                    else:
                        c1, c2 = (OWN + NPH + l, XM2 + hx) if sl == 0 else (XM2 + hx, XM3 + hx)
                    yb, nyc = (YM, N[3]) if not sp > 0 else (YP, N[2])
                    c3, c4 = yb + sl * nyc + hy, yb + (2 + sl) * nyc + hy
                    chunks = [OWN + sl * NPH + l] * 2 + [c1, c2, c1, c2, c3, c4, c3, c4] + [BASE + sl * NPH + l] * 2
                    jA, jB = jp, NTH - 1 - jp
                    lines = [jA, jB, jA, jA, jB, jB, jA, jA, jB, jB, jA, jB]
                    # the unstaged kernel's global lines
                    x = x0 + sl
                    sx, sy = (-1 if cp > 0 else 1), (-1 if sp > 0 else 1)
                    x1, x2, y1, y2 = (x + sx) % nx, (x + 2 * sx) % nx, (y + sy) % ny, (y + 2 * sy) % ny
                    sites = [y * nx + x] * 2 + [y * nx + x1, y * nx + x2] * 2 + [y1 * nx + x, y2 * nx + x] * 2 \
                        + [y * nx + x] * 2
                    for i in range(12 if mode == 1 else 10):
                        s0 = chunks[i] * CH + lines[i] * NXI
                        g0 = sites[i] * NN + (l * NTH + lines[i]) * NXI
                        want = (fb if i >= 10 else f)[g0:g0 + NXI]
                        assert np.array_equal(stg[s0:s0 + NXI], want), (nx, ny, y, x0, t, i)
