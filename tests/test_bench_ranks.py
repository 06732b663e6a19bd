"""Multi-rank bookkeeping of bench.py on CPU (gloo, world size 2).

With N GPUs every rank runs the same workload (weak scaling, no data-path
exchange); the job time is the maximum over ranks and the job throughput is
N x units per rank / that time.  Two gloo ranks with different timed regions
check the maximum, the barrier and the aggregation.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, os, sys
sys.path.insert(0, sys.argv[1])
import bench
r = bench.Ranks("gloo")
t = 1.5 if r.rank == 0 else 2.5          # the slower rank sets the job time
r.barrier()
tmax = r.max(t, device="cpu")
rate = bench.job_rate(1000.0, r.world, tmax)
print(json.dumps({"rank": r.rank, "world": r.world, "tmax": tmax, "rate": rate}))
r.close()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_single_rank_needs_no_process_group(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    r = bench.Ranks("gloo")
    assert (r.rank, r.world, r.dist) == (0, 1, None)
    r.barrier()
    assert r.max(3.25, device="cpu") == 3.25
    assert bench.job_rate(10.0, 1, 2.0) == 5.0
    r.close()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_take_the_slowest_time():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD, ROOT], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=110)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    assert sorted(o["rank"] for o in outs) == [0, 1]
    for o in outs:
        assert o["world"] == 2
        assert o["tmax"] == 2.5
        assert o["rate"] == pytest.approx(2 * 1000.0 / 2.5)
