"""The multi-process path of bench.py on CPU: two gloo ranks (world size 2),
each a replica of the step with its own time and work; the whole-job figure
is all ranks' units over the slowest rank's time, the same on every rank.
The path shards into independent instances, so there is no data exchange to
test beyond this reduction (no GPU; rendezvous on 127.0.0.1)."""
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
import torch.distributed as dist
import bench
rank, world, local = bench.dist_env()
dist.init_process_group("gloo", init_method="env://")
ms = [10.0, 25.0][rank]
units = [100.0, 300.0][rank]
value, t, u = bench.aggregate_replicas(ms, units, dist, "cpu")
print(json.dumps({"rank": rank, "world": world, "local": local, "value": value, "ms": t, "units": u}))
dist.barrier()
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_aggregate_single_process():
    import bench

    value, ms, units = bench.aggregate_replicas(20.0, 442401 * 100)
    assert ms == 20.0 and units == 442401 * 100
    assert value == pytest.approx(442401 * 100 / 0.020, rel=1e-15)


def test_two_gloo_ranks_agree_on_max_time_and_summed_work():
    pytest.importorskip("torch.distributed")
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD, ROOT], env=env, cwd=ROOT,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            out, err = p.communicate(timeout=120)
        except subprocess.TimeoutExpired:
            for q in procs:
                q.kill()
            raise
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    by_rank = {o["rank"]: o for o in outs}
    assert set(by_rank) == {0, 1}
    for r, o in by_rank.items():
        assert o["world"] == 2 and o["local"] == r
        assert o["ms"] == 25.0  # the slowest rank
        assert o["units"] == 400.0  # both ranks' work
        assert o["value"] == pytest.approx(400.0 / 0.025, rel=1e-15)
