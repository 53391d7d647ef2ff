"""Multi-GPU runs are replicas (no data-path exchange): the host logic of bench.py's
torchrun path -- barrier, max over the ranks' times, whole-job throughput -- on two
gloo ranks on the CPU."""
import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, outdir):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    d = bench.Dist("gloo")
    d.barrier()
    ms = 100.0 * (rank + 1)                       # rank 1 is the slower replica
    value, ms_max = bench.replica_value(d, 5, ms)
    d.barrier()
    d.close()
    with open(os.path.join(outdir, "rank%d.json" % rank), "w") as f:
        json.dump({"value": value, "ms_max": ms_max, "world": d.world, "backend": d.backend}, f)


def test_two_gloo_replicas(tmp_path):
    world, port = 2, _free_port()
    mp.spawn(_rank, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(world)]
    for r in res:
        assert r["world"] == 2 and r["backend"] == "gloo"
        assert r["ms_max"] == 200.0                   # the slowest rank's time
        assert abs(r["value"] - 5 * 2 / 0.2) < 1e-9   # all ranks' steps over that time
