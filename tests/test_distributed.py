"""The multi-rank path of the benchmark on CPU: two gloo ranks run the
replica host logic (rank context, barrier, max over ranks of the timing,
per-rank seeds, weak-scaling value) exactly as the GPU ranks do, and the
reference arm of rank 1 does no work."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      LOCAL_RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    from paper_1808_02281_gb300 import synth
    ctx = bench.RankContext("gloo")
    ctx.barrier()
    ms = 10.0 + 5.0 * rank                     # the slower rank decides
    ms_max = ctx.max_over_ranks(ms)
    seed = bench.replica_seed(0, rank)
    draw = float(synth.normals(seed, 1)[0])
    value = bench.weak_scaling_value(1000, ctx.world, 4, ms_max)
    ctx.barrier()
    ctx.close()
    out.put((rank, ms_max, seed, draw, value))


def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]              # max over ranks on every rank
    assert res[0][2] != res[1][2] and res[0][3] != res[1][3]  # distinct replicas
    assert res[0][4] == res[1][4] == pytest.approx(2 * 1000 * 4 / 15e-3 / 1e9)


def test_reference_arm_other_ranks_do_nothing(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    args = type("A", (), {"steps": 1, "warmup": 3, "gpus": 2})()
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(args) == 0
    assert buf.getvalue() == ""
