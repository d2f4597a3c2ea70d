"""The benchmark's multi-rank path on CPU: two gloo ranks, as torchrun would
start them.  Each rank runs its own stations (no exchange on the data path);
the job's throughput is the units of all ranks over the slowest rank's time,
and the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, out):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(ws), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    r, w, _ = bench.dist_init("gloo")
    assert (r, w) == (rank, ws)
    bench.barrier(w)
    # rank r: 100 * (r + 1) units in (r + 1) seconds -> job: 300 units / 2 s
    rate = bench.whole_job_rate(100 * (rank + 1), float(rank + 1), w)
    mx = bench.max_over_ranks(float(rank), w)
    out.put((rank, rate, mx, bench.rank_seed(rank)))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, rate, mx, seed in res:
        assert rate == pytest.approx(150.0)
        assert mx == 1.0
    assert res[0][3] != res[1][3]


def test_reference_arm_only_on_rank0(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")

    class A:
        n_envs, warmup, steps, gpus = 64, 0, 1, 2
    bench.run_reference(A())
    assert capsys.readouterr().out == ""
