"""The multi-GPU form is replicas: every rank runs the whole inference on its
own queries and nothing is exchanged on the data path.  This checks the host
side of bench.py's N > 1 path with two gloo ranks on the CPU: the barrier,
the max-over-ranks timing and the whole-job throughput."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    os.environ.update({"WORLD_SIZE": str(ws), "RANK": str(rank), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist

    import bench
    got_ws, got_rank, _ = bench.dist_setup()
    assert dist.get_backend() == "gloo"
    bench.barrier(got_ws)
    # rank r "took" (r + 1) * 100 ms for 10 inferences
    slowest = bench.max_over_ranks((got_rank + 1) * 100.0, got_ws)
    value = bench.job_throughput(10, (got_rank + 1) * 100.0, got_ws)
    q.put((got_rank, got_ws, slowest, value))
    dist.destroy_process_group()


def test_two_replicas_gloo():
    if torch.cuda.is_available():
        pytest.skip("host-side test (gloo); GPUs present")
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(ws))
    for rank, got_ws, slowest, value in res:
        assert got_ws == ws
        assert slowest == 200.0          # the max over ranks
        assert abs(value - 2 * 10 / 0.2) < 1e-9   # all ranks' inferences / slowest time
