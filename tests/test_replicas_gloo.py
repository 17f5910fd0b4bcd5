"""The multi-process path of bench.py on CPU: two gloo ranks (no GPU).

The scan does not shard (a leg is one unit of work here), so N GPUs run N
replicas: the only cross-rank steps are a barrier around the timed region and
the maximum of the ranks' times; the reference arm runs on rank 0 alone.
"""
import multiprocessing as mp
import os
import socket
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import sys
    sys.path.insert(0, ROOT)
    try:
        import bench
        D = bench.Dist()
        D.barrier()
        got = D.max(1.5 + rank)
        args = types.SimpleNamespace(workload="tls", small=True, steps=1, warmup=0, cpu_sample_s=0.2)
        ref = bench.run_reference(args, D)
        D.barrier()
        D.close()
        q.put((rank, D.world, got, None if ref is None else (ref["impl"], ref["n_gpus"], ref["value"] > 0)))
    except Exception as e:           # reported to the parent, which fails the test
        q.put((rank, -1, repr(e), None))


def test_two_gloo_ranks_barrier_max_and_reference_on_rank0():
    torch = pytest.importorskip("torch")
    if not torch.distributed.is_available():
        pytest.skip("torch.distributed not available")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        rank, world, got, ref = q.get(timeout=300)
        res[rank] = (world, got, ref)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in (0, 1):
        world, got, ref = res[rank]
        assert world == 2, got
        assert got == 2.5            # max over ranks of 1.5 + rank
    assert res[0][2] == ("reference", 2, True)
    assert res[1][2] is None         # rank 1 does no work in the reference arm
