"""Multi-rank host logic on CPU (gloo, world size 2).

Subsystems and requests are independent problems, so ranks exchange no
data; they only agree on timing (max over ranks) and on totals (sum), and
split a request trace between them.
"""
import multiprocessing as mp
import os
import socket



def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    import bench
    from paper_2101_05916_gb300 import serve, workloads as wl
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        bench.barrier(ws)
        m = bench.reduce_max(ws, float(rank + 1) * 1.5)
        s = bench.reduce_sum(ws, 10.0 * (rank + 1))
        trace = wl.serving_trace(count=10)
        mine = [r.rid for r in serve.shard(trace, rank, ws)]
        q.put((rank, m, s, mine))
    finally:
        dist.destroy_process_group()


def test_two_rank_timing_and_sharding():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert all(o[1] == 3.0 for o in out)       # max over ranks
    assert all(o[2] == 30.0 for o in out)      # sum over ranks
    ids = out[0][3] + out[1][3]
    assert sorted(ids) == list(range(10)) and not set(out[0][3]) & set(out[1][3])
