"""Multi-rank logic of bench.py on CPU: two gloo ranks (world size 2) check
the timing reductions (max of the step times, sum of the particle-steps)
and that only rank 0 runs and prints the reference (oracle) arm."""
import io
import json
import multiprocessing as mp
import os
import socket
import sys
from contextlib import redirect_stdout

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, q):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port), BENCH_BACKEND="gloo")
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    ws, r, local = bench.dist_setup()
    bench.barrier(ws)
    mx = bench.allreduce_max(10.0 + rank, ws)
    sm = bench.allreduce_sum(1.5 * (rank + 1), ws)

    class A:
        n_per_species, ref_sample, steps, warmup, gpus = 2000, 300, 2, 1, 2
    out = io.StringIO()
    with redirect_stdout(out):
        bench.run_reference(A, ws, r)
    bench.barrier(ws)
    dist.destroy_process_group()
    q.put((r, ws, mx, sm, out.getvalue()))


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, port, q)) for r in (0, 1)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        r, ws, mx, sm, text = q.get(timeout=240)
        res[r] = (ws, mx, sm, text)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        ws, mx, sm, _ = res[r]
        assert ws == 2 and mx == 11.0 and sm == 4.5
    assert res[1][3] == ""                       # rank 1 does no reference work
    line = json.loads(res[0][3].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
