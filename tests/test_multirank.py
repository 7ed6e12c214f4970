"""The N > 1 host path of bench.py on CPU: two gloo ranks (world size 2).  The path does
not shard a grid (replicas only), so the only cross-rank operations are the timing
reductions (max of the timed region, sum of the units processed) and the barrier; the
reference arm runs on rank 0 alone and the other ranks exit 0 without work."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "WORLD_SIZE": str(world), "RANK": str(rank), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import bench
    w, r, _ = bench.dist_setup()
    assert (w, r) == (world, rank)
    res = {"max": bench.max_over_ranks(1.5 + rank, w), "sum": bench.sum_over_ranks(10.0 * (rank + 1), w)}
    bench.barrier(w)
    buf = io.StringIO()
    with redirect_stdout(buf):
        rc = bench.run_reference(
            bench.argparse.Namespace(n=64, ref_edge=8, steps=1, warmup=3), w, r)
    res["rc"] = rc
    res["stdout"] = buf.getvalue()
    import torch.distributed as dist
    dist.destroy_process_group()
    out.put((rank, res))


def test_two_gloo_ranks_reduce_and_reference_on_rank0():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for r in range(2):
        assert got[r]["max"] == 2.5 and got[r]["sum"] == 30.0 and got[r]["rc"] == 0
    assert got[1]["stdout"] == ""
    line = json.loads(got[0]["stdout"].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
