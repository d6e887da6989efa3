"""The N > 1 path of bench.py (independent replicas, one rank per GPU) on
CPU with the gloo backend: whole-job aggregation (max time, summed work) and
the reference arm running on rank 0 only."""
import contextlib
import io
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        t, m = bench.combine_over_ranks(1.0 + rank, 10 * (rank + 1), torch.device("cpu"), ws)
        printed = io.StringIO()
        args = bench.parse_args(["--impl", "reference", "--steps", "1", "--warmup", "0",
                                 "--workload", "grid4k", "--gpus", str(ws)])
        with contextlib.redirect_stdout(printed):
            bench.run_reference(args)
        out[rank] = (t, m, printed.getvalue())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2])
def test_replicas_aggregate_and_reference_on_rank0(ws):
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, ws, port, out)) for r in range(ws)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=300)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(ws):
        t, m, printed = res[r]
        assert t == float(ws) and m == float(sum(10 * (k + 1) for k in range(ws)))
        if r == 0:
            assert '"impl": "reference"' in printed and '"value"' in printed
        else:
            assert printed == ""


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_over_ranks(2.5, 7, None, 1) == (2.5, 7.0)
