"""The multi-process path of bench.py on the CPU (gloo, world size 2): one
replica per rank, the timing barrier, max-over-ranks time and summed units,
and the reference arm printing on rank 0 only. No GPU: the data path has no
collective (every rank simulates its own circuit), so these helpers are the
whole of the N > 1 logic."""
import contextlib
import datetime
import io
import json
import os
import socket
import types

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    try:
        # a short collective timeout: a rank that fails ends its peer's next barrier
        dist.init_process_group("gloo", rank=rank, world_size=ws,
                                timeout=datetime.timedelta(seconds=60))
        import bench
        w, r, local = bench.dist_env()
        bench.barrier(w)
        mx = bench.reduce_max(1.5 * (rank + 1), w)
        sm = bench.reduce_sum(float(rank + 1), w)
        args = types.SimpleNamespace(n=300, depth=1000, cpu_layers=2, cpu_rows=8, steps=1,
                                     warmup=0)
        buf = io.StringIO()
        with contextlib.redirect_stdout(buf):
            bench.run_reference(args)
        bench.barrier(w)
        q.put((rank, w, r, local, mx, sm, buf.getvalue()))
        dist.destroy_process_group()
    except BaseException as e:  # reported to the parent instead of hanging it
        q.put((rank, "error", repr(e)))
        raise


def test_two_replicas_on_gloo():
    ws = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = []
    try:
        for _ in range(ws):
            item = q.get(timeout=300)
            assert item[1] != "error", f"rank {item[0]} failed: {item[2]}"
            out.append(item)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.terminate()
                p.join()
    out.sort()
    for p in procs:
        assert p.exitcode == 0
    for rank, w, r, local, mx, sm, printed in out:
        assert (w, r, local) == (ws, rank, rank)
        assert mx == 3.0 and sm == 3.0
        if rank == 0:
            line = json.loads(printed.strip().splitlines()[-1])
            assert line["impl"] == "reference" and line["value"] > 0
        else:
            assert printed == ""
