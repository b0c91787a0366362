"""The N > 1 path of bench.py (independent replicas, no data-path collective) on CPU with the
gloo backend, world size 2: each rank builds its own seeded problem, the timed region is the
slowest rank's, whole-job throughput counts every rank's reconstructions, only rank 0 prints,
and the oracle reference arm runs on rank 0 alone."""
import json
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


def _rank(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # each replica draws its own problem (seed + rank)
    P = bench.make_problem("par2d_64", rank)
    digest = float(abs(P.b).sum())
    slowest = bench.max_over_ranks(1.0 + rank, dist)
    gathered = [None] * world
    dist.all_gather_object(gathered, digest)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"slowest": slowest, "digests": gathered,
                   "value": bench.replica_value(1, world, slowest)}, f)
    import io
    import contextlib
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.emit({"rank": rank}, rank)
    with open(os.path.join(out_dir, f"p{rank}.txt"), "w") as f:
        f.write(buf.getvalue())
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_two_ranks_gloo(tmp_path):
    port = _free_port()
    mp.spawn(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    r0 = json.load(open(tmp_path / "r0.json"))
    r1 = json.load(open(tmp_path / "r1.json"))
    assert r0["slowest"] == r1["slowest"] == 2.0
    assert r0["digests"][0] != r0["digests"][1]          # distinct problems per replica
    assert r0["value"] == pytest.approx(1.0)                 # 2 reconstructions / 2 s
    assert (tmp_path / "p0.txt").read_text().strip() == json.dumps({"rank": 0})
    assert (tmp_path / "p1.txt").read_text() == ""


def test_reference_arm_only_rank_zero(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        workload = "par2d_512"
        steps = 1
        warmup = 0

    bench.reference_arm(A(), 1, 2)     # rank 1 of 2: returns without work or output
    assert capsys.readouterr().out == ""
