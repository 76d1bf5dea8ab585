"""CPU tests of the multi-GPU (replicas only) bench path with two gloo ranks:
frames are independent, so every rank detects its own slice of the stream
and the only collective is the max of the ranks' times; the whole-job rate
is all ranks' frames over the slowest rank's time.  The reference arm runs
on rank 0 only; other ranks exit 0 without work."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    w, r, _ = bench.dist_env()
    slowest = bench.max_over_ranks(0.5 + rank)          # rank r took 0.5 + r seconds
    q.put((r, w, slowest, bench.whole_job_rate(w, 1000, slowest),
           bench.replica_frames(r, 1000)))
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert all(o[2] == 1.5 for o in out)                 # every rank sees the slowest time
    assert all(abs(o[3] - 2 * 1000 / 1.5) < 1e-9 for o in out)
    assert [o[4] for o in out] == [0, 1000]              # disjoint slices of the stream


def test_max_over_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.whole_job_rate(1, 1000, 0.5) == 2000.0


def test_reference_arm_other_rank_exits_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, env=env, timeout=300, cwd=ROOT)
    assert r.returncode == 0 and r.stdout.strip() == ""
