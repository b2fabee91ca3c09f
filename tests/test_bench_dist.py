"""Multi-rank logic of bench.py with two gloo ranks on the CPU: the timed region is the
slowest rank's, the value sums every rank's units (independent replicas, weak scaling)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, ws, port, out):
    import sys
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    w, r, _ = bench.dist_setup()
    assert (w, r) == (ws, rank)
    t = 1.0 + rank                      # rank 1 is the slow one
    tmax = bench.max_over_ranks(t, ws, torch.device("cpu"))
    out[rank] = (tmax, bench.job_value(1000.0, ws, tmax))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_units():
    ws = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, ws, port, out)) for r in range(ws)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        for r in range(ws):
            tmax, value = out[r]
            assert tmax == 2.0
            assert value == pytest.approx(1000.0 * 2 / 2.0)


def test_gpus_must_match_the_ranks():
    """A plain `python bench.py --gpus 2` (one rank) refuses to run instead of measuring one
    replica under an N-GPU label."""
    import subprocess
    import sys
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2"], capture_output=True,
                       text=True, env=env, timeout=120)
    assert r.returncode != 0
    assert "--gpus 2 but 1 rank" in r.stderr
