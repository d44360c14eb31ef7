"""The multi-process path of bench.py on CPU: two gloo ranks (replicas, no
data-path collective; the timing is the slowest rank's), and the reference
arm, which only rank 0 runs."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    w, r, _ = bench._dist()
    bench._barrier(w)
    ms_max = bench._max_over_ranks(w, 10.0 + 5.0 * rank)   # rank 1 is the slow one
    q.put((r, w, ms_max, bench._whole_job_rate(w, 3, 1000, ms_max)))
    bench._barrier(w)
    dist.destroy_process_group()


def test_two_gloo_ranks_time_by_the_slowest_and_sum_the_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, ms_max, rate in out:
        assert w == 2 and ms_max == 15.0
        assert rate == pytest.approx(2 * 3 * 1000 / 15e-3)
    assert sorted(o[0] for o in out) == [0, 1]


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                                      "--warmup", "0"])
    assert bench.main() == 0
    assert capsys.readouterr().out == ""
