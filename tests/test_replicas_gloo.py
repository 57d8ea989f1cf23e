"""Host logic of the multi-GPU path (replicas: every rank renders its own
copy of the workload, no data exchange): the timed region is the slowest
rank's and the job rate counts every rank's frames.  Two gloo ranks on CPU."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    local = [120.0, 150.0][rank]
    total = bench.job_time_ms(local, ws, torch.device("cpu"))
    q.put((rank, total, bench.frame_times(total, 40, ws)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank_and_all_frames():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total, (ms_step, ms_frame) in out:
        assert total == 150.0
        assert ms_step == pytest.approx(150.0 / 40)
        assert ms_frame == pytest.approx(150.0 / 80)
