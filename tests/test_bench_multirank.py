"""The N > 1 path of bench.py on CPU: world-size-2 gloo ranks, each timing its own replica;
the job rate uses the slowest rank's time (MAX over ranks) and counts every rank's steps."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_s = [2.0, 3.0][rank]            # the second replica is slower
    rate, job_s = bench.job_rate(local_s, steps=5, world=world, device="cpu")
    out[rank] = (rate, job_s)
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        for r in range(2):
            rate, job_s = out[r]
            assert job_s == 3.0                        # slowest rank
            assert abs(rate - 2 * 5 / 3.0) < 1e-12     # every rank's steps over the job time


def test_job_rate_single_rank():
    import bench
    rate, job_s = bench.job_rate(0.5, steps=4, world=1)
    assert job_s == 0.5 and rate == 8.0


def test_traffic_record_requires_same_source_and_shape(tmp_path, monkeypatch):
    """The roofline's traffic figure is reported only for the kernel source and launch shape
    it was captured with."""
    import bench
    rec = bench.TRAFFIC_RECORDS[0]
    assert bench.traffic_of(rec["workload"], rec["precision"], rec["shape"]) == rec["bytes_per_launch"]
    assert bench.traffic_of(rec["workload"], rec["precision"], [1, 8192, 1]) is None
    assert bench.traffic_of("config3", rec["precision"], rec["shape"]) is None
    # another band.cu: no record
    fake = tmp_path / "paper_2509_06673_gb300" / "csrc"
    fake.mkdir(parents=True)
    (fake / "band.cu").write_text("// changed\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_of(rec["workload"], rec["precision"], rec["shape"]) is None
