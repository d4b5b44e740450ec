"""bench.py on CPU: the N > 1 path with world-size-2 gloo ranks, each timing its own replica
(the job rate uses the slowest rank's time, MAX over ranks, and counts every rank's steps); the
JSON line of the reference arm (the oracle on the host cores) and its rank-0-only rule."""
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


def _bench(args, env_extra=None):
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(root, "bench.py")] + args, capture_output=True,
                          text=True, timeout=900, env=env, cwd=root)


def test_reference_arm_json_line():
    """`bench.py --impl reference` times the oracle on a bounded sample and prints one JSON line
    with the contract's keys; the reference line reports no host<->device bytes."""
    import json
    r = _bench(["--impl", "reference", "--config", "config5", "--steps", "1", "--warmup", "3"])
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "config5" in d["config"]["workload"]


def test_reference_arm_other_ranks_exit_quietly():
    r = _bench(["--impl", "reference", "--steps", "1", "--warmup", "3"], {"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0 and not r.stdout.strip(), (r.returncode, r.stdout, r.stderr)


def test_traffic_record_keyed_on_solve_section(tmp_path, monkeypatch):
    """The traffic record follows the band solve's source only: an edit above the solve's section
    of band.cu (the factorisation) keeps it, an edit inside the section drops it."""
    import bench
    rec = bench.TRAFFIC_RECORDS[0]
    src = open(os.path.join(bench.ROOT, "paper_2509_06673_gb300", "csrc", "band.cu"), "rb").read()
    i = src.find(bench._SOLVE_MARK)
    assert i > 0
    fake = tmp_path / "paper_2509_06673_gb300" / "csrc"
    fake.mkdir(parents=True)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (fake / "band.cu").write_bytes(b"// factorisation edited\n" + src[i:])
    assert bench.traffic_of(rec["workload"], rec["precision"], rec["shape"]) == rec["bytes_per_launch"]
    (fake / "band.cu").write_bytes(src[i:] + b"// solve edited\n")
    assert bench.traffic_of(rec["workload"], rec["precision"], rec["shape"]) is None
