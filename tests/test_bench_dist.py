"""The multi-rank path of bench.py on CPU (gloo, world size 2): each rank
runs an independent replica, the job's time is the slowest rank's and its
work the sum over the ranks; the reference arm runs on rank 0 only."""
import os
import socket
import types

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _replica(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench as b
    r, w, local = b.dist_env()
    ms = 10.0 * (rank + 1)  # rank 1 is the slow one
    slowest = b.max_over_ranks(ms, dist, "cpu")
    rate = b.job_rate(1e9, w, slowest * 1e-3)
    q.put((rank, r, w, local, slowest, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_sum_the_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_replica, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, r, w, local, slowest, rate in out:
        assert (r, w, local) == (rank, 2, rank)
        assert slowest == 20.0
        assert rate == pytest.approx(2 * 1e9 / 0.020 / 1e9)


def test_single_process_needs_no_group():
    assert bench.max_over_ranks(7.5, None, "cpu") == 7.5
    assert bench.job_rate(3e9, 1, 1.5) == pytest.approx(2.0)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    args = types.SimpleNamespace(seed=2, nnz=1000, rank=16, steps=1, warmup=0, gpus=2)
    assert bench.reference_arm(args, 1, 2) is None  # rank 1: no work, no output
    assert capsys.readouterr().out == ""


def test_byte_models_take_the_factor_element_size():
    # the byte model of one root-mode MTTKRP: 8 bytes per non-zero, 8 per
    # upper-level fiber, each distinct factor row once per level (s_f bytes
    # per element), the FP32 output; the "every gather" model counts a row
    # per fiber and leaf below the root
    csf = types.SimpleNamespace(nmodes=3, nfibs=[5, 40, 100], order=[2, 0, 1], root=2)
    dims, R, distinct = [30, 20, 5], 16, [25, 18, 5]
    for s_f in (4, 2):
        want = 100 * 8 + (5 + 40) * 8 + (distinct[0] + distinct[1]) * R * s_f + dims[2] * R * 4
        assert bench.byte_model(csf, dims, R, distinct, s_f) == want
        assert bench.every_gather_model(csf, R, s_f) == (40 + 100) * R * s_f
    assert bench.flop_model(csf, R) == 2 * R * (100 + 40)


def test_bench_accepts_the_gather_precision(monkeypatch):
    monkeypatch.setattr("sys.argv", ["bench.py", "--precision", "bf16", "--steps", "2"])
    a = bench.parse()
    assert a.precision == "bf16" and a.steps == 2 and a.e2e_steps == 3
    monkeypatch.setattr("sys.argv", ["bench.py"])
    assert bench.parse().precision == "fp32"
