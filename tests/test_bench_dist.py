"""The benchmark's multi-replica logic on CPU ranks (gloo, world size 2):
environment parsing, the max-over-ranks timing, the whole-job rate, and the
reference arm's rank-0-only rule.  The GPU path itself runs one replica per
GPU with no data-path collective, so these are its only cross-rank steps."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    r, local, ws, dist = bench.dist_setup()
    assert (r, local, ws) == (rank, rank, world) and dist is not None
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(dist, 10.0 + 5.0 * rank, "cpu")
        rate = bench.job_rate(1000, ws, 4, t)
        with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as f:
            f.write("%r %r\n" % (t, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    for rank in (0, 1):
        t, rate = map(float, open(tmp_path / ("rank%d.txt" % rank)).read().split())
        assert t == 15.0                         # the slower rank's time, on both
        assert rate == 2 * 1000 * 4 / 0.015       # both replicas' units over that time


def test_single_rank_needs_no_process_group(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    assert bench.dist_setup() == (0, 0, 1, None)
    assert bench.max_over_ranks(None, 12.5, "cpu") == 12.5
    assert bench.job_rate(100, 1, 10, 1000.0) == 1000.0


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        workload = "blobs64"
        steps = warmup = 1
        gpus = 2
        ref_budget = 0.05

    bench.run_reference(Args(), rank=1)           # other ranks exit without work
    assert capsys.readouterr().out == ""


def _rank_fail_main(rank, world, port, out_dir):
    """Rank 1 joins the group and then dies before the timing collective, as a
    failed replica would; rank 0 must get an error from its collective within
    the process group's timeout instead of waiting for ever."""
    import datetime
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    _, _, ws, dist = bench.dist_setup()
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=20))
    if rank == 1:
        os._exit(3)
    try:
        bench.max_over_ranks(dist, 10.0, "cpu")
        result = "no error"
    except Exception as e:  # the collective fails: peer gone or timed out
        result = "error " + type(e).__name__
    with open(os.path.join(out_dir, "rank0.txt"), "w") as f:
        f.write(result)
    os._exit(0)


@pytest.mark.timeout(120)
def test_failed_replica_is_detected_not_waited_for(tmp_path):
    pytest.importorskip("torch")
    import multiprocessing
    sp = multiprocessing.get_context("spawn")
    port = _free_port()
    procs = [sp.Process(target=_rank_fail_main, args=(r, 2, port, str(tmp_path))) for r in (0, 1)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=90)
    assert [p.exitcode for p in procs] == [0, 3]
    assert open(tmp_path / "rank0.txt").read().startswith("error")


def test_profiled_bench_commands_parse():
    """Every bench.py argument list that the ncu summaries were captured from
    (bench.PROFILE_COMMANDS, which the summaries name) parses with the
    benchmark's own argument parser."""
    import shlex
    sys.path.insert(0, ROOT)
    import bench
    parser = bench.make_parser()
    assert len(bench.PROFILE_COMMANDS) >= 5
    for name, argv in bench.PROFILE_COMMANDS.items():
        parser.parse_args(shlex.split(argv))
