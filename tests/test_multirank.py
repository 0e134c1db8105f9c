"""The multi-rank (replica) path of the benchmark on CPU: world size 2 over gloo.

Every rank serves its own stream of events (rank-shifted seeds); the job's time is the slowest
rank's and its work the sum of the ranks' particle-steps, with no collective on the data path.
"""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, local = bench.dist_env()
    sizes, arrivals, offset = bench.replica_stream(rank, nevents=3)
    ev = bench.c4_event(0 + offset, int(sizes[0]))
    ms, units = bench.combine_ranks(100.0 + 50.0 * rank, float(ev.n * 10))
    out[rank] = (ws, r, ms, units, ev.n, float(ev.S.sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_combine_max_time_and_summed_work():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    (ws0, r0, ms0, u0, n0, s0), (ws1, r1, ms1, u1, n1, s1) = out[0], out[1]
    assert (ws0, ws1, r0, r1) == (2, 2, 0, 1)
    assert ms0 == ms1 == 150.0  # max over ranks
    assert u0 == u1 == float(n0 * 10 + n1 * 10)  # total particle-steps
    assert s0 != s1  # independent events (rank-shifted seeds)


def test_single_rank_is_identity():
    import bench
    assert bench.combine_ranks(12.5, 7.0) == (12.5, 7.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup, events = 1, 0, 3

    assert bench.run_reference(A()) == 0
    assert capsys.readouterr().out == ""
