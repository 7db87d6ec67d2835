"""Weak scaling over ranks, on CPU with the gloo backend (world size 2): every
rank runs its own box (its own seed), the timed region's length is the
slowest rank's, the whole-job rate counts all ranks' units, and the
reference arm runs on rank 0 only."""
import io
import os
import socket
import contextlib

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1912_04457_gb300 import inputs as I
    t_max = bench.max_over_ranks(1.0 + 0.5 * rank, world)
    w = I.qgp_box(n=8, seed=bench.rank_seed(2, rank))
    state_sum = int(w.state().sum())
    rate = bench.whole_job_rate(1000, 4, world, t_max)

    class Args:
        workload, steps, warmup, gpus = "gluon_step", 1, 0, world
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        rc = bench.run_reference(Args()) if rank != 0 else 0
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, t_max, state_sum, rate, rc, buf.getvalue()))


def test_two_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, s0, v0, rc0, o0), (r1, t1, s1, v1, rc1, o1) = res
    assert t0 == t1 == 1.5                    # the slowest rank's time on every rank
    assert v0 == v1 == pytest.approx(1000 * 4 * 2 / 1.5)
    assert s0 != s1                           # each rank samples its own box
    assert rc1 == 0 and o1 == ""              # the reference arm does no work off rank 0
    assert bench_seed_is_rank0_identity()


def bench_seed_is_rank0_identity():
    import bench
    return bench.rank_seed(7, 0) == 7 and bench.rank_seed(7, 1) != 7
