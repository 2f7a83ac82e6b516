"""Multi-rank host logic on CPU: two gloo ranks take disjoint shares of the
independent units, draw independent wall-source propagators, agree on the
slowest rank's time and on the whole-job throughput; a rank that fails
between steps is detected by the other at the next barrier."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import synth
        from paper_1510_00903_gb300 import shard
        mine = shard.units_of_rank(11, rank, world)
        shares = [None] * world
        dist.all_gather_object(shares, mine)
        F = synth.flavour_set(2, 4, 0, 0.3, 0.4, **shard.rank_source(rank), times=[1])
        sums = [None] * world
        dist.all_gather_object(sums, complex(F["u"].sum()))
        shard.barrier(world)
        ms_local = 10.0 + 5.0 * rank
        ms = shard.max_over_ranks(ms_local, world)
        v = shard.job_throughput(1000, world, ms)
        vals = [None] * world
        dist.all_gather_object(vals, v)
        q.put((rank, shares, sums, ms, vals))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, shares, sums, ms, vals in res:
        flat = sorted(u for s in shares for u in s)
        assert flat == list(range(11))                       # every unit once
        assert set(shares[0]).isdisjoint(shares[1])
        assert sums[0] != sums[1]                            # independent sources
        assert ms == 15.0                                    # slowest rank
        assert vals[0] == vals[1] == pytest.approx(2 * 1000 / 0.015)


def test_shard_single_rank_and_errors():
    from paper_1510_00903_gb300 import shard
    assert shard.units_of_rank(5, 0, 1) == [0, 1, 2, 3, 4]
    assert shard.units_of_rank(0, 1, 2) == []
    assert shard.max_over_ranks(3.5, 1) == 3.5
    assert shard.job_throughput(100, 1, 50.0) == pytest.approx(2000.0)
    with pytest.raises(ValueError):
        shard.units_of_rank(4, 2, 2)
    with pytest.raises(ValueError):
        shard.job_throughput(1, 1, 0.0)
    k0, k1 = shard.rank_source(0), shard.rank_source(1)
    assert k0 != k1 and np.isscalar(k0["seed"])


def _failing_rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1510_00903_gb300 import shard
    shard.barrier(world, timeout_s=30)      # step 1: both ranks arrive

    def report_and_exit(msg, code):
        q.put((rank, msg))
        q.close()
        q.join_thread()                     # the message is out before the process ends
        os._exit(code)

    if rank == 1:
        report_and_exit("failed", 3)        # fails between steps, never reaches the next barrier
    try:
        shard.barrier(world, timeout_s=3)
        msg = "no error"
    except RuntimeError as e:
        msg = "detected: " + str(e)
    report_and_exit(msg, 0)


def test_failed_rank_is_detected_at_the_next_barrier():
    """Host-side failure detection (no GPU): rank 1 exits between steps; rank 0's
    monitored barrier ends with an error naming rank 1 instead of hanging."""
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_failing_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
    assert res[1] == "failed"
    assert res[0].startswith("detected") and "1" in res[0], res[0]
    assert procs[1].exitcode == 3 and procs[0].exitcode == 0
