"""The N > 1 benchmark path on CPU: two gloo ranks run the host logic that
bench.py runs under torchrun (per-rank inputs, max-over-ranks timing, the
whole-job throughput).  The query batches shard across ranks with no
data-path collective, so the only exchange is the timing reduction."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import types
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    r, w, local = bench.dist_env()
    assert (r, w, local) == (rank, world, rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    a = types.SimpleNamespace(n_db=3000, nq=50, dtype="u8")
    db, q = bench.make_inputs(a, rank)
    # rank r's timed region lasts 10 (r + 1) ms over 4 steps
    slowest = bench.max_over_ranks(10.0 * (rank + 1), world, "cpu")
    ms_per_step = slowest / 4
    value = bench.job_throughput(ms_per_step, a.nq, world)
    np.savez(os.path.join(out_dir, "rank%d.npz" % rank), db=db, q=q,
             slowest=slowest, value=value)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_gloo_ranks_weak_scaling(tmp_path):
    world = 2
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, str(tmp_path)))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(240)
        assert p.exitcode == 0
    res = [np.load(tmp_path / ("rank%d.npz" % r)) for r in range(world)]
    # every rank holds the same database and its own query batch
    assert np.array_equal(res[0]["db"], res[1]["db"])
    assert not np.array_equal(res[0]["q"], res[1]["q"])
    # both ranks see the slowest rank's time, and the value counts all ranks' queries
    for r in res:
        assert float(r["slowest"]) == 20.0
        assert float(r["value"]) == pytest.approx(2 * 50 / (5.0 / 1000.0))


def test_single_rank_throughput_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.job_throughput(2.0, 1000, 1) == pytest.approx(500_000.0)
