"""Multi-rank bench logic on CPU (gloo, world size 2): every rank runs an
independent job on its own seeded corpus; the reported throughput is all
ranks' scanned bytes over the slowest rank's time."""
import os

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)

    def reduce_max(x):
        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    elapsed = [120.0, 150.0][rank]          # ms: rank 1 is the slowest
    value, t = bench.aggregate(elapsed, bytes_per_step=1_000_000, passes=6, steps=3, world=world,
                               reduce_max=reduce_max)
    out[rank] = (value, t, bench.rank_seed(7, rank))
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    (v0, t0, s0), (v1, t1, s1) = out[0], out[1]
    assert t0 == t1 == 150.0                       # max over ranks
    assert v0 == v1 == pytest.approx(2 * 1e6 * 6 * 3 / 0.150 / 1e9)
    assert s0 != s1                                 # independent corpora per rank


def test_reference_arm_prints_one_line(capsys):
    import json
    import bench
    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0", "--ref-mb", "1"]) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["value"] > 0
    assert line["ms_per_step"] > 0 and line["higher_is_better"] is True
