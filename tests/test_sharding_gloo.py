"""The multi-rank path on CPU: world_size-2 gloo groups split the items of a
ragged batch (modular and contiguous partitions), each rank runs the CPU
oracle on its shard, results gather on rank 0 and equal a one-process run;
the timing reduction takes the max over ranks; a rank that fails before the
gather surfaces on the other rank as an error of that collective, within the
process group's timeout, instead of a hang."""
import datetime
import os
import socket
import time

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2003_02256_gb300 import sharding
from paper_2003_02256_gb300 import workloads as W


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, mode, out_path):
    import torch.distributed as dist

    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m, g = W.ragged_batch(n_models=6, layers=(3, 6), lambdas=(5, 12), grid=W.Grid(60.0, 1.0, 900))
    item_model = np.repeat(np.arange(m.n_models), m.n_lambda)
    mine = sharding.shard(m.n_items, rank, world, mode)
    ct = np.empty(mine.size)
    for t, it in enumerate(mine):
        h, a, b, r, _ = m.model(item_model[it])
        ct[t] = oracle.scan(h, a, b, r, m.lam[it], g.c0, g.dc, g.n_c)[1]
    full = sharding.gather(ct, mine, m.n_items)
    tmax = sharding.max_over_ranks(float(rank + 1))
    if rank == 0:
        np.save(out_path, np.r_[full, tmax])
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["modular", "contiguous"])
def test_two_rank_gloo_shards_gather_to_the_single_process_result(tmp_path, oracle_lib, mode):
    out = str(tmp_path / "res.npy")
    mp.spawn(_worker, args=(2, _port(), mode, out), nprocs=2, join=True)
    res = np.load(out)
    full, tmax = res[:-1], res[-1]
    m, g = W.ragged_batch(n_models=6, layers=(3, 6), lambdas=(5, 12), grid=W.Grid(60.0, 1.0, 900))
    ref, _, _ = oracle_lib.dispersion(m.as_dict(), g.c0, g.dc, g.n_c)
    assert np.array_equal(full, ref, equal_nan=True)
    assert tmax == 2.0


def test_partitions_cover_every_unit_once():
    for n in (0, 1, 7, 40, 41):
        for world in (1, 2, 3, 8):
            for mode in ("modular", "contiguous"):
                parts = [sharding.shard(n, r, world, mode) for r in range(world)]
                allidx = np.sort(np.concatenate(parts)) if parts else np.zeros(0)
                assert np.array_equal(allidx, np.arange(n))
    with pytest.raises(ValueError):
        sharding.shard(4, 2, 2)


def test_modular_partition_balances_a_variable_curve_better(oracle_lib):
    """Section 3.2: on a curve with decreasing wavelengths the per-wavelength
    work (determinants evaluated by Algorithm 1) trends with the index, so the
    modular partition beats the contiguous one at 3 and 8 ranks."""
    m, g = W.single_curve()
    h, a, b, r, _ = m.model(0)
    lam = sharding.variable_curve_wavelengths(40)
    work = []
    for l in lam:
        st, ct, idx = oracle_lib.scan(h, a, b, r, l, g.c0, g.dc, g.n_c)
        assert st == 0
        work.append(idx + 1)
    work = np.array(work)
    assert work[0] > work[-1]  # long wavelengths scan further
    for P in (3, 8):
        mod = sharding.partition_speedup(work, P, "modular")
        con = sharding.partition_speedup(work, P, "contiguous")
        assert mod > con
        assert mod <= P + 1e-12 and con <= P + 1e-12
    assert sharding.partition_speedup(work, 1) == 1.0


def _failing_worker(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=10))
    if rank == 1:
        raise RuntimeError("rank 1 fails before its shard is gathered")
    t0 = time.time()
    try:
        sharding.gather(np.zeros(3), np.arange(3), 6)
        status = "no-error"
    except Exception as e:  # the peer's failure reaches this rank through the collective
        status = "error:" + type(e).__name__
    with open(out_path, "w") as f:
        f.write(f"{status} {time.time() - t0:.2f}")


def test_a_failed_rank_surfaces_as_an_error_on_the_others(tmp_path):
    out = str(tmp_path / "status.txt")
    ctx = mp.start_processes(_failing_worker, args=(2, _port(), out), nprocs=2, join=False,
                             start_method="spawn")
    for proc in ctx.processes:
        proc.join(120)
    codes = [proc.exitcode for proc in ctx.processes]
    assert codes[1] not in (0, None), codes  # the failing rank
    status, elapsed = open(out).read().split()
    assert status.startswith("error:"), status
    assert float(elapsed) < 60.0


def test_timed_partition_study_on_cpu_ranks():
    """The timed CPU-rank study of Section 3.2 (spawned processes running the
    oracle on their shares) gathers exactly the one-rank indices for both
    partitions and reports a wall time and a speedup per rank count."""
    import bench
    out = bench.cpu_partition_study(ranks=(1, 2, 3), reps=2)
    assert set(out["ranks"]) == {"1", "2", "3"}
    for P, row in out["ranks"].items():
        for mode in ("contiguous", "modular"):
            assert row[mode]["wall_s"] > 0 and row[mode]["speedup"] > 0
            assert row[mode]["cost_model_speedup"] >= 1.0
    assert out["ranks"]["3"]["modular"]["cost_model_speedup"] > \
        out["ranks"]["3"]["contiguous"]["cost_model_speedup"]
