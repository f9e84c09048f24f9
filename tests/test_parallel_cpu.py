"""Multi-rank sample sharding and the rank-ordered statistics merge, as world_size-2 gloo processes
on the CPU (no GPU): each rank takes its shard of the ensemble, computes its Welford accumulator,
the accumulators are all-gathered, and the rank-order merge equals the single-process statistics."""
import os

import numpy as np
import pytest

from paper_1912_07645_gb300.parallel import shard


def test_shard_ranges_cover_the_ensemble():
    for total in (0, 1, 7, 4096, 4099):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                f, c = shard(r, world, total)
                seen.extend(range(f, f + c))
            assert seen == list(range(total))
    with pytest.raises(ValueError):
        shard(2, 2, 10)


def _worker(rank, world, port, total, out_path):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_1912_07645_gb300.parallel import gather, shard
    from inputs import kh_theta
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    d = oracle.make_desc(ndim=2, n=(12, 10), eq="euler", recon="mc", flux="hllc", rk="ssprk2", cfl=0.4)
    th = kh_theta(total, 17)
    first, count = shard(rank, world, total)
    U = oracle.init(d, "kh", count, th[first:first + count])
    U, _, _ = oracle.evolve(d, U, T=0.02)
    c, m, M2 = oracle.welford(d, U)
    packed = torch.from_numpy(np.concatenate([[float(c)], m.ravel(), M2.ravel()]))
    gathered = gather(packed)
    if rank == 0:
        acc = (0, np.zeros_like(m), np.zeros_like(M2))
        for g in gathered:
            g = g.numpy()
            k = m.size
            acc = oracle.stats_merge(d, acc, (int(g[0]), g[1:1 + k].reshape(m.shape), g[1 + k:].reshape(m.shape)))
        np.savez(out_path, c=acc[0], m=acc[1], M2=acc[2])
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_rank_merge_equals_single_process(tmp_path):
    import socket

    import torch.multiprocessing as mp

    import oracle
    from inputs import kh_theta
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    total = 10      # 5 + 5: equal shards so the all-gather sizes agree
    out = str(tmp_path / "merged.npz")
    mp.start_processes(_worker, args=(2, port, total, out), nprocs=2, join=True, start_method="spawn")
    r = np.load(out)
    d = oracle.make_desc(ndim=2, n=(12, 10), eq="euler", recon="mc", flux="hllc", rk="ssprk2", cfl=0.4)
    U = oracle.init(d, "kh", total, kh_theta(total, 17))
    U, _, _ = oracle.evolve(d, U, T=0.02)
    c, m, M2 = oracle.welford(d, U)
    assert int(r["c"]) == c == total
    np.testing.assert_allclose(r["m"], m, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(r["M2"], M2, rtol=1e-11, atol=1e-14)
