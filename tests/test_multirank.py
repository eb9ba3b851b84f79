"""Multi-process host logic on CPU (gloo, world size 2 and 3): the k-slab split
and the rank-ordered sum of paper_1710_10789_gb300.shard. The per-rank DOS is
computed by the oracle here (no GPU); the GPU side of each rank is the same
single-device path the GPU tests cover."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
import tbgen  # noqa: E402
from paper_1710_10789_gb300 import shard  # noqa: E402

N = (6, 5, 7)
NW = 200


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _problem():
    model = tbgen.tb_model(5, n_orb=4)
    eps, w = oracle.eig(model, *N)
    om = tbgen.uniform_grid(float(eps.min()) - 0.1, float(eps.max()) + 0.1, NW).astype(np.float64)
    return eps, w, om


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        eps, w, om = _problem()
        z0, z1 = shard.slab_ranges(N[2], world)[rank]
        if z1 > z0:
            local = oracle.dos(eps, w, *N, om, z_range=(z0, z1), nthreads=1)
        else:
            local = np.zeros((w.shape[2], NW))
        total = shard.gather_slabs(torch.from_numpy(local.astype(np.float32)))
        np.save(os.path.join(out_dir, f"rank{rank}.npy"), total.numpy())
    finally:
        dist.destroy_process_group()


def test_slab_ranges_cover_the_grid():
    for n3 in (1, 2, 7, 10, 256):
        for world in (1, 2, 3, 8, 12):
            r = shard.slab_ranges(n3, world)
            assert len(r) == world and r[0][0] == 0 and r[-1][1] == n3
            assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
            sizes = [b - a for a, b in r]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 0
    with pytest.raises(ValueError):
        shard.slab_ranges(0, 2)


@pytest.mark.parametrize("world", [2, 3])
def test_slab_sum_over_gloo_ranks(tmp_path, world):
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    eps, w, om = _problem()
    full = oracle.dos(eps, w, *N, om, nthreads=1)
    res = [np.load(tmp_path / f"rank{r}.npy") for r in range(world)]
    for r in res[1:]:
        assert np.array_equal(r, res[0])          # every rank gets the same bits
    assert np.max(np.abs(res[0] - full)) <= 1e-6 * np.max(np.abs(full))
