"""Multi-rank path on CPU (gloo, world size 2): rows shard with no data-path
collective; the timing reduction is a max over ranks.  Each rank transforms
its own row range (host emulation of the kernels) and rank 0 checks the
union against the oracle."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2410_05934_gb300 import shard  # noqa: E402


def test_shard_rows_partitions():
    for total in (0, 1, 7, 96, 1000):
        for world in (1, 2, 3, 8):
            ranges = [shard.shard_rows(total, r, world) for r in range(world)]
            covered = []
            for b, c in ranges:
                covered += list(range(b, b + c))
            assert covered == list(range(total))
            counts = [c for _, c in ranges]
            assert max(counts) - min(counts) <= 1
    with pytest.raises(ValueError):
        shard.shard_rows(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, result_dir):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    sys.path.insert(0, os.path.join(root, "tests"))
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        from paper_2410_05934_gb300 import shard as S
        from paper_2410_05934_gb300 import workloads as W
        import emu
        log2n, mods, batch = 10, [W.POOL50[0], W.POOL50[1], W.POOL50[2]], 5
        rows = batch * len(mods)
        x = W.rows_uniform(11, 1, [mods[r % 3] for r in range(rows)], 1 << log2n)
        b, c = S.shard_rows(rows, rank, world)
        plan = emu.EmuPlan(log2n, mods, batch)
        out = x.copy()
        plan.transform(x, 0, out=out, row_begin=b, n_rows=c)
        np.save(os.path.join(result_dir, "rank%d.npy" % rank), out[b:b + c])
        t = S.max_over_ranks(0.25 + rank)
        S.barrier()
        with open(os.path.join(result_dir, "max%d.txt" % rank), "w") as f:
            f.write(repr(t))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo(tmp_path, oracle):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    from paper_2410_05934_gb300 import workloads as W
    mods = [W.POOL50[0], W.POOL50[1], W.POOL50[2]]
    per_row = [mods[r % 3] for r in range(15)]
    x = W.rows_uniform(11, 1, per_row, 1024)
    got = np.concatenate([np.load(os.path.join(tmp_path, "rank%d.npy" % r)) for r in range(world)])
    assert np.array_equal(got, oracle.transform_rows(x, per_row))
    for r in range(world):
        assert float(open(os.path.join(tmp_path, "max%d.txt" % r)).read()) == 1.25
