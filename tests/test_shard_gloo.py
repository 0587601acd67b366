"""Tree-sharded forests across processes (CPU, gloo, world size 2): each rank grows its own tree
range with the oracle, the ranks all-reduce their exact int64 per-query leaf sums, and the
rounded mean equals the single-process forest's prediction. This is the exchange step
bench.py performs with NCCL when it runs on several GPUs."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

T_PER_RANK = 4


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    from paper_1811_00156_gb300 import synth
    wl = synth.small_case(90, 700, 8, card=15)
    Xq = synth.small_case(91, 257, 8, card=15).X
    part = O.fit(wl.X, wl.y, T_PER_RANK, 3, 2, seed=4, t0=rank * T_PER_RANK, t1=(rank + 1) * T_PER_RANK)
    _, s = part.predict(Xq, total_trees=world * T_PER_RANK)
    t = torch.from_numpy(s.copy())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    T = world * T_PER_RANK
    pred = [(2 * int(v) + T) // (2 * T) for v in t.tolist()]
    np.save(os.path.join(out_dir, f"pred{rank}.npy"), np.array(pred, np.int64))
    dist.destroy_process_group()


def test_tree_shards_allreduce_equals_full_forest(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    import oracle as O
    from paper_1811_00156_gb300 import synth
    wl = synth.small_case(90, 700, 8, card=15)
    Xq = synth.small_case(91, 257, 8, card=15).X
    full = O.fit(wl.X, wl.y, world * T_PER_RANK, 3, 2, seed=4)
    exp, _ = full.predict(Xq)
    for r in range(world):
        assert np.array_equal(np.load(tmp_path / f"pred{r}.npy"), exp)
