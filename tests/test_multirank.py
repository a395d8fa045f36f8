"""The multi-process path without a GPU: two gloo ranks on the CPU.  Each rank draws its own data
segment (independent seeds, same shapes: weak scaling), and the step time and work are combined
the way the bench combines them (maximum time, summed work)."""
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


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_1810_09784_gb300 import ranks, workloads
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        r, w, lr = ranks.rank_env()
        spec, pm, grids = workloads.plain_small(seed=ranks.rank_seed(1, r))
        x = spec.series()[:4096]
        ms, work = ranks.combine(10.0 + 5.0 * r, 1000.0 * (r + 1))
        out[rank] = (r, w, lr, spec.seed, float(x[:16].sum()), len(grids), grids[0]["n_k"],
                     spec.n_fft, ms, work)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
        res = [out[0], out[1]]
    (r0, w0, l0, s0, x0, g0, k0, n0, ms0, wk0), (r1, w1, l1, s1, x1, g1, k1, n1, ms1, wk1) = res
    assert (r0, r1, w0, w1, l0, l1) == (0, 1, 2, 2, 0, 1)
    assert s0 != s1 and x0 != x1                 # independent segments
    assert (g0, k0, n0) == (g1, k1, n1)           # of the same shape: weak scaling
    assert ms0 == ms1 == 15.0                     # the step time is the slowest rank's
    assert wk0 == wk1 == 3000.0                   # the work is the whole job's


def test_single_process_combine_is_identity():
    from paper_1810_09784_gb300 import ranks
    assert ranks.combine(3.5, 7.0) == (3.5, 7.0)
    assert ranks.rank_seed(2, 0) == 2 and ranks.rank_seed(2, 3) == 2 + 3 * ranks.SEED_STRIDE
