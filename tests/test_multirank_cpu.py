"""Multi-rank host logic of bench.py on CPU: two gloo ranks (no GPU)."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    from paper_2606_17212_b300 import synth
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    w = synth.config("c1_plain_4k", n_states=6)
    masks = bench.rank_states(w, rank)
    # data-parallel gradient: views into one flat buffer, summed over the ranks
    import torch
    grads = {"mu0": torch.zeros(5, 3), "logit": torch.zeros(7), "res": torch.zeros(2, 3, 4)}
    views, flat = bench.flat_gradients(grads, device="cpu")
    for k, v in views.items():
        v.fill_(float(rank + 1))
    bench.reduce_gradients(flat)
    summed = {k: v.clone().numpy() for k, v in views.items()}
    out[rank] = (masks.copy(), bench.max_over_ranks(10.0 * (rank + 1)), summed)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_states_and_take_the_max_time():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        (m0, t0, g0), (m1, t1, g1) = out[0], out[1]
    assert m0.shape == m1.shape and not np.array_equal(m0, m1)   # each rank its own states
    assert t0 == t1 == 20.0                                        # max over ranks
    for k in g0:                                                   # 1 + 2 on every element, both ranks
        assert np.all(g0[k] == 3.0) and np.all(g1[k] == 3.0), k
