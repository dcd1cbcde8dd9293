"""Multi-rank path on CPU (gloo, world size 2): ranks own disjoint slice
ranges, solve them independently (here with the oracle, on the host), and
the gathered result equals the single-process solve of the whole batch;
the timing reduction takes the slowest rank."""
import os

import numpy as np
import pytest


def _worker(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle as O
        from paper_2412_07631_b300 import replicas, synth
        k = 2
        first, seed = replicas.rank_slices(rank, world, k, 1234)
        g = O.Geometry(12, 20, 18, sqrt_lambda=0.05)
        csr = O.siddon_csr(g)
        X = synth.phantom_batch(12, k, 6, seed)
        B = O.forward(csr, X)
        Xs, _, _ = O.qr_solve(g, O.dense_system(g, csr), np.asarray(B))
        t = replicas.max_over_ranks(1.0 + rank, dist)
        full = replicas.gather_slices(torch.from_numpy(np.ascontiguousarray(Xs.T)), dist)
        if rank == 0:
            np.save(os.path.join(out_dir, "gathered.npy"), full.numpy())
            np.save(os.path.join(out_dir, "tmax.npy"), np.array([t]))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_slices(tmp_path):
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    import oracle as O
    from paper_2412_07631_b300 import synth
    g = O.Geometry(12, 20, 18, sqrt_lambda=0.05)
    csr = O.siddon_csr(g)
    X = synth.phantom_batch(12, 4, 6, 1234)  # the 4 slices of both ranks, seeds 1234..1237
    Xs, _, _ = O.qr_solve(g, O.dense_system(g, csr), np.asarray(O.forward(csr, X)))
    got = np.load(tmp_path / "gathered.npy")
    np.testing.assert_allclose(got, Xs.T, rtol=0, atol=1e-12 * np.abs(Xs).max())
    assert float(np.load(tmp_path / "tmax.npy")[0]) == 2.0


def test_rank_slices():
    from paper_2412_07631_b300 import replicas
    assert replicas.rank_slices(0, 4, 512, 1234) == (0, 1234)
    assert replicas.rank_slices(3, 4, 512, 1234) == (1536, 1234 + 1536)
    with pytest.raises(ValueError):
        replicas.rank_slices(4, 4, 512, 1234)
