"""The multi-GPU path of bench.py is replicas only: each rank solves its own
incidence direction and the ranks exchange nothing but the final timing
(max) and work (sum).  This runs that host logic as two gloo ranks on CPU."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    khat, pols = bench.replica_incidence(rank)
    ms, totals = bench.reduce_over_ranks(dist, 100.0 + 10 * rank, [400 + rank, 2], "cpu")
    out[rank] = (list(khat), [list(p) for p in pols], ms, totals)
    dist.destroy_process_group()


def test_two_gloo_replicas():
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
    k0, p0, ms0, t0 = out[0]
    k1, p1, ms1, t1 = out[1]
    # each replica has its own unit incidence direction with orthonormal polarisations
    assert not np.allclose(k0, k1)
    for k, pols in ((k0, p0), (k1, p1)):
        assert abs(np.linalg.norm(k) - 1) < 1e-12
        for e in pols:
            assert abs(np.dot(e, k)) < 1e-12 and abs(np.linalg.norm(e) - 1) < 1e-12
        assert abs(np.dot(pols[0], pols[1])) < 1e-12
    # whole-job figures: slowest rank's time, summed work, identical on both ranks
    assert ms0 == ms1 == 110.0
    assert t0 == t1 == [801.0, 4.0]


def test_single_process_reduction_is_identity():
    import bench
    assert bench.reduce_over_ranks(None, 12.5, [3, 4], "cpu") == (12.5, [3.0, 4.0])
