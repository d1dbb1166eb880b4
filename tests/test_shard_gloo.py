"""Multi-rank host logic on CPU: two gloo ranks split one propagator set by sink-site
ranges, evaluate their partial correlators with the oracle and all-reduce them; the sum
equals the single-rank correlator.  Also the set partition used for weak scaling."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2201_04269_gb300 import shard  # noqa: E402


def test_site_range_partition():
    for n in (0, 1, 7, 512, 663552):
        for world in (1, 2, 3, 8):
            spans = [shard.site_range(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [e - b for b, e in spans]
            assert max(sizes) - min(sizes) <= 1
    assert list(shard.local_sets(64, 1, 4)) == list(range(16, 32))
    with pytest.raises(ValueError):
        shard.site_range(10, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import mbc_inputs as mi
    from oracle import correlator as ocor
    from oracle import operators as oops
    U, D = mi.workload_fields("proton_4x8")
    T, V3 = U.shape[:2]
    b, e = shard.site_range(V3, rank, world)
    plan = ocor.CanonicalPlan(oops.build("proton"))
    part = plan.site_values(U[:, b:e].reshape(-1, 12, 12), D[:, b:e].reshape(-1, 12, 12)).reshape(T, e - b)
    C = torch.from_numpy(part.sum(axis=1).copy())
    shard.allreduce_correlator(C)
    if rank == 0:
        np.save(out, C.numpy())
    dist.destroy_process_group()


def test_two_rank_site_split_allreduce(tmp_path):
    out = str(tmp_path / "c.npy")
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    got = np.load(out)
    import mbc_inputs as mi
    from oracle import correlator as ocor
    from oracle import operators as oops
    U, D = mi.workload_fields("proton_4x8")
    ref = ocor.CanonicalPlan(oops.build("proton")).site_values(U.reshape(-1, 12, 12), D.reshape(-1, 12, 12))
    ref = ref.reshape(U.shape[:2]).sum(axis=1)
    assert np.allclose(got, ref, rtol=1e-13, atol=0)
