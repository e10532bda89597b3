"""The multi-rank (replicas) path with two gloo ranks on the CPU: sharding,
max-over-ranks timing and the optional output all-gather, with each rank's
shard evaluated by the oracle (the GPU kernels need a GPU)."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch
    import torch.distributed as dist
    import oracle
    import synth
    from paper_1809_01029_gb300 import replicas
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m = synth.make_mechanism("h2co13")
        n = 37
        phi, par = synth.make_states(m, n, 4, synth.CONP)
        lo, hi = replicas.shard(n, world, rank)
        f_local = oracle.source_terms(m, synth.CONP, phi[:, lo:hi], par[lo:hi])
        f_all = replicas.gather_states(torch.from_numpy(f_local), n, dist).numpy()
        t_max = replicas.max_over_ranks(10.0 + rank, dist)
        # adjoint parameter gradient: per-shard sums, all-reduced
        uw, uT = synth.make_cotangents(m.n_species, n, 6)
        _, g_th = oracle.vjp(m, synth.CONP, phi[:, lo:hi], par[lo:hi], uw[:, lo:hi], uT[lo:hi])
        g_all = replicas.allreduce_sum(torch.from_numpy(np.ascontiguousarray(g_th)), dist).numpy()
        q.put((rank, lo, hi, f_all, t_max, g_all))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_gather_and_time():
    import torch.multiprocessing as mp
    import oracle
    import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort(key=lambda x: x[0])
    (_, lo0, hi0, f0, t0, g0), (_, lo1, hi1, f1, t1, g1) = res
    assert (lo0, hi0, lo1, hi1) == (0, 19, 19, 37)
    assert t0 == t1 == 11.0
    m = synth.make_mechanism("h2co13")
    phi, par = synth.make_states(m, 37, 4, synth.CONP)
    ref = oracle.source_terms(m, synth.CONP, phi, par)
    assert np.array_equal(f0, f1)
    assert np.allclose(f0, ref, rtol=1e-13, atol=0)
    uw, uT = synth.make_cotangents(m.n_species, 37, 6)
    _, g_ref = oracle.vjp(m, synth.CONP, phi, par, uw, uT)
    assert np.array_equal(g0, g1)
    assert np.allclose(g0, g_ref, rtol=1e-12, atol=1e-12 * np.abs(g_ref).max())


@pytest.mark.parametrize("n,world", [(0, 3), (1, 4), (10, 3), (1048576, 8)])
def test_shards_cover_batch_disjointly(n, world):
    from paper_1809_01029_gb300 import replicas
    spans = [replicas.shard(n, world, r) for r in range(world)]
    assert spans[0][0] == 0 and spans[-1][1] == n
    for (a, b), (c, d) in zip(spans, spans[1:]):
        assert b == c and b >= a
    sizes = [b - a for a, b in spans]
    assert max(sizes) - min(sizes) <= 1
