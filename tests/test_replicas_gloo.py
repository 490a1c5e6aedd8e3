"""The N>1 path on CPU: world size 2 over gloo, no GPU.

The paper scales the Semantic Embedding stage by giving each GPU a subset of
the views and summing the per-GPU aggregation tensors ("Scaling semantic
embedding to a multi-GPU environment"). The bench runs one replica per GPU
(weak scaling); these tests check the two host-side pieces that N>1 relies
on: that view-sharded partial sums reduce to the whole-scene sums, and that
the bench's timing is the max over ranks with whole-job throughput."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import sys
    import torch
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import synth
    from oracle import oracle as O
    import bench

    scene = synth.config_tiny(seed=3)
    views = [scene.view(i) for i in range(scene.n_views)]
    # this rank's views: the shard a GPU would own
    num, den, _ = O.lift(scene.gaussians, views[rank::world])
    t_num = torch.from_numpy(num)
    t_den = torch.from_numpy(den)
    dist.all_reduce(t_num, op=dist.ReduceOp.SUM)
    dist.all_reduce(t_den, op=dist.ReduceOp.SUM)

    # bench timing: every rank reports its own time; the line uses the slowest rank
    local_ms = 10.0 + 5.0 * rank
    ms = bench.max_over_ranks(local_ms, dist, "cpu")
    rate = bench.job_rate(1000.0, world, ms / 1e3)
    if rank == 0:
        np.savez(os.path.join(out_dir, "r0.npz"), num=t_num.numpy(), den=t_den.numpy(), ms=ms, rate=rate)
    dist.barrier()
    dist.destroy_process_group()


def test_view_sharded_sums_reduce_to_the_whole_scene(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = np.load(tmp_path / "r0.npz")

    import synth
    from oracle import oracle as O
    scene = synth.config_tiny(seed=3)
    views = [scene.view(i) for i in range(scene.n_views)]
    num, den, _ = O.lift(scene.gaussians, views)
    assert den.sum() > 0
    # a sum of float64 partials in another order: equal to rounding
    np.testing.assert_allclose(r["den"], den, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(r["num"], num, rtol=1e-12, atol=1e-12)
    E_sharded = O.normalise(r["num"], r["den"])
    E_whole = O.normalise(num, den)
    np.testing.assert_allclose(E_sharded, E_whole, rtol=1e-10, atol=1e-12)

    # the slowest rank sets the time; throughput counts every rank's work
    assert float(r["ms"]) == 15.0
    assert float(r["rate"]) == pytest.approx(1000.0 * world / 0.015)
