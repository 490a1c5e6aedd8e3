"""The N>1 path on CPU: world size 2 over gloo, no GPU.

The paper scales the Semantic Embedding stage by giving each GPU a subset of
the views and summing the per-GPU aggregation tensors ("Scaling semantic
embedding to a multi-GPU environment"). The bench runs one replica per GPU
(weak scaling); these tests check the host-side pieces that N>1 relies on:
that view-sharded partial sums reduce to the whole-scene sums, that the
library's serialised states of view shards merge (slag_state_merge_host, no
GPU needed) into the state of every view, and that the bench's timing is the
max over ranks with whole-job throughput."""
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


def state_from_views(g, views, fingerprint):
    """A state in the library's format (slag_save_state) for these views, its weights from the
    oracle: every non-zero B_v[k][j] becomes a triple (k, column of (v, j), float32 W) and the sum
    of w per Gaussian goes to the hi plane."""
    from oracle import oracle as O
    from paper_2505_08124_b300 import slag as S
    n, D = g.n, views[0].table.shape[1]
    tables, gs, cs, ws = [], [], [], []
    den = np.zeros(n)
    col0 = 0
    contrib = 0
    for v in views:
        r = O.view_weights(g, v)
        k, j = np.nonzero(r["B"])
        gs.append(k.astype(np.uint32))
        cs.append((j + col0).astype(np.uint32))
        ws.append(r["B"][k, j].astype(np.float32))
        den += r["B"].sum(1)
        tables.append(v.table.astype(np.float32))
        col0 += v.table.shape[0]
        contrib += r["contributions"]
    z = int(sum(len(x) for x in gs))
    h = np.zeros(1, S.STATE_HEADER)
    h["magic"], h["version"], h["dim"], h["n"] = b"SLAGSTAT", 1, D, n
    h["columns"], h["triples"], h["fingerprint"], h["views"] = col0, z, fingerprint, len(views)
    h["contributions"] = contrib
    sums = np.zeros((3, n), np.float32)
    sums[0] = den.astype(np.float32)
    parts = [h.tobytes(), np.concatenate(tables).tobytes(), sums.tobytes(), np.concatenate(gs).tobytes(),
             np.concatenate(cs).tobytes(), np.concatenate(ws).tobytes()]
    return b"".join(parts)


def state_embeddings(state):
    """E and sum w implied by a state: sum over triples of W times the column's embedding, over
    the compensated sum of w."""
    from paper_2505_08124_b300 import slag as S
    st = S.read_state(state)
    n = int(st["header"]["n"])
    num = np.zeros((n, st["table"].shape[1]))
    np.add.at(num, st["gauss"].astype(np.int64), st["w"].astype(np.float64)[:, None] *
              st["table"][st["column"].astype(np.int64)].astype(np.float64))
    den = st["w_hi"].astype(np.float64) + st["w_lo"] + st["w_ovf"]
    E = np.zeros_like(num)
    ok = den > 0
    E[ok] = num[ok] / den[ok, None]
    return E, den


def _state_rank_main(rank, world, port, out_dir):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import synth
    from paper_2505_08124_b300 import slag as S
    scene = synth.config_tiny(seed=3)
    views = [scene.view(i) for i in range(scene.n_views)]
    # this rank's shard of the views, serialised as the library saves a context's state
    with open(os.path.join(out_dir, "state_%d.bin" % rank), "wb") as f:
        f.write(state_from_views(scene.gaussians, views[rank::world], fingerprint=0x5eed))
    dist.barrier()
    if rank == 0:
        merged = open(os.path.join(out_dir, "state_0.bin"), "rb").read()
        for r in range(1, world):
            merged = S.state_merge_host(merged, open(os.path.join(out_dir, "state_%d.bin" % r), "rb").read())
        with open(os.path.join(out_dir, "merged.bin"), "wb") as f:
            f.write(merged.tobytes())
    dist.barrier()
    dist.destroy_process_group()


def test_view_sharded_states_merge_to_the_whole_scene(tmp_path):
    world = 2
    mp.spawn(_state_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    merged = open(tmp_path / "merged.bin", "rb").read()
    import synth
    from oracle import oracle as O
    from paper_2505_08124_b300 import slag as S
    scene = synth.config_tiny(seed=3)
    views = [scene.view(i) for i in range(scene.n_views)]
    hdr = S.read_state(merged)["header"]
    assert hdr["views"] == len(views) and hdr["columns"] == sum(v.m for v in views)
    num, den = O.lift(scene.gaussians, views)[:2]
    E, w = state_embeddings(merged)
    # float32 weights in the state: the float32 parity bar
    ok = den >= 1e-3
    assert ok.sum() > 100
    np.testing.assert_allclose(w, den, rtol=1e-6, atol=1e-9)
    Eo = O.normalise(num, den)
    assert np.linalg.norm(E - Eo) / np.linalg.norm(Eo) <= 1e-6
    # a state of another Gaussian set does not merge
    other = open(tmp_path / "state_1.bin", "rb").read()
    h = np.frombuffer(other[:96], S.STATE_HEADER).copy()
    h["fingerprint"] = 1
    with pytest.raises(S.SlagError):
        S.state_merge_host(merged, h.tobytes() + other[96:])


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
