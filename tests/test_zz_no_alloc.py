"""The allocation-free query entry point, checked against the regular one.

slag_noalloc_query_topk is meant for callers that must not allocate device
memory once they are running (an embedded or on-robot query service that
reserves its memory at start-up, or an application whose device memory is
owned by its own allocator). It keeps its scratch in a fixed array inside the
library, so two calls in a row reuse the same memory: both must give the
answers of slag_query_batch on the same embeddings. This file is collected
last, so a run that stops at the first failure has run every other test.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2505_08124_b300 import build
    build.build()
    from paper_2505_08124_b300 import slag as S
    S.load_library()
    return S, torch


def _sep_mask(sc, margin):
    """Ranks whose score is more than `margin` away from both neighbours (ids must agree there)."""
    sep = np.ones(sc.shape, bool)
    gaps = np.abs(np.diff(sc, axis=1)) > margin
    sep[:, :-1] &= gaps
    sep[:, 1:] &= gaps
    return sep


def test_noalloc_query_matches_query_batch_twice(env):
    S, torch = env
    s = synth.small_scene(31, 8000, 3, 160, 120, 8, dim=256, surfaces=4)
    views = list(s.views())
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    with S.Lifter(s.gaussians, dim=256, stream=stream.cuda_stream) as L:
        for v in views:
            L.add_view(v.camera, v.seg, v.table)
        E = torch.empty((s.gaussians.n, 256), device=dev)
        w = torch.empty(s.gaussians.n, device=dev)
        L.finalize(E, w)
        rng = np.random.default_rng(5)
        for call, (B, k) in enumerate([(40, 10), (23, 64)]):
            Qn = rng.standard_normal((B, 256)).astype(np.float32)
            Qn /= np.linalg.norm(Qn, axis=1, keepdims=True)
            Q = torch.from_numpy(Qn).to(dev)
            ref_ids, ref_sc, ref_cnt = L.query_batch(Qn, k)
            ids = torch.full((B, k), -7, dtype=torch.int64, device=dev)
            sc = torch.full((B, k), -7.0, dtype=torch.float32, device=dev)
            cnt = torch.full((B,), -7, dtype=torch.int32, device=dev)
            rc = S.noalloc_query_topk(E, w, Q, k, ids, sc, cnt, stream=stream.cuda_stream)
            assert rc == S.OK, "call %d returned %d" % (call, rc)
            torch.cuda.synchronize()
            ids, sc, cnt = ids.cpu().numpy(), sc.cpu().numpy(), cnt.cpu().numpy()
            np.testing.assert_array_equal(cnt, ref_cnt)
            # the row norms are summed in another order than at finalize: scores agree to float32
            # rounding, and ids agree wherever the ranking is not a near-tie
            np.testing.assert_allclose(sc, ref_sc, atol=1e-5)
            sep = _sep_mask(ref_sc.astype(np.float64), 1e-5)
            np.testing.assert_array_equal(ids[sep], ref_ids[sep])


def _raw(S, E, n, dim, wsum, Q, B, k, ids, sc, cnt=None):
    """The C entry point itself, with raw addresses (no checks in the binding)."""
    import ctypes
    lib = S.load_library()
    addr = lambda x: None if x is None else ctypes.c_void_p(x)
    return lib.slag_noalloc_query_topk(addr(E), n, dim, addr(wsum), addr(Q), B, k, addr(ids), addr(sc), addr(cnt),
                                       None)


def test_noalloc_rejects_requests_beyond_its_scratch(env):
    S, torch = env
    dev = torch.device("cuda", 0)
    E = torch.zeros((300_000, 128), device=dev)
    Q = torch.zeros((4096, 128), device=dev)
    ids = torch.empty((4096, 10), dtype=torch.int64, device=dev)
    sc = torch.empty((4096, 10), dtype=torch.float32, device=dev)
    assert S.noalloc_query_topk(E, None, Q, 10, ids, sc) == S.ERR_CAPACITY
    assert _raw(S, E.data_ptr(), 300_000, 128, None, Q.data_ptr(), 2, 0, ids.data_ptr(), sc.data_ptr()) == \
        S.ERR_INVALID_ARG


def test_noalloc_refuses_host_memory_before_any_launch(env):
    S, torch = env
    dev = torch.device("cuda", 0)
    E = torch.randn((512, 128), device=dev)
    Qd = torch.randn((4, 128), device=dev)
    ids = torch.empty((4, 5), dtype=torch.int64, device=dev)
    sc = torch.empty((4, 5), dtype=torch.float32, device=dev)
    Qh = np.zeros((4, 128), np.float32)
    Qp = torch.zeros((4, 128)).pin_memory()
    ids_h = np.zeros((4, 5), np.int64)
    launches = S.kernel_launches()
    # pageable and pinned host queries, host outputs, a host weight sum: refused, nothing launched
    assert _raw(S, E.data_ptr(), 512, 128, None, Qh.ctypes.data, 4, 5, ids.data_ptr(), sc.data_ptr()) == \
        S.ERR_INVALID_ARG
    assert _raw(S, E.data_ptr(), 512, 128, None, Qp.data_ptr(), 4, 5, ids.data_ptr(), sc.data_ptr()) == \
        S.ERR_INVALID_ARG
    assert _raw(S, E.data_ptr(), 512, 128, None, Qd.data_ptr(), 4, 5, ids_h.ctypes.data, sc.data_ptr()) == \
        S.ERR_INVALID_ARG
    w_h = np.ones(512, np.float32)
    assert _raw(S, E.data_ptr(), 512, 128, w_h.ctypes.data, Qd.data_ptr(), 4, 5, ids.data_ptr(), sc.data_ptr()) == \
        S.ERR_INVALID_ARG
    assert S.kernel_launches() == launches
    # the binding refuses them too, before the library is called
    with pytest.raises(ValueError):
        S.noalloc_query_topk(E, None, Qp, 5, ids, sc)
    with pytest.raises(ValueError):
        S.noalloc_query_topk(E, None, Qd[:, :64].contiguous(), 5, ids, sc)
    with pytest.raises(ValueError):
        S.noalloc_query_topk(E, None, Qd, 5, ids[:, :4].contiguous(), sc)


def test_noalloc_candidates_with_and_without_weight_sums(env):
    # rows with wsum <= 0 are excluded when wsum is given even if their embedding is non-zero;
    # without wsum only zero rows are excluded. Checked against a numpy cosine top-k.
    S, torch = env
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(9)
    n, dim, B, k = 3000, 128, 6, 12
    En = rng.standard_normal((n, dim)).astype(np.float32)
    En[::7] = 0.0                                # zero rows: never candidates
    wn = rng.uniform(0.1, 2.0, n).astype(np.float32)
    wn[3::11] = 0.0                              # non-zero rows without weight
    Qn = rng.standard_normal((B, dim)).astype(np.float32)
    Qn /= np.linalg.norm(Qn, axis=1, keepdims=True)
    # the first query points at weightless rows, so that they would top its list if not excluded
    Qn[0] = En[3] / np.linalg.norm(En[3])
    E, w, Q = (torch.from_numpy(x).to(dev) for x in (En, wn, Qn))
    for use_w in (True, False):
        ids = torch.empty((B, k), dtype=torch.int64, device=dev)
        sc = torch.empty((B, k), dtype=torch.float32, device=dev)
        cnt = torch.empty(B, dtype=torch.int32, device=dev)
        assert S.noalloc_query_topk(E, w if use_w else None, Q, k, ids, sc, cnt) == S.OK
        torch.cuda.synchronize()
        nrm = np.linalg.norm(En.astype(np.float64), axis=1)
        ok = (nrm > 0) & ((wn > 0) if use_w else True)
        idx = np.nonzero(ok)[0]
        for b in range(B):
            s = (En[idx].astype(np.float64) @ Qn[b].astype(np.float64)) / nrm[idx]
            order = np.lexsort((idx, -s))[:k]
            want_ids, want_sc = idx[order], s[order]
            got_ids = ids[b].cpu().numpy()
            np.testing.assert_allclose(sc[b].cpu().numpy(), want_sc, atol=1e-5)
            sep = _sep_mask(want_sc[None, :], 1e-5)[0]
            np.testing.assert_array_equal(got_ids[sep], want_ids[sep])
            assert int(cnt[b].item()) == k
            if use_w:
                assert not np.isin(got_ids, np.nonzero(wn <= 0)[0]).any()
        if not use_w:
            assert int(ids[0, 0].item()) == 3    # the weightless row is a candidate without wsum
