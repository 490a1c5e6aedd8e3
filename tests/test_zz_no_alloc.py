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


def test_noalloc_rejects_requests_beyond_its_scratch(env):
    S, torch = env
    dev = torch.device("cuda", 0)
    E = torch.zeros((300_000, 128), device=dev)
    Q = torch.zeros((4096, 128), device=dev)
    ids = torch.empty((4096, 10), dtype=torch.int64, device=dev)
    sc = torch.empty((4096, 10), dtype=torch.float32, device=dev)
    assert S.noalloc_query_topk(E, None, Q, 10, ids, sc) == S.ERR_CAPACITY
    assert S.noalloc_query_topk(E, None, Q[:2], 0, ids, sc) == S.ERR_INVALID_ARG
