"""The batched form: several independent scenes in one call, and the query
path's autotuned split and CUDA-graph replay.

slag_add_views_batched adds the scenes one after another and queues each
scene's last second half before the next; each scene's result must be that of
adding its views alone. Device-side queries
replay a captured CUDA graph and must return what a fresh launch returns,
also after the embeddings change (a new finalize), and with the autotuner on
or off."""
import numpy as np
import pytest

import synth
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def slag():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2505_08124_b300 import build
    build.build()
    from paper_2505_08124_b300 import slag as S
    S.load_library()
    return S


def _scenes():
    # uneven scenes: sizes, view counts, resolutions and segment counts differ
    return [synth.small_scene(51, 3000, 2, 96, 64, 5, dim=128),
            synth.small_scene(52, 9000, 5, 200, 120, 9, dim=128, surfaces=4),
            synth.small_scene(53, 6000, 3, 160, 160, 7, dim=128, surfaces=3)]


def test_batched_scenes_match_single(slag):
    scenes = _scenes()
    single = []
    for s in scenes:
        with slag.Lifter(s.gaussians, dim=s.dim) as L:
            for v in s.views():
                L.add_view(v.camera, v.seg, v.table)
            single.append(L.finalize())
    lifters = [slag.Lifter(s.gaussians, dim=s.dim) for s in scenes]
    try:
        slag.add_views_batched(lifters, [[(v.camera, v.seg, v.table) for v in s.views()] for s in scenes])
        for L, s, (E, w) in zip(lifters, scenes, single):
            Eb, wb = L.finalize()
            assert L.stats()["views"] == s.n_views
            np.testing.assert_allclose(wb, w, rtol=1e-6, atol=0)
            np.testing.assert_allclose(Eb, E, rtol=1e-5, atol=1e-7)
            # and the float64 oracle over the scene's views: the float32 parity bar
            num, den, _ = O.lift(s.gaussians, list(s.views()))
            Eo = O.normalise(num, den)
            assert np.linalg.norm(Eb - Eo) / np.linalg.norm(Eo) <= 1e-4
            assert np.linalg.norm(wb - den) / np.linalg.norm(den) <= 1e-4
            ok = den >= 1e-3
            cos = (Eb[ok] * Eo[ok]).sum(1) / (np.linalg.norm(Eb[ok], axis=1) * np.linalg.norm(Eo[ok], axis=1))
            assert cos.min() >= 0.99999
    finally:
        for L in lifters:
            L.close()


def test_batched_reports_the_failing_scene(slag):
    scenes = _scenes()[:2]
    lifters = [slag.Lifter(s.gaussians, dim=s.dim) for s in scenes]
    try:
        views = [[(v.camera, v.seg, v.table) for v in s.views()] for s in scenes]
        cam, seg, tab = views[1][1]
        bad = seg.copy()
        bad[0, 0] = tab.shape[0]        # a segment id outside [-1, M)
        views[1][1] = (cam, bad, tab)
        with pytest.raises(slag.SlagError) as e:
            slag.add_views_batched(lifters, views)
        assert e.value.status == slag.ERR_INVALID_ARG and "scene 1" in str(e.value)
    finally:
        for L in lifters:
            L.close()


@pytest.mark.parametrize("autotune", [True, False])
def test_graph_replayed_queries_match(slag, autotune):
    import torch
    s = synth.small_scene(54, 20000, 3, 200, 160, 9, dim=256, surfaces=5)
    rng = np.random.default_rng(9)
    Q = rng.standard_normal((1500, s.dim)).astype(np.float32)
    Q /= np.linalg.norm(Q, axis=1, keepdims=True)
    dQ = torch.from_numpy(Q).cuda()
    ids = torch.empty((1500, 10), dtype=torch.int64, device="cuda")
    sc = torch.empty((1500, 10), dtype=torch.float32, device="cuda")
    cnt = torch.empty(1500, dtype=torch.int32, device="cuda")
    with slag.Lifter(s.gaussians, dim=s.dim) as L:
        L.set_autotune(autotune)
        views = list(s.views())
        for v in views[:2]:
            L.add_view(v.camera, v.seg, v.table)
        L.finalize()
        ref_ids, ref_sc, _ = L.query_batch(Q, 10)                  # host path: plain launches
        for _ in range(3):                                         # capture, then replays
            L.query_batch(dQ, 10, ids, sc, cnt)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(ids.cpu().numpy(), ref_ids)
            np.testing.assert_allclose(sc.cpu().numpy(), ref_sc, rtol=1e-6, atol=1e-7)
        # new embeddings: the graph must not replay stale candidates
        L.add_view(views[2].camera, views[2].seg, views[2].table)
        L.finalize()
        ref2, _, _ = L.query_batch(Q, 10)
        L.query_batch(dQ, 10, ids, sc, cnt)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ids.cpu().numpy(), ref2)
