"""slag_finalize_async (asynchronous outputs, double-buffered results).

Three finalizes run back to back on one context, each with its outputs still being copied
when the next one starts: every output must equal a synchronous finalize of the same views
(up to the float32 summation order of the weight atomics), and queries issued right after
each finalize must see that finalize's embeddings, not the previous ones."""
import numpy as np
import pytest

import synth

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


def test_async_outputs_match_sync_and_do_not_overwrite(slag):
    import torch
    s = synth.small_scene(41, 6000, 6, 160, 120, 8, dim=256, surfaces=4)
    views = list(s.views())
    groups = [views[0:2], views[2:4], views[4:6]]
    ref = []
    for gv in groups:
        with slag.Lifter(s.gaussians, dim=256) as L:
            for v in gv:
                L.add_view(v.camera, v.seg, v.table)
            ref.append(L.finalize())
    n = s.gaussians.n
    outs = [(torch.empty((n, 256), dtype=torch.float32).pin_memory().numpy(),
             torch.empty(n, dtype=torch.float32).pin_memory().numpy()) for _ in groups]
    tops = []
    with slag.Lifter(s.gaussians, dim=256) as L:
        for gv, (E, w) in zip(groups, outs):
            L.reset()
            for v in gv:
                L.add_view(v.camera, v.seg, v.table)
            L.finalize_async(E, w)
            q = gv[0].table[0] / np.linalg.norm(gv[0].table[0])
            tops.append(L.query(q.astype(np.float32), 5))
        L.wait_outputs()
    for (E, w), (Er, wr), (ids, sc), gv in zip(outs, ref, tops, groups):
        np.testing.assert_allclose(E, Er, rtol=1e-5, atol=1e-6)
        np.testing.assert_allclose(w, wr, rtol=1e-5, atol=1e-7)
        # the query saw this group's embeddings: its candidates are this group's touched
        # Gaussians and its best score is the best score over this group's result
        assert len(ids) == 5 and (wr[ids] > 0).all()
        q = gv[0].table[0].astype(np.float64) / np.linalg.norm(gv[0].table[0])
        nrm = np.linalg.norm(Er.astype(np.float64), axis=1)
        ok = (wr > 0) & (nrm > 0)
        best = ((Er[ok].astype(np.float64) @ q) / nrm[ok]).max()
        assert abs(float(sc[0]) - best) < 1e-4


def test_async_outputs_on_device(slag):
    import torch
    s = synth.small_scene(42, 3000, 2, 128, 96, 6, dim=128)
    views = list(s.views())
    with slag.Lifter(s.gaussians, dim=128) as L:
        for v in views:
            L.add_view(v.camera, v.seg, v.table)
        Er, wr = L.finalize()
        dE = torch.empty((s.gaussians.n, 128), dtype=torch.float32, device="cuda")
        dw = torch.empty(s.gaussians.n, dtype=torch.float32, device="cuda")
        L.finalize_async(dE, dw)
        L.wait_outputs()
        np.testing.assert_array_equal(dE.cpu().numpy(), Er)
        np.testing.assert_array_equal(dw.cpu().numpy(), wr)


def test_async_rejects_converted_outputs(slag):
    s = synth.small_scene(43, 500, 1, 64, 48, 3, dim=128)
    v = s.view(0)
    with slag.Lifter(s.gaussians, dim=128) as L:
        L.add_view(v.camera, v.seg, v.table)
        with pytest.raises(ValueError):
            L.finalize_async(np.empty((s.gaussians.n, 128), np.float64), None)
