"""Checkpoint, resume and merge of the accumulated state, against the oracle.

The aggregation's numerator and denominator are sums over views (Aggregation
step), which is what the paper's multi-GPU section relies on when it sums
per-GPU tensors. So:
  * saving a context's state after some views, loading it into a new context
    and adding the remaining views gives the result of one context fed every
    view;
  * merging the states of disjoint view sets (on the device, or on the host
    without a GPU) gives the float64 oracle's result over all views at the
    float32 parity bar.
"""
import numpy as np
import pytest

import synth
from oracle import oracle as O

pytestmark = pytest.mark.gpu

REL_L2 = 1e-4
COS_MIN = 0.99999
W_FLOOR = 1e-3


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


@pytest.fixture(scope="module")
def scene():
    s = synth.small_scene(12, 6000, 6, 176, 120, 9, dim=128, surfaces=5, empty_fraction=0.15)
    views = [s.view(i) for i in range(s.n_views)]
    num, den, _ = O.lift(s.gaussians, views)
    return s, views, O.normalise(num, den), den


def _gate(E, w, Eo, den):
    rel = np.linalg.norm(E.astype(np.float64) - Eo) / np.linalg.norm(Eo)
    relw = np.linalg.norm(w.astype(np.float64) - den) / np.linalg.norm(den)
    ok = den >= W_FLOOR
    a, b = E[ok].astype(np.float64), Eo[ok]
    cos = (a * b).sum(1) / np.maximum(np.linalg.norm(a, axis=1) * np.linalg.norm(b, axis=1), 1e-300)
    assert rel <= REL_L2 and relw <= REL_L2, (rel, relw)
    assert cos.min() >= COS_MIN, cos.min()
    assert np.all(E[den == 0] == 0) and np.all(w[den == 0] == 0)


def _lift(S, s, views):
    L = S.Lifter(s.gaussians, dim=s.dim)
    for v in views:
        L.add_view(v.camera, v.seg, v.table)
    return L


def test_save_load_resume_equals_one_context(slag, scene):
    s, views, Eo, den = scene
    with _lift(slag, s, views) as L:
        E1, w1 = L.finalize()
        st1 = L.stats()
    with _lift(slag, s, views[:3]) as A:
        state = A.save_state()
    hdr = slag.read_state(state)["header"]
    assert hdr["views"] == 3 and hdr["columns"] == 3 * s.view(0).m and hdr["triples"] > 0
    with slag.Lifter(s.gaussians, dim=s.dim) as B:
        B.load_state(state)
        for v in views[3:]:
            B.add_view(v.camera, v.seg, v.table)
        E2, w2 = B.finalize()
        st2 = B.stats()
        ids, sc = B.query(views[0].table[0] / np.linalg.norm(views[0].table[0]), 5)
    assert st2["views"] == st1["views"] and st2["columns"] == st1["columns"]
    assert st2["contributions"] == st1["contributions"] and st2["triples"] == st1["triples"]
    np.testing.assert_allclose(E2, E1, rtol=0, atol=2e-6)
    np.testing.assert_allclose(w2, w1, rtol=1e-6, atol=1e-7)
    _gate(E2, w2, Eo, den)
    assert len(ids) == 5


def test_merge_of_disjoint_view_sets_matches_the_oracle(slag, scene):
    s, views, Eo, den = scene
    with _lift(slag, s, views[0::2]) as X:
        sx = X.save_state()
    with _lift(slag, s, views[1::2]) as Y:
        sy = Y.save_state()
    with slag.Lifter(s.gaussians, dim=s.dim) as M:
        M.load_state(sx)
        M.merge_state(sy)
        assert M.stats()["views"] == len(views)
        E, w = M.finalize()
    _gate(E, w, Eo, den)
    # the same merge on the host, without a context, loaded back
    sm = slag.state_merge_host(sx, sy)
    with slag.Lifter(s.gaussians, dim=s.dim) as H:
        H.load_state(sm)
        Eh, wh = H.finalize()
    np.testing.assert_allclose(Eh, E, rtol=0, atol=1e-6)
    np.testing.assert_array_equal(wh, w)


def test_state_errors(slag, scene):
    s, views, _, _ = scene
    with _lift(slag, s, views[:1]) as A:
        state = A.save_state()
    other = synth.small_scene(13, 5000, 1, 64, 64, 4, dim=128)
    with slag.Lifter(other.gaussians, dim=128) as B:
        with pytest.raises(slag.SlagError) as e:
            B.merge_state(state)             # another Gaussian set
        assert e.value.status == slag.ERR_INVALID_ARG
    bad = state.copy()
    bad[0] ^= 0xFF
    with slag.Lifter(s.gaussians, dim=s.dim) as C:
        with pytest.raises(slag.SlagError) as e:
            C.load_state(bad)                # not a state
        assert e.value.status == slag.ERR_INVALID_ARG
        with pytest.raises(slag.SlagError) as e:
            C.merge_state(state[:-4])        # truncated
        assert e.value.status == slag.ERR_INVALID_ARG
    with slag.Lifter(s.gaussians, dim=256) as D:
        with pytest.raises(slag.SlagError):
            D.merge_state(state)             # another width
