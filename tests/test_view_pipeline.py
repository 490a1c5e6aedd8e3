"""The two halves of slag_add_view.

A view's first half (uploads, segment-id check, projection, depth sort, tile-count scan) is
queued by its own slag_add_view. Its second half (binning, compositing, masking, reduction) is
queued by the same call when earlier views give an estimate of its pair count (the binning then
reads the counts on the device and flags a view whose pairs exceed the estimate; such a view is
binned again with its exact count when its slot is reused or the views are joined), and
otherwise by the next call on the context, once the host has read the count. These tests check
that every way of ending a view's wait gives the result of the plain sequence, up to the
float32 summation order of the weight atomics:
- calls between views (diagnostics, profiles);
- a rejected view after an accepted one;
- slag_reset with a view still waiting;
- the caller's input buffers reused as soon as slag_add_view returns (host and device);
- views whose pair counts outgrow the estimate (against the oracle);
- views whose Gaussians reach more segments than their tables hold, beyond the spill list's
  capacity (composited again, against the oracle);
- degenerate views sized on the device: no visible Gaussian, no segment, one segment, ragged and
  1x1 images (against the oracle);
- a view with more super-tiles than the single-pass binning takes, between views sized on the
  device (against the oracle);
- replayed graphs against kernel-by-kernel launches."""
import math

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


@pytest.fixture(scope="module")
def scene():
    s = synth.small_scene(43, 6000, 9, 176, 120, 8, dim=128, surfaces=4)
    return s, list(s.views())


def _plain(slag, s, views):
    with slag.Lifter(s.gaussians, dim=128) as L:
        for v in views:
            L.add_view(v.camera, v.seg, v.table)
        E, w = L.finalize()
        return E, w, L.stats()


def _close(a, b):
    (E, w), (Er, wr) = a, b
    np.testing.assert_allclose(E, Er, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(w, wr, rtol=1e-5, atol=1e-7)


def test_calls_between_views(slag, scene):
    s, views = scene
    Er, wr, st_r = _plain(slag, s, views)
    with slag.Lifter(s.gaussians, dim=128) as L:
        L.set_profiling(True)
        for i, v in enumerate(views):
            L.add_view(v.camera, v.seg, v.table)
            if i == 1:
                L.render_debug(views[5].camera)
            elif i == 3:
                L.bin_view(views[0].camera)
            elif i == 4:
                prof = L.profile()
                assert prof["composite"][1] == 5   # the second halves of views 0..4 are queued
        E, w = L.finalize()
        st = L.stats()
    _close((E, w), (Er, wr))
    for k in ("views", "pairs", "columns", "triples"):
        assert st[k] == st_r[k], k


def test_rejected_view_after_accepted(slag, scene):
    s, views = scene
    Er, wr, _ = _plain(slag, s, [views[0], views[2]])
    bad = views[1].seg.copy()
    bad[7, 11] = views[1].m
    with slag.Lifter(s.gaussians, dim=128) as L:
        L.add_view(views[0].camera, views[0].seg, views[0].table)
        with pytest.raises(slag.SlagError) as e:
            L.add_view(views[1].camera, bad, views[1].table)
        assert e.value.status == slag.ERR_INVALID_ARG
        L.add_view(views[2].camera, views[2].seg, views[2].table)
        E, w = L.finalize()
        assert L.stats()["views"] == 2
    _close((E, w), (Er, wr))


def test_reset_drops_waiting_view(slag, scene):
    s, views = scene
    Er, wr, _ = _plain(slag, s, [views[3], views[4]])
    with slag.Lifter(s.gaussians, dim=128) as L:
        for v in views[:3]:
            L.add_view(v.camera, v.seg, v.table)
        L.reset()
        L.add_view(views[3].camera, views[3].seg, views[3].table)
        L.add_view(views[4].camera, views[4].seg, views[4].table)
        E, w = L.finalize()
        assert L.stats()["views"] == 2
    _close((E, w), (Er, wr))


def test_input_buffers_free_on_return(slag, scene):
    import torch
    s, views = scene
    Er, wr, _ = _plain(slag, s, views)
    H, W = views[0].seg.shape
    M = max(v.m for v in views)
    # one pinned host buffer pair and one device buffer pair, rewritten for every view; the
    # device buffers are rewritten on the caller's stream right after the call returns
    h_seg = torch.empty((H, W), dtype=torch.int32).pin_memory().numpy()
    h_tab = torch.empty((M, 128), dtype=torch.float32).pin_memory().numpy()
    d_seg = torch.empty((H, W), dtype=torch.int32, device="cuda")
    d_tab = torch.empty((M, 128), dtype=torch.float32, device="cuda")
    junk = np.full((H, W), -1, np.int32)
    for device in (False, True):
        with slag.Lifter(s.gaussians, dim=128, stream=torch.cuda.current_stream().cuda_stream) as L:
            for v in views:
                if device:
                    d_seg.copy_(torch.from_numpy(v.seg))
                    d_tab[:v.m].copy_(torch.from_numpy(v.table))
                    L.add_view(v.camera, d_seg, d_tab[:v.m])
                    d_seg.fill_(-1)
                    d_tab.fill_(7.0)
                else:
                    h_seg[:] = v.seg
                    h_tab[:v.m] = v.table
                    L.add_view(v.camera, h_seg, h_tab[:v.m])
                    h_seg[:] = junk
                    h_tab[:] = 7.0
            E, w = L.finalize()
        _close((E, w), (Er, wr))


def _zoomed(views, radii):
    """The views' segment maps and tables, seen from an orbit of the given radius per view."""
    out = []
    for i, (v, r) in enumerate(zip(views, radii)):
        az = 2.0 * math.pi * i / len(radii)
        cam = synth.look_at([r * math.cos(az), r * math.sin(az), 0.3 * r], [0.0, 0.0, 0.0],
                            v.camera.width, v.camera.height)
        out.append(synth.View(cam, v.seg, v.table))
    return out


def test_views_outgrowing_the_estimate_are_binned_again(slag):
    # two views from afar, then seven close up with about twice the super-tile pairs: the close
    # views' binning, sized from the far ones, overflows; each is binned again with its exact
    # count when its slot is reused (views 6..8) or at the finalize, and the result is the oracle's
    s = synth.small_scene(43, 20000, 9, 480, 320, 8, dim=128, surfaces=4)
    zv = _zoomed(list(s.views()), [9.0, 9.0] + [2.2] * 7)
    with slag.Lifter(s.gaussians, dim=128) as L:
        for v in zv:
            L.add_view(v.camera, v.seg, v.table)
        E, w = L.finalize()
        st = L.stats()
    pairs = [int(O.bin_f32(s.gaussians, v.camera)[2].sum()) for v in zv]
    assert pairs[2] > 2 * pairs[0]
    assert st["resized_views"] >= 5
    assert st["pairs"] == sum(pairs)
    assert st["views"] == len(zv)
    num, den, _ = O.lift(s.gaussians, zv)
    Eo = O.normalise(num, den)
    rel = np.linalg.norm(E.astype(np.float64) - Eo) / np.linalg.norm(Eo)
    relw = np.linalg.norm(w.astype(np.float64) - den) / np.linalg.norm(den)
    assert rel <= 1e-4 and relw <= 1e-4, (rel, relw)



def test_views_overflowing_the_spill_list_are_composited_again(slag):
    # per-pixel random segment maps over 64 segments: each Gaussian reaches dozens of segments in
    # a view, far more than its table's slots, and the spilled sums of one view (at least 370,000
    # by the oracle's distinct (Gaussian, segment) counts) exceed the spill list's first capacity;
    # such a view is composited again with a list that holds them, and counted once
    s = synth.small_scene(43, 12000, 3, 320, 240, 8, dim=128, surfaces=4)
    base = list(s.views())
    zv = _zoomed(base[:2], [2.2, 2.2])
    rng = np.random.default_rng(7)
    views = [base[2]]
    for v in zv:
        seg = rng.integers(0, 64, size=(v.camera.height, v.camera.width)).astype(np.int32)
        table = rng.standard_normal((64, 128)).astype(np.float32)
        views.append(synth.View(v.camera, seg, table))
    lower = [int(np.maximum((O.view_weights(s.gaussians, v)["B"] > 0).sum(1) - 4, 0).sum()) for v in views[1:]]
    assert min(lower) > 300_000
    out = {}
    # replayed graphs, kernel-by-kernel launches, and a spilling first view (sized on the host)
    for case, order in (("graphs", views), ("direct", views), ("first", views[1:] + views[:1])):
        with slag.Lifter(s.gaussians, dim=128) as L:
            L.set_graphs(case == "graphs")
            for v in order:
                L.add_view(v.camera, v.seg, v.table)
            E, w = L.finalize()
            out[case] = (E, w, L.stats())
    num, den, info = O.lift(s.gaussians, views)
    Eo = O.normalise(num, den)
    contrib = sum(c for _, c in info)
    for graphs, (E, w, st) in out.items():
        # a view composited twice counts its composited pairs once
        assert st["recomposited_views"] >= 1, graphs
        assert st["views"] == len(views), graphs
        assert abs(st["contributions"] - contrib) <= 1e-4 * contrib, (graphs, st["contributions"], contrib)
        rel = np.linalg.norm(E.astype(np.float64) - Eo) / np.linalg.norm(Eo)
        relw = np.linalg.norm(w.astype(np.float64) - den) / np.linalg.norm(den)
        assert rel <= 1e-4 and relw <= 1e-4, (graphs, rel, relw)


def test_degenerate_views_sized_on_the_device(slag):
    # after a first view gives the pair estimate, the second halves are sized on the device (and
    # replayed from graphs, or launched kernel by kernel): a view facing away from the scene (no
    # visible Gaussian, no pairs), a view without segments (every id -1), a single segment, a
    # ragged 17x33 view and a 1x1 view; the sums are the oracle's
    s = synth.small_scene(45, 4000, 2, 96, 64, 6, dim=128, surfaces=3)
    base = list(s.views())
    rng = np.random.default_rng(11)
    v0 = base[0]
    away = synth.look_at([3.0, 0.0, 1.0], [6.0, 0.0, 2.0], 96, 64)
    views = [v0, synth.View(away, v0.seg, v0.table)]
    views.append(synth.View(base[1].camera, np.full((64, 96), -1, np.int32), base[1].table))
    views.append(synth.View(base[1].camera, np.zeros((64, 96), np.int32), base[1].table[:1]))
    for W, H in ((17, 33), (1, 1)):
        cam = synth.look_at([2.4, 0.8, 0.9], [0.0, 0.0, 0.0], W, H)
        seg = rng.integers(-1, 3, size=(H, W)).astype(np.int32)
        views.append(synth.View(cam, seg, rng.standard_normal((3, 128)).astype(np.float32)))
    views.append(base[1])
    num, den, info = O.lift(s.gaussians, views)
    assert info[1] == (0, 0)   # the view facing away: no pairs, no contributions
    Eo = O.normalise(num, den)
    for graphs in (True, False):
        with slag.Lifter(s.gaussians, dim=128) as L:
            L.set_graphs(graphs)
            for v in views:
                L.add_view(v.camera, v.seg, v.table)
            E, w = L.finalize()
            st = L.stats()
        assert st["views"] == len(views) and st["resized_views"] == 0, (graphs, st)
        contrib = sum(c for _, c in info)
        assert abs(st["contributions"] - contrib) <= 1e-4 * contrib, (graphs, st["contributions"], contrib)
        rel = np.linalg.norm(E.astype(np.float64) - Eo) / np.linalg.norm(Eo)
        relw = np.linalg.norm(w.astype(np.float64) - den) / np.linalg.norm(den)
        assert rel <= 1e-4 and relw <= 1e-4, (graphs, rel, relw)


def test_views_with_more_bins_than_the_single_pass_binning(slag):
    # a 4096x2176 view has 64 x 34 super-tiles, more than the single-pass binning's 2048 bins: its
    # second half is sized on the host (pair emission and a two-pass sort), between views sized on
    # the device; the sums are the oracle's
    s = synth.small_scene(46, 3000, 1, 96, 64, 4, dim=128, surfaces=3)
    rng = np.random.default_rng(5)
    cam = synth.look_at([2.2, 0.9, 0.8], [0.0, 0.0, 0.0], 4096, 2176)
    blocks = rng.integers(-1, 24, size=(2176 // 64 + 1, 4096 // 64 + 1)).astype(np.int32)
    seg = np.ascontiguousarray(np.repeat(np.repeat(blocks, 64, 0), 64, 1)[:2176, :4096])
    big = synth.View(cam, seg, rng.standard_normal((24, 128)).astype(np.float32))
    small = next(iter(s.views()))
    views = [small, big, small]
    parts = {id(v): O.view_weights(s.gaussians, v) for v in (small, big)}
    num = sum(parts[id(v)]["B"] @ v.table.astype(np.float64) for v in views)
    den = sum(parts[id(v)]["B"].sum(axis=1) for v in views)
    Eo = O.normalise(num, den)
    with slag.Lifter(s.gaussians, dim=128) as L:
        for v in views:
            L.add_view(v.camera, v.seg, v.table)
        E, w = L.finalize()
        st = L.stats()
    assert st["pairs"] == sum(parts[id(v)]["P"] for v in views)
    rel = np.linalg.norm(E.astype(np.float64) - Eo) / np.linalg.norm(Eo)
    relw = np.linalg.norm(w.astype(np.float64) - den) / np.linalg.norm(den)
    assert rel <= 1e-4 and relw <= 1e-4, (rel, relw)


def test_graph_replays_match_kernel_launches(slag):
    # views sized on the device replay the slot's captured graphs (on by default) or launch kernel
    # by kernel, with two image sizes in one context; the two give the same sums, and the oracle's
    g = synth.small_scene(44, 6000, 1, 16, 16, 4, dim=128, surfaces=4).gaussians
    s = synth.make_scene("alt", 44, g, n_views=14, width=176, height=120, n_segments=8, n_protos=8, dim=128,
                         jitter=True, resolutions=[(176, 120), (176, 120), (208, 96)])
    views = list(s.views())
    out = {}
    for graphs in (True, False):
        with slag.Lifter(g, dim=128) as L:
            L.set_graphs(graphs)
            n0 = slag.kernel_launches()
            for v in views:
                L.add_view(v.camera, v.seg, v.table)
            E, w = L.finalize()
            out[graphs] = (E, w, L.stats(), slag.kernel_launches() - n0)
    _close(out[True][:2], out[False][:2])
    for k in ("views", "pairs", "triples", "contributions", "columns"):
        assert out[True][2][k] == out[False][2][k], k
    # the launch counter counts the replayed graphs' kernels, not their captures
    assert out[True][3] == out[False][3]
    num, den, _ = O.lift(g, views)
    Eo = O.normalise(num, den)
    rel = np.linalg.norm(out[True][0].astype(np.float64) - Eo) / np.linalg.norm(Eo)
    assert rel <= 1e-4, rel
