"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Gates (the float32 path):
  * integer stages -- tiles touched per Gaussian, per-tile Gaussian lists and
    tile ranges -- bit-exact against the oracle's float32 binning mirror;
  * embeddings: relative L2 of E <= 1e-4 over all Gaussians, cosine >= 0.99999
    for every Gaussian whose weight sum is at least 1e-3 (below that a single
    contribution at the alpha floor or the transmittance stop can flip between
    float32 and float64 and dominate the Gaussian's average);
  * weight sums: relative L2 <= 1e-4;
  * per-pixel transmittance within 2e-5 of the oracle, and sum w = 1 - T to 1e-5;
  * queries: the returned ids equal the oracle's wherever the oracle's scores
    are separated by more than 1e-5 (the float32 score error), and every
    returned id is a valid answer within that margin.
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


def _lift_gpu(S, scene, views, mode=0):
    with S.Lifter(scene.gaussians, dim=scene.dim, weight_mode=mode) as L:
        for v in views:
            L.add_view(v.camera, v.seg, v.table)
        E, w = L.finalize()
        st = L.stats()
    return E, w, st


def _compare(E, w, num, den, label=""):
    Eo = O.normalise(num, den)
    rel = np.linalg.norm(E.astype(np.float64) - Eo) / np.linalg.norm(Eo)
    relw = np.linalg.norm(w.astype(np.float64) - den) / np.linalg.norm(den)
    ok = den >= W_FLOOR
    a = E[ok].astype(np.float64)
    b = Eo[ok]
    cos = (a * b).sum(1) / np.maximum(np.linalg.norm(a, axis=1) * np.linalg.norm(b, axis=1), 1e-300)
    assert rel <= REL_L2, (label, rel)
    assert relw <= REL_L2, (label, relw)
    assert cos.min() >= COS_MIN, (label, cos.min(), int(np.argmin(cos)))
    # untouched Gaussians get the zero vector and zero weight on both sides
    assert np.all(E[den == 0] == 0) and np.all(w[den == 0] == 0)
    return rel, relw, cos.min()


# ----------------------------------------------------------------------------
# integer stages
# ----------------------------------------------------------------------------

def _binning_cases():
    s = synth.config_tiny()
    yield "tiny", s.gaussians, [s.view(i).camera for i in range(s.n_views)]
    s2 = synth.small_scene(5, 4000, 2, 200, 120, 7, dim=128, surfaces=6)
    yield "ragged", s2.gaussians, [s2.view(i).camera for i in range(2)]
    # Gaussians behind the camera, straddling the image border, exact depth ties
    g = synth.random_gaussians(9, 3000, -2.5, 2.5)
    g.means[100:140] = g.means[100]
    g.means[200] = [0.0, 0.0, 0.0]
    yield "edges", g, [synth.look_at([0.0, -1.5, 0.2], [0, 0, 0], 97, 61, 70.0)]
    # a single tile
    yield "onetile", s.gaussians.subset(np.arange(300)), [synth.look_at([0, -3, 0.5], [0, 0, 0], 16, 16)]
    # large Gaussians (hundreds of tiles each): one Gaussian's pairs span several of the binning
    # sort's 4096-pair tiles
    g = synth.random_gaussians(11, 800, -1.0, 1.0)
    g.scales *= 15.0
    yield "wide", g, [synth.look_at([0.0, -3.0, 0.4], [0, 0, 0], 960, 540)]
    # more tiles (2304) than the single-pass binning takes: pair emission and a two-pass sort
    g = synth.random_gaussians(12, 30000, -1.0, 1.0)
    yield "manytiles", g, [synth.look_at([0.3, -3.0, 0.4], [0, 0, 0], 1024, 576)]


@pytest.mark.parametrize("case", [c[0] for c in _binning_cases()])
def test_binning_bit_exact(slag, case):
    name, g, cams = next(c for c in _binning_cases() if c[0] == case)
    with slag.Lifter(g, dim=128) as L:
        for cam in cams:
            touched, lst, rng = L.bin_view(cam)
            _, _, t_ref = O.bin_f32(g, cam)
            lst_ref, rng_ref = O.tile_lists(g, cam)
            np.testing.assert_array_equal(touched, t_ref)
            assert lst.shape == lst_ref.shape
            np.testing.assert_array_equal(lst, lst_ref)
            np.testing.assert_array_equal(rng, rng_ref)


def _super_lists(g, cam, shift):
    """Expected bins of 2^shift x 2^shift tiles from the oracle's float32 mirror: a Gaussian is in
    every bin its tile rectangle meets; each bin's members in (float32 depth, index) order."""
    depth, rect, touched = O.bin_f32(g, cam)
    tx, ty = (cam.width + 15) // 16, (cam.height + 15) // 16
    bx, by = ((tx - 1) >> shift) + 1, ((ty - 1) >> shift) + 1
    members = [[] for _ in range(bx * by)]
    for k in np.nonzero(touched)[0]:
        x0, y0, x1, y1 = rect[k]
        for yb in range(y0 >> shift, ((y1 - 1) >> shift) + 1):
            for xb in range(x0 >> shift, ((x1 - 1) >> shift) + 1):
                members[yb * bx + xb].append(k)
    lst, rng, at = [], np.zeros((bx * by, 2), np.int64), 0
    for b, m in enumerate(members):
        m = np.array(m, np.int64)
        order = np.lexsort((m, depth[m])) if len(m) else m
        lst.extend(m[order].tolist())
        rng[b] = (at, at + len(m))
        at += len(m)
    return np.array(lst, np.int32), rng


@pytest.mark.parametrize("case", [c[0] for c in _binning_cases()])
def test_super_tile_binning_bit_exact(slag, case):
    # the binning slag_add_view composites from: 4x4-tile super-tile lists and ranges, and the
    # per-tile sequences the compositing kernel itself stages from them
    name, g, cams = next(c for c in _binning_cases() if c[0] == case)
    with slag.Lifter(g, dim=128) as L:
        for cam in cams:
            for shift in (0, 2):
                lst, rng = L.bin_view_bins(cam, shift)
                lst_ref, rng_ref = _super_lists(g, cam, shift)
                assert lst.shape == lst_ref.shape, (name, shift)
                np.testing.assert_array_equal(lst, lst_ref)
                np.testing.assert_array_equal(rng, rng_ref)
            staged, trng = L.composite_trace(cam)
            lst_ref, rng_ref = O.tile_lists(g, cam)
            np.testing.assert_array_equal(trng, rng_ref)
            np.testing.assert_array_equal(staged, lst_ref)


# ----------------------------------------------------------------------------
# compositing state per pixel
# ----------------------------------------------------------------------------

def test_pixel_transmittance_and_telescoping(slag):
    s = synth.small_scene(6, 5000, 2, 160, 112, 5, dim=128, surfaces=4)
    with slag.Lifter(s.gaussians, dim=128) as L:
        for vi in range(2):
            v = s.view(vi)
            T, ws, cnt = L.render_debug(v.camera)
            r = O.view_weights(s.gaussians, v, per_pixel=True)
            np.testing.assert_allclose(T, r["T_final"], atol=2e-5)
            np.testing.assert_allclose(ws, 1.0 - T, atol=1e-5)
            assert np.mean(cnt == r["count_px"]) > 0.999
            assert cnt.max() > 20


# ----------------------------------------------------------------------------
# end to end
# ----------------------------------------------------------------------------

def test_tiny_config_parity(slag):
    s = synth.config_tiny()
    views = list(s.views())
    E, w, st = _lift_gpu(slag, s, views)
    num, den, info = O.lift(s.gaussians, views, threads=4)
    _compare(E, w, num, den, "tiny")
    assert st["views"] == 4 and st["pairs"] == sum(p for p, _ in info)
    c_ref = sum(c for _, c in info)
    assert abs(st["contributions"] - c_ref) <= 1e-4 * c_ref


@pytest.mark.parametrize("seed,mode,empty", [(11, 0, 0.25), (12, 1, 0.0), (13, 0, 0.0)])
def test_small_scene_parity(slag, seed, mode, empty):
    s = synth.small_scene(seed, 6000, 3, 200, 120, 9, dim=256, surfaces=5, empty_fraction=empty)
    views = list(s.views())
    E, w, _ = _lift_gpu(slag, s, views, mode)
    num, den, _ = O.lift(s.gaussians, views, weight_mode=mode, threads=3)
    _compare(E, w, num, den, "small%d" % seed)


@pytest.mark.parametrize("dim", [384, 4096])
def test_embedding_widths(slag, dim):
    # D = 384 (the contraction in 128-wide passes) and the largest D, 4096 (sixteen 256-wide passes,
    # 128 K-chunks per query tile): embeddings and top-10 queries against the oracle
    s = synth.small_scene(16, 3000, 2, 128, 96, 5, dim=dim, surfaces=3)
    views = list(s.views())
    rng = np.random.default_rng(8)
    with slag.Lifter(s.gaussians, dim=dim) as L:
        for v in views:
            L.add_view(v.camera, v.seg, v.table)
        E, w = L.finalize()
        Q = rng.standard_normal((20, dim)).astype(np.float32)
        Q /= np.linalg.norm(Q, axis=1, keepdims=True)
        ids, sc, cnt = L.query_batch(Q, 10)
    num, den, _ = O.lift(s.gaussians, views, threads=2)
    _compare(E, w, num, den, "dim%d" % dim)
    for b in range(Q.shape[0]):
        _check_topk(ids[b, :cnt[b]], sc[b, :cnt[b]], E.astype(np.float64), w.astype(np.float64),
                    Q[b].astype(np.float64), 10)


@pytest.mark.parametrize("n", [1, 2, 129])
def test_few_gaussians(slag, n):
    # one Gaussian, two, and one block of 128 plus one (a ragged second block): embeddings against
    # the oracle, and a top-5 query that can return fewer ids than asked
    s = synth.small_scene(17, 2000, 2, 96, 64, 4, dim=128, surfaces=2)
    g = s.gaussians.subset(np.arange(n))
    views = list(s.views())
    q = views[0].table[0] / np.linalg.norm(views[0].table[0])
    with slag.Lifter(g, dim=128) as L:
        for v in views:
            L.add_view(v.camera, v.seg, v.table)
        E, w = L.finalize()
        ids, sc, cnt = L.query_batch(q[None, :].astype(np.float32), 5)
    num, den, _ = O.lift(g, views)
    assert (den > 0).sum() == n
    _compare(E, w, num, den, "n%d" % n)
    assert cnt[0] == min(5, n)
    _check_topk(ids[0, :cnt[0]], sc[0, :cnt[0]], E.astype(np.float64), w.astype(np.float64), q.astype(np.float64),
                min(5, n))


def test_constant_features(slag):
    s = synth.small_scene(14, 3000, 3, 96, 80, 7, dim=128, empty_fraction=0.2)
    c = np.random.default_rng(2).standard_normal(128).astype(np.float32)
    c /= np.linalg.norm(c)
    views = [synth.View(v.camera, v.seg, np.tile(c, (v.m, 1))) for v in s.views()]
    E, w, _ = _lift_gpu(slag, s, views)
    ok = w > 0
    assert ok.sum() > 500
    np.testing.assert_allclose(E[ok], np.tile(c, (ok.sum(), 1)), rtol=2e-6, atol=2e-7)


def test_view_order_invariance(slag):
    s = synth.small_scene(15, 4000, 4, 128, 96, 6, dim=128, surfaces=3)
    views = list(s.views())
    E1, w1, _ = _lift_gpu(slag, s, views)
    E2, w2, _ = _lift_gpu(slag, s, [views[i] for i in (2, 0, 3, 1)])
    np.testing.assert_allclose(E2, E1, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(w2, w1, rtol=1e-5, atol=1e-7)


def test_reset_and_refinalize(slag):
    s = synth.small_scene(16, 3000, 3, 128, 96, 6, dim=128)
    views = list(s.views())
    with slag.Lifter(s.gaussians, dim=128) as L:
        for v in views[:2]:
            L.add_view(v.camera, v.seg, v.table)
        L.finalize()
        L.add_view(views[2].camera, views[2].seg, views[2].table)
        E_inc, w_inc = L.finalize()
        L.reset()
        for v in views:
            L.add_view(v.camera, v.seg, v.table)
        E_all, w_all = L.finalize()
    np.testing.assert_allclose(E_inc, E_all, rtol=1e-5, atol=1e-6)
    num, den, _ = O.lift(s.gaussians, views)
    _compare(E_all, w_all, num, den, "reset")


def test_device_inputs_match_host_inputs(slag):
    import torch
    s = synth.small_scene(17, 3000, 2, 128, 96, 6, dim=128)
    views = list(s.views())
    E_h, w_h, _ = _lift_gpu(slag, s, views)
    g = s.gaussians
    dg = synth.Gaussians(*(torch.from_numpy(np.ascontiguousarray(a)).cuda()
                           for a in (g.means, g.scales, g.quats, g.opacities)))
    with slag.Lifter(dg, dim=128) as L:
        for v in views:
            L.add_view(v.camera, torch.from_numpy(v.seg).cuda(), torch.from_numpy(v.table).cuda())
        E = torch.empty((g.n, 128), device="cuda")
        w = torch.empty(g.n, device="cuda")
        L.finalize(E, w)
        torch.cuda.synchronize()
    # float32 atomics accumulate in a run-dependent order: equal up to the last bits
    np.testing.assert_allclose(E.cpu().numpy(), E_h, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(w.cpu().numpy(), w_h, rtol=1e-6)


# ----------------------------------------------------------------------------
# queries
# ----------------------------------------------------------------------------

def _check_topk(ids, sc, E_ref, den, q, k, margin=1e-5):
    ref_ids1, ref_sc1 = O.topk(E_ref, den, q, k + 1)
    ref_ids, ref_sc = ref_ids1[:k], ref_sc1[:k]
    assert len(ids) == len(ref_ids)
    # every returned id is a candidate scoring within the margin of the oracle's score at its rank
    nrm = np.linalg.norm(E_ref, axis=1)
    true = (E_ref[ids] @ q) / nrm[ids]
    assert np.all(den[ids] > 0)
    assert np.all(true >= ref_sc - margin)
    # where the oracle's ranking is separated by more than the margin, ids agree exactly
    gaps = np.abs(np.diff(ref_sc1))          # includes the gap to the (k+1)-th candidate
    sep = np.ones(len(ref_sc1), bool)
    sep[:-1] &= gaps > margin
    sep[1:] &= gaps > margin
    sep = sep[:len(ref_ids)]
    np.testing.assert_array_equal(ids[sep], ref_ids[sep])
    np.testing.assert_allclose(sc, true, atol=margin)


def test_query_topk(slag):
    s = synth.small_scene(18, 8000, 3, 160, 120, 8, dim=256, surfaces=4)
    views = list(s.views())
    rng = np.random.default_rng(3)
    with slag.Lifter(s.gaussians, dim=256) as L:
        for v in views:
            L.add_view(v.camera, v.seg, v.table)
        E, w = L.finalize()
        Q = rng.standard_normal((37, 256)).astype(np.float32)
        Q[:5] = views[0].table[:5]
        Q /= np.linalg.norm(Q, axis=1, keepdims=True)
        for k in (1, 10, 200):
            ids, sc, cnt = L.query_batch(Q, k)
            for b in range(Q.shape[0]):
                _check_topk(ids[b, :cnt[b]], sc[b, :cnt[b]], E.astype(np.float64), w.astype(np.float64),
                            Q[b].astype(np.float64), k)
        i1, s1 = L.query(Q[3], 10)
        np.testing.assert_array_equal(i1, ids[3, :10] if k == 10 else L.query_batch(Q[3:4], 10)[0][0])


@pytest.mark.parametrize("dim,B", [(128, 1000), (512, 300)])
def test_query_tensor_core_tiles(slag, dim, B):
    # several tiles of 128 queries (the last one ragged), several tiles of 256 candidates per split
    # (both TMEM accumulators reused), four and sixteen K-chunks of 32; host and device query
    # buffers (the latter replayed as a graph) return the same ids
    import torch
    s = synth.small_scene(24, 30000, 4, 320, 240, 12, dim=dim, surfaces=6)
    views = list(s.views())
    rng = np.random.default_rng(11)
    with slag.Lifter(s.gaussians, dim=dim) as L:
        for v in views:
            L.add_view(v.camera, v.seg, v.table)
        E, w = L.finalize()
        assert (w > 0).sum() > 256 * 20
        Q = rng.standard_normal((B, dim)).astype(np.float32)
        Q[:8] = views[0].table[:8]
        Q /= np.linalg.norm(Q, axis=1, keepdims=True)
        k = 16
        ids, sc, cnt = L.query_batch(Q, k)
        E64, w64 = E.astype(np.float64), w.astype(np.float64)
        for b in sorted(set(range(0, B, 17)) | {B - 1, 127, 128}):
            _check_topk(ids[b, :cnt[b]], sc[b, :cnt[b]], E64, w64, Q[b].astype(np.float64), k)
        dQ = torch.from_numpy(Q).cuda()
        d_ids = torch.empty((B, k), dtype=torch.int64, device="cuda")
        d_sc = torch.empty((B, k), dtype=torch.float32, device="cuda")
        d_cnt = torch.empty(B, dtype=torch.int32, device="cuda")
        for _ in range(2):
            d_ids.fill_(-7)
            L.query_batch(dQ, k, d_ids, d_sc, d_cnt)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(d_ids.cpu().numpy(), ids)
            np.testing.assert_array_equal(d_sc.cpu().numpy(), sc)


def test_threshold_query(slag):
    # the binary response at cosine >= 0.28 (Experiments) against the oracle's cosines: every id
    # clearly above the threshold is returned, none clearly below, in increasing order
    s = synth.small_scene(8, 6000, 3, 160, 112, 6, dim=128, surfaces=4, n_protos=4)
    views = [s.view(i) for i in range(s.n_views)]
    num, den, _ = O.lift(s.gaussians, views)
    Eo = O.normalise(num, den)
    nrm = np.linalg.norm(Eo, axis=1)
    with slag.Lifter(s.gaussians, dim=128) as L:
        for v in views:
            L.add_view(v.camera, v.seg, v.table)
        L.finalize()
        for q in (views[0].table[0], views[1].table[3], -views[2].table[1]):
            q = q / np.linalg.norm(q)
            ids = L.query_threshold(q, 0.28)
            cos = np.where(nrm > 0, (Eo @ q.astype(np.float64)) / np.maximum(nrm, 1e-300), -2.0)
            cos[den <= 0] = -2.0
            assert np.all(np.diff(ids) > 0)
            sure_in = np.nonzero(cos >= 0.28 + 1e-4)[0]
            sure_out = np.nonzero(cos < 0.28 - 1e-4)[0]
            assert np.isin(sure_in, ids).all()
            assert not np.isin(ids, sure_out).any()
        # sizing call and a cut-off output
        q = views[0].table[0] / np.linalg.norm(views[0].table[0])
        full = L.query_threshold(q, 0.28)
        assert len(full) > 10


def test_query_more_than_candidates(slag):
    s = synth.small_scene(19, 500, 1, 64, 64, 3, dim=128)
    with slag.Lifter(s.gaussians, dim=128) as L:
        v = s.view(0)
        L.add_view(v.camera, v.seg, v.table)
        E, w = L.finalize()
        n_valid = int(((w > 0) & (np.linalg.norm(E, axis=1) > 0)).sum())
        q = v.table[0] / np.linalg.norm(v.table[0])
        ids, sc = L.query(q, 1024)
        assert len(ids) == n_valid
        assert len(set(ids.tolist())) == n_valid


@pytest.mark.parametrize("k", [5, 300])   # tensor-core path and CUDA-core path
def test_query_without_candidates(slag, k):
    # a view whose pixels all lie outside every segment touches no Gaussian: every
    # query has an empty result
    s = synth.small_scene(23, 500, 1, 64, 64, 3, dim=128)
    v = s.view(0)
    with slag.Lifter(s.gaussians, dim=128) as L:
        L.add_view(v.camera, np.full_like(v.seg, -1), v.table)
        E, w = L.finalize()
        assert not w.any() and not E.any()
        Q = np.tile(v.table[:1] / np.linalg.norm(v.table[0]), (3, 1)).astype(np.float32)
        ids, sc, cnt = L.query_batch(Q, k)
        assert (cnt == 0).all()
        assert (ids == -1).all()


# ----------------------------------------------------------------------------
# errors
# ----------------------------------------------------------------------------

def test_errors_are_status_codes(slag):
    s = synth.small_scene(20, 500, 1, 64, 48, 3, dim=128)
    v = s.view(0)
    with slag.Lifter(s.gaussians, dim=128) as L:
        with pytest.raises(slag.SlagError) as e:
            L.query(np.ones(128, np.float32), 5)
        assert e.value.status == slag.ERR_STATE
        with pytest.raises(slag.SlagError) as e:
            L.finalize()
        assert e.value.status == slag.ERR_STATE
        bad = v.seg.copy()
        bad[3, 7] = v.m
        with pytest.raises(slag.SlagError) as e:
            L.add_view(v.camera, bad, v.table)
        assert e.value.status == slag.ERR_INVALID_ARG
        # the rejected view left no trace
        L.add_view(v.camera, v.seg, v.table)
        E, w = L.finalize()
        assert L.stats()["views"] == 1
    g = s.gaussians
    bad_g = synth.Gaussians(g.means.copy(), g.scales, g.quats, g.opacities)
    bad_g.means[4, 1] = np.nan
    with pytest.raises(slag.SlagError) as e:
        slag.Lifter(bad_g, dim=128)
    assert e.value.status == slag.ERR_INVALID_ARG
