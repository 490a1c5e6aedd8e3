"""Pins for the CPU oracle, checked against things other than the oracle itself.

* projection: scipy's quaternion-to-rotation routine, a finite-difference
  Jacobian of the pinhole map and numpy's matrix inverse / eigenvalues;
* closed forms: one isotropic Gaussian on the optical axis split by a
  vertical segment boundary; a co-centred stack of Gaussians (w_2 =
  alpha_2 (1 - alpha_1), early stop below 1e-4);
* invariants: sum_k w_kp = 1 - T_final(p); constant features reproduce the
  constant; invariance to view order; literal form == factored form;
* brute force: an independent numpy compositor over tiny scenes;
* the alpha floor: the float32 decision equals the float64 one away from the floor;
* queries: numpy's stable argsort of the cosine scores.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import synth
from oracle import oracle as O


def _cam(W, H, f, R=None, t=(0.0, 0.0, 2.0)):
    return synth.Camera(fx=f, fy=f, cx=W / 2.0, cy=H / 2.0, width=W, height=H,
                        R=np.eye(3, dtype=np.float32) if R is None else np.asarray(R, np.float32),
                        t=np.asarray(t, np.float32))


def _gauss(means, scales, quats=None, op=None):
    means = np.asarray(means, np.float32).reshape(-1, 3)
    n = means.shape[0]
    scales = np.asarray(scales, np.float32).reshape(n, 3)
    quats = np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)) if quats is None else np.asarray(quats, np.float32)
    op = np.full(n, 0.8, np.float32) if op is None else np.asarray(op, np.float32)
    return synth.Gaussians(means, scales, quats, op)


# ----------------------------------------------------------------------------
# independent numpy projection
# ----------------------------------------------------------------------------

def _np_project(g, cam):
    """Projection written from the pinhole model, with scipy's rotation routine and an FD Jacobian."""
    R = cam.R.astype(np.float64)
    t = cam.t.astype(np.float64)
    out = []
    tanx = 0.5 * cam.width / cam.fx
    tany = 0.5 * cam.height / cam.fy
    for k in range(g.n):
        q = g.quats[k].astype(np.float64)
        Rq = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()   # scipy is scalar-last
        S3 = Rq @ np.diag(g.scales[k].astype(np.float64) ** 2) @ Rq.T
        pc = R @ g.means[k].astype(np.float64) + t
        # Jacobian of the pinhole map at the mean, with x/z and y/z clamped to 1.3 tan(half fov)
        x, y, z = pc
        xc = np.clip(x / z, -1.3 * tanx, 1.3 * tanx) * z
        yc = np.clip(y / z, -1.3 * tany, 1.3 * tany) * z

        def pin(p):
            return np.array([cam.fx * p[0] / p[2] + cam.cx, cam.fy * p[1] / p[2] + cam.cy])

        J = np.zeros((2, 3))
        for a in range(3):
            h = 1e-6 * max(1.0, abs(z))
            e = np.zeros(3)
            e[a] = h
            p0 = np.array([xc, yc, z])
            J[:, a] = (pin(p0 + e) - pin(p0 - e)) / (2 * h)
        C2 = J @ R @ S3 @ R.T @ J.T + 0.3 * np.eye(2)
        conic = np.linalg.inv(C2)
        mu = pin(pc)
        lam = np.linalg.eigvalsh(C2).max()
        out.append(dict(mx=mu[0], my=mu[1], A=conic[0, 0], B=conic[0, 1], C=conic[1, 1],
                        c00=C2[0, 0], c01=C2[0, 1], c11=C2[1, 1], depth=z, lam=lam))
    return {k: np.array([o[k] for o in out]) for k in out[0]}


def test_projection_matches_scipy_and_fd_jacobian(oracle_lib):
    s = synth.config_tiny()
    g = s.gaussians.subset(np.arange(400))
    for vi in range(s.n_views):
        cam = s.view(vi).camera
        p = O.project_f64(g, cam)
        ref = _np_project(g, cam)
        depth32, rect, touched = O.bin_f32(g, cam)
        vis = touched > 0
        assert vis.sum() > 100
        for key in ("mx", "my", "depth"):
            np.testing.assert_allclose(p[key][vis], ref[key][vis], rtol=1e-12, atol=1e-9)
        for key in ("c00", "c01", "c11", "A", "B", "C"):
            np.testing.assert_allclose(p[key][vis], ref[key][vis], rtol=2e-6, atol=1e-7)


def test_projection_clamp_branch(oracle_lib):
    # Gaussians far outside the field of view: the Jacobian is taken at the clamped point.
    cam = _cam(64, 64, 60.0, t=(0.0, 0.0, 2.0))
    g = _gauss([[3.0, 0.2, 0.0], [-2.5, -2.9, 0.5], [0.1, 2.0, 1.0]], [[0.3, 0.1, 0.2]] * 3,
               quats=synth.scenes._unit_quats(np.random.default_rng(5), 3).astype(np.float32))
    p = O.project_f64(g, cam)
    ref = _np_project(g, cam)
    for key in ("c00", "c01", "c11"):
        np.testing.assert_allclose(p[key], ref[key], rtol=2e-6)


def test_mirror_depth_and_rect_against_float64(oracle_lib):
    s = synth.config_tiny()
    g = s.gaussians
    cam = s.view(1).camera
    depth32, rect, touched = O.bin_f32(g, cam)
    ref = _np_project(g.subset(np.arange(1000)), cam)
    d64 = ref["depth"]
    ulp = np.spacing(np.abs(d64).astype(np.float32))
    assert np.all(np.abs(depth32[:1000].astype(np.float64) - d64) <= 4 * ulp)
    # rect from the float64 mean and covariance; the radius convention floors the eigenvalue
    # discriminant at 0.1, which can only enlarge the largest eigenvalue
    mid = 0.5 * (ref["c00"] + ref["c11"])
    det = ref["c00"] * ref["c11"] - ref["c01"] ** 2
    lam = mid + np.sqrt(np.maximum(0.1, mid * mid - det))
    assert np.all(lam >= ref["lam"] * (1 - 1e-12))
    r64 = np.ceil(3 * np.sqrt(lam))
    tx, ty = (cam.width + 15) // 16, (cam.height + 15) // 16
    x0 = np.clip(np.floor((ref["mx"] - r64) / 16), 0, tx)
    x1 = np.clip(np.floor((ref["mx"] + r64) / 16) + 1, 0, tx)
    y0 = np.clip(np.floor((ref["my"] - r64) / 16), 0, ty)
    y1 = np.clip(np.floor((ref["my"] + r64) / 16) + 1, 0, ty)
    rr = np.stack([x0, y0, x1, y1], 1).astype(np.int32)
    empty = (rr[:, 0] >= rr[:, 2]) | (rr[:, 1] >= rr[:, 3])
    rr[empty] = 0
    diff = np.any(rr != rect[:1000], axis=1)
    assert diff.mean() < 2e-3
    area = (rect[:, 2] - rect[:, 0]) * (rect[:, 3] - rect[:, 1])
    np.testing.assert_array_equal(touched, np.where(touched > 0, area, 0))


def test_tile_lists_are_sorted_membership(oracle_lib):
    s = synth.config_tiny()
    g = s.gaussians
    cam = s.view(2).camera
    depth32, rect, touched = O.bin_f32(g, cam)
    lst, ranges = O.tile_lists(g, cam)
    tx = (cam.width + 15) // 16
    assert lst.shape[0] == int(touched.sum())
    for t in range(ranges.shape[0]):
        x, y = t % tx, t // tx
        mem = np.nonzero((touched > 0) & (rect[:, 0] <= x) & (x < rect[:, 2]) & (rect[:, 1] <= y) & (y < rect[:, 3]))[0]
        want = mem[np.lexsort((mem, depth32[mem]))]
        np.testing.assert_array_equal(lst[ranges[t, 0]:ranges[t, 1]], want)


# ----------------------------------------------------------------------------
# closed forms
# ----------------------------------------------------------------------------

def _onaxis_alpha(W, H, f, s, z, o, mode="alpha"):
    sig2 = (f * s / z) ** 2 + 0.3
    r = math.ceil(3 * math.sqrt(sig2))
    cx, cy = W / 2.0, H / 2.0
    tx0, tx1 = math.floor((cx - r) / 16), math.floor((cx + r) / 16) + 1
    ty0, ty1 = math.floor((cy - r) / 16), math.floor((cy + r) / 16) + 1
    ys, xs = np.mgrid[0:H, 0:W]
    d2 = (xs + 0.5 - cx) ** 2 + (ys + 0.5 - cy) ** 2
    kern = np.exp(-0.5 * d2 / sig2)
    a = np.minimum(0.99, o * kern)
    inrect = (xs // 16 >= tx0) & (xs // 16 < tx1) & (ys // 16 >= ty0) & (ys // 16 < ty1)
    ok = inrect & (a >= 1 / 255)
    return np.where(ok, a, 0.0), np.where(ok, kern, 0.0)


@pytest.mark.parametrize("o,mode", [(0.8, O.ALPHA_T), (1.0, O.ALPHA_T), (0.8, O.KERNEL)])
def test_single_gaussian_two_segments(oracle_lib, o, mode):
    W = H = 64
    f, s, z = 60.0, 0.05, 2.0
    cam = _cam(W, H, f, t=(0, 0, z))
    g = _gauss([[0, 0, 0]], [[s, s, s]], op=[o])
    seg = np.where(np.arange(W)[None, :] < 30, 0, 1).astype(np.int32).repeat(H, 0)
    rng = np.random.default_rng(0)
    tab = rng.standard_normal((2, 8))
    tab /= np.linalg.norm(tab, axis=1, keepdims=True)
    v = synth.View(cam, seg, tab.astype(np.float32))
    # the inputs are float32: the closed form takes the rounded values
    alpha, kern = _onaxis_alpha(W, H, f, float(np.float32(s)), z, float(np.float32(o)))
    w = alpha if mode == O.ALPHA_T else kern
    WL, WR = w[seg == 0].sum(), w[seg == 1].sum()
    assert WL > 0 and WR > 0
    num, den, _ = O.lift(g, [v], weight_mode=mode)
    E = O.normalise(num, den)[0]
    want = (WL * v.table[0].astype(np.float64) + WR * v.table[1].astype(np.float64)) / (WL + WR)
    np.testing.assert_allclose(den[0], WL + WR, rtol=1e-12)
    np.testing.assert_allclose(E, want, rtol=1e-12, atol=1e-14)


def test_stack_of_cocentred_gaussians(oracle_lib):
    # Four isotropic Gaussians on the optical axis at increasing depth; index order is
    # shuffled so that only the depth sort gives the compositing order.
    W = H = 48
    f = 50.0
    depths = [2.0, 2.2, 2.4, 2.6]
    order = [2, 0, 3, 1]                  # Gaussian index -> depth rank
    z0 = 2.0
    means = [[0, 0, depths[r] - z0] for r in order]
    scales = [[0.2 * depths[r]] * 3 for r in order]      # screen sigma 10 px for all
    ops = [0.95, 0.9, 0.97, 0.8]
    g = _gauss(means, scales, op=ops)
    cam = _cam(W, H, f, t=(0, 0, z0))
    seg = np.zeros((H, W), np.int32)
    v = synth.View(cam, seg, np.ones((1, 4), np.float32))
    r = O.view_weights(g, v, per_pixel=True)
    # closed form per pixel, compositing in depth order with the early stop
    ys, xs = np.mgrid[0:H, 0:W]
    want = np.zeros(4)
    T = np.ones((H, W))
    alive = np.ones((H, W), bool)
    for rank in range(4):
        k = order.index(rank)
        z = depths[rank]
        sig2 = (f * float(np.float32(scales[k][0])) / (float(np.float32(z - z0)) + z0)) ** 2 + 0.3
        rad = math.ceil(3 * math.sqrt(sig2))
        lo, hi = math.floor((W / 2 - rad) / 16), math.floor((W / 2 + rad) / 16) + 1
        inrect = (xs // 16 >= lo) & (xs // 16 < hi) & (ys // 16 >= lo) & (ys // 16 < hi)
        d2 = (xs + 0.5 - W / 2) ** 2 + (ys + 0.5 - H / 2) ** 2
        a = np.minimum(0.99, float(np.float32(ops[k])) * np.exp(-0.5 * d2 / sig2))
        use = alive & inrect & (a >= 1 / 255)
        Tn = T * (1 - a)
        stop = use & (Tn < 1e-4)
        alive &= ~stop
        use &= ~stop
        want[k] = np.where(use, a * T, 0).sum()
        T = np.where(use, Tn, T)
    assert (~alive).any(), "the stack must trigger the early stop"
    np.testing.assert_allclose(r["B"][:, 0], want, rtol=1e-12)
    np.testing.assert_allclose(r["T_final"], T, rtol=1e-12)


# ----------------------------------------------------------------------------
# invariants
# ----------------------------------------------------------------------------

def test_weights_telescope_to_one_minus_T(oracle_lib):
    s = synth.config_tiny()
    for vi in range(2):
        r = O.view_weights(s.gaussians, s.view(vi), per_pixel=True)
        np.testing.assert_allclose(r["wsum_px"], 1.0 - r["T_final"], atol=1e-12)
        assert r["count_px"].max() > 10
        # masked sums: every pixel of these maps is in some segment
        assert abs(r["B"].sum() - r["wsum_px"].sum()) < 1e-9 * r["wsum_px"].sum()


def test_constant_features_reproduce_constant(oracle_lib):
    s = synth.small_scene(3, 3000, 3, 96, 80, 7, dim=16, empty_fraction=0.2)
    c = np.random.default_rng(1).standard_normal(16)
    c /= np.linalg.norm(c)
    views = []
    for v in s.views():
        views.append(synth.View(v.camera, v.seg, np.tile(c.astype(np.float32), (v.m, 1))))
    num, den, _ = O.lift(s.gaussians, views)
    E = O.normalise(num, den)
    ok = den > 0
    assert ok.sum() > 500
    np.testing.assert_allclose(E[ok], np.tile(c.astype(np.float32).astype(np.float64), (ok.sum(), 1)),
                               rtol=1e-12, atol=1e-13)


def test_view_order_invariance_and_literal_equals_factored(oracle_lib):
    s = synth.config_tiny()
    views = list(s.views())
    n1, d1, _ = O.lift(s.gaussians, views)
    n2, d2, _ = O.lift(s.gaussians, [views[i] for i in (3, 1, 0, 2)], threads=2)
    np.testing.assert_allclose(n2, n1, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(d2, d1, rtol=1e-12)
    nl, dl = None, None
    for v in views:
        nl, dl = O.view_literal(s.gaussians, v, num=nl, den=dl)
    np.testing.assert_allclose(nl, n1, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(dl, d1, rtol=1e-11)


def test_subset_accumulation_matches_full(oracle_lib):
    s = synth.config_tiny()
    sub = np.array([3, 17, 400, 4999, 2500])
    views = list(s.views())
    n1, d1, _ = O.lift(s.gaussians, views)
    ns, ds, _ = O.lift(s.gaussians, views, sub_ids=sub)
    np.testing.assert_allclose(ns, n1[sub], rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(ds, d1[sub], rtol=1e-13)


def test_tile_row_windows_partition_the_view(oracle_lib):
    # a window of tile rows composites exactly the whole view's pixels of those rows, and the
    # windows of a partition of the rows add up to the whole view's sums
    s = synth.small_scene(8, 2500, 1, 136, 90, 5, dim=8, surfaces=2)
    v = s.view(0)
    full = O.view_weights(s.gaussians, v, per_pixel=True)
    rows = (v.camera.height + 15) // 16
    B = np.zeros_like(full["B"])
    contrib = 0
    for ty0, ty1 in ((0, 2), (2, 3), (3, rows)):
        r = O.view_weights(s.gaussians, v, per_pixel=True, tile_rows=(ty0, ty1))
        y0, y1 = 16 * ty0, min(v.camera.height, 16 * ty1)
        np.testing.assert_array_equal(r["T_final"][y0:y1], full["T_final"][y0:y1])
        np.testing.assert_array_equal(r["count_px"][y0:y1], full["count_px"][y0:y1])
        B += r["B"]
        contrib += r["contributions"]
    assert contrib == full["contributions"] > 1000
    np.testing.assert_allclose(B, full["B"], rtol=1e-12, atol=1e-15)


def test_invalid_segment_id_rejected(oracle_lib):
    s = synth.config_tiny()
    v = s.view(0)
    seg = v.seg.copy()
    seg[5, 5] = v.m
    with pytest.raises(ValueError):
        O.view_weights(s.gaussians, synth.View(v.camera, seg, v.table))


# ----------------------------------------------------------------------------
# brute force
# ----------------------------------------------------------------------------

def _brute_B(g, view, mode=O.ALPHA_T):
    """Per pixel, every Gaussian whose tile rectangle holds the pixel's tile, in (float32 depth, index)
    order, composited in float64 with the numpy projection."""
    cam = view.camera
    depth32, rect, touched = O.bin_f32(g, cam)
    ref = _np_project(g, cam)
    B = np.zeros((g.n, view.m))
    Tf = np.ones((cam.height, cam.width))
    for py in range(cam.height):
        for px in range(cam.width):
            tx, ty = px // 16, py // 16
            cand = [k for k in range(g.n) if touched[k] and rect[k, 0] <= tx < rect[k, 2]
                    and rect[k, 1] <= ty < rect[k, 3]]
            cand.sort(key=lambda k: (depth32[k], k))
            T = 1.0
            for k in cand:
                dx, dy = ref["mx"][k] - (px + 0.5), ref["my"][k] - (py + 0.5)
                power = -0.5 * (ref["A"][k] * dx * dx + ref["C"][k] * dy * dy) - ref["B"][k] * dx * dy
                if power > 0:
                    continue
                kern = math.exp(power)
                a = min(0.99, float(g.opacities[k]) * kern)
                if a < 1 / 255:
                    continue
                Tn = T * (1 - a)
                if Tn < 1e-4:
                    break
                w = a * T if mode == O.ALPHA_T else kern
                j = view.seg[py, px]
                if j >= 0:
                    B[k, j] += w
                T = Tn
            Tf[py, px] = T
    return B, Tf


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_brute_force_tiny_scenes(oracle_lib, seed):
    rng = np.random.default_rng(100 + seed)
    n = 8
    means = rng.uniform(-0.3, 0.3, (n, 3))
    scales = np.exp(rng.normal(-2.5, 0.4, (n, 3)))
    quats = synth.scenes._unit_quats(rng, n)
    op = 1 / (1 + np.exp(-rng.standard_normal(n)))
    if seed == 2:
        means[3] = means[5]            # exact depth tie: index order decides
    g = _gauss(means, scales, quats, op)
    cam = synth.look_at([0.3, -2.0, 0.4], [0, 0, 0], 40, 36, 60.0)
    seg = synth.voronoi_segments(rng, 40, 36, 4)
    seg[seg == 3] = -1
    view = synth.View(cam, seg, np.eye(4, 6, dtype=np.float32))
    for mode in (O.ALPHA_T, O.KERNEL):
        Bb, Tb = _brute_B(g, view, mode)
        r = O.view_weights(g, view, weight_mode=mode, per_pixel=True)
        assert Bb.sum() > 0
        np.testing.assert_allclose(r["B"], Bb, rtol=2e-6, atol=1e-9)
        np.testing.assert_allclose(r["T_final"], Tb, rtol=2e-6, atol=1e-9)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_alpha_floor_decision(oracle_lib, seed):
    # one Gaussian per view: a pixel counts a contribution exactly when alpha >= 1/255 there. The
    # oracle takes that decision in float32 (a mirror of the compositing kernel's evaluation); it
    # must equal the float64 decision (alpha from the numpy projection) at every pixel whose alpha
    # is not within 1e-5 (relative) of the floor, with the floor's boundary crossing the image
    rng = np.random.default_rng(300 + seed)
    means = rng.uniform(-0.2, 0.2, (1, 3))
    scales = np.exp(rng.normal(-2.2, 0.5, (1, 3)))
    quats = synth.scenes._unit_quats(rng, 1)
    op = np.array([0.2 + 0.7 * rng.uniform()])
    g = _gauss(means, scales, quats, op)
    W, H = 72, 56
    cam = synth.look_at([0.2, -2.0, 0.3], [0, 0, 0], W, H, 60.0)
    view = synth.View(cam, np.zeros((H, W), np.int32), np.eye(1, 4, dtype=np.float32))
    r = O.view_weights(g, view, per_pixel=True)
    ref = _np_project(g, cam)
    px = np.arange(W) + 0.5
    py = np.arange(H) + 0.5
    dx = ref["mx"][0] - px[None, :]
    dy = ref["my"][0] - py[:, None]
    power = -0.5 * (ref["A"][0] * dx * dx + ref["C"][0] * dy * dy) - ref["B"][0] * dx * dy
    alpha = np.minimum(0.99, op[0] * np.exp(power))
    above = alpha >= 1 / 255
    clear = np.abs(alpha * 255.0 - 1.0) > 1e-5
    assert 20 < above.sum() < W * H - 20
    np.testing.assert_array_equal(r["count_px"][clear], above[clear].astype(np.int32))


# ----------------------------------------------------------------------------
# queries
# ----------------------------------------------------------------------------

def test_topk_matches_stable_argsort():
    rng = np.random.default_rng(7)
    E = rng.standard_normal((500, 32))
    E[10] = E[20]                      # exact tie: lower index first
    E[30] = 0.0                        # zero embedding: never returned
    den = rng.uniform(0.1, 2.0, 500)
    den[40] = 0.0                      # untouched: never returned
    q = E[10] / np.linalg.norm(E[10])
    ids, sc = O.topk(E, den, q, 10)
    cos = (E @ q) / np.maximum(np.linalg.norm(E, axis=1), 1e-300)
    cos[[30, 40]] = -np.inf
    want = np.argsort(-cos, kind="stable")[:10]
    np.testing.assert_array_equal(ids, want)
    assert ids[0] == 10 and ids[1] == 20
    np.testing.assert_allclose(sc, cos[want], rtol=1e-12)
