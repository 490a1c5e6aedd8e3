"""Python face of the CPU oracle (test infrastructure only).

Only the test-suite, the smoke check and the benchmark's CPU-baseline leg use
this module; the product path never imports it. It wraps the plain C oracle in
`slag_oracle.c` (float64 compositing, float32 binning mirror) and adds the two
steps that are library primitives:

* Aggregation (SLAG, Method section, "Semantic Embedding", Aggregation step):
  E_k = sum_views B_v[k] . E_v / sum_views sum_j B_v[k, j], where B_v[k, j]
  is the sum over the pixels of segment j of view v of the weights of
  Gaussian k. The product B_v . E_v is a float64 matmul.
* Query (same section, "Query processing for inference"): cosine similarity
  of a text vector with every aggregated embedding, top-k by descending score,
  ties to the lower Gaussian index.
"""
from __future__ import annotations

import concurrent.futures as cf
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "slag_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

ALPHA_T = 0
KERNEL = 1


def build(force: bool = False, extra_flags=()) -> str:
    """Compile the oracle with gcc (no fused multiply-add, strict IEEE)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC) \
            and not extra_flags:
        return _LIB
    out = _LIB if not extra_flags else _LIB.replace(".so", "_%x.so" % (hash(tuple(extra_flags)) & 0xffffffff))
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           *extra_flags, "-o", out, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    return out


class OCam(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float),
                ("cy", ctypes.c_float), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3),
                ("near_z", ctypes.c_float), ("far_z", ctypes.c_float)]


def _ocam(cam) -> OCam:
    c = OCam()
    c.fx, c.fy, c.cx, c.cy = cam.fx, cam.fy, cam.cx, cam.cy
    c.width, c.height = cam.width, cam.height
    c.R[:] = [float(x) for x in np.asarray(cam.R, np.float32).reshape(9)]
    c.t[:] = [float(x) for x in np.asarray(cam.t, np.float32).reshape(3)]
    c.near_z, c.far_z = cam.near, cam.far
    return c


def load(path: str | None = None):
    global _lib
    with _lock:
        if path is not None:
            return _bind(ctypes.CDLL(path))
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
        return _lib


def _bind(lib):
    P = ctypes.c_void_p
    i64, i32 = ctypes.c_int64, ctypes.c_int32
    lib.oracle_bin_f32.argtypes = [i64, P, P, P, ctypes.POINTER(OCam), P, P, P]
    lib.oracle_bin_f32.restype = None
    lib.oracle_tile_lists_f32.argtypes = [i64, P, P, P, ctypes.POINTER(OCam), i64, P, P]
    lib.oracle_tile_lists_f32.restype = i64
    lib.oracle_view_weights.argtypes = [i64, P, P, P, P, ctypes.POINTER(OCam), P, i32, ctypes.c_int,
                                        i64, P, P, P, P, P, P]
    lib.oracle_view_weights.restype = ctypes.c_int
    lib.oracle_view_weights_rows.argtypes = [i64, P, P, P, P, ctypes.POINTER(OCam), P, i32, ctypes.c_int,
                                             i64, P, P, P, P, P, P, i32, i32]
    lib.oracle_view_weights_rows.restype = ctypes.c_int
    lib.oracle_view_literal.argtypes = [i64, P, P, P, P, ctypes.POINTER(OCam), P, i32, P, i32,
                                        ctypes.c_int, P, P]
    lib.oracle_view_literal.restype = ctypes.c_int
    lib.oracle_project_f64.argtypes = [i64, P, P, P, P, ctypes.POINTER(OCam), P]
    lib.oracle_project_f64.restype = None
    return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _garr(g):
    return (np.ascontiguousarray(g.means, np.float32), np.ascontiguousarray(g.scales, np.float32),
            np.ascontiguousarray(g.quats, np.float32), np.ascontiguousarray(g.opacities, np.float32))


# ----------------------------------------------------------------------------
# binning mirror
# ----------------------------------------------------------------------------

def bin_f32(g, cam, lib=None):
    """float32 mirror of the projection's discrete outputs: depth, rect, tiles touched."""
    lib = lib or load()
    m, s, q, _ = _garr(g)
    n = m.shape[0]
    depth = np.empty(n, np.float32)
    rect = np.empty((n, 4), np.int32)
    touched = np.empty(n, np.uint32)
    c = _ocam(cam)
    lib.oracle_bin_f32(n, _p(m), _p(s), _p(q), ctypes.byref(c), _p(depth), _p(rect), _p(touched))
    return depth, rect, touched


def tile_lists(g, cam, lib=None):
    """Per-tile Gaussian lists sorted by (float32 depth, index) and [start, end) ranges."""
    lib = lib or load()
    m, s, q, _ = _garr(g)
    n = m.shape[0]
    c = _ocam(cam)
    tiles = ((cam.width + 15) // 16) * ((cam.height + 15) // 16)
    ranges = np.zeros((tiles, 2), np.int64)
    P = lib.oracle_tile_lists_f32(n, _p(m), _p(s), _p(q), ctypes.byref(c), 0, None, _p(ranges))
    if P == -1:
        raise MemoryError("oracle_tile_lists_f32")
    P = -(P + 2) if P < 0 else P
    lst = np.empty(max(P, 1), np.int32)
    got = lib.oracle_tile_lists_f32(n, _p(m), _p(s), _p(q), ctypes.byref(c), P, _p(lst), _p(ranges))
    assert got == P
    return lst[:P], ranges


def project_f64(g, cam, lib=None):
    """float64 projection: dict of mx, my, conic A/B/C, opacity, 2D covariance c00/c01/c11, depth."""
    lib = lib or load()
    m, s, q, o = _garr(g)
    n = m.shape[0]
    out = np.empty((n, 10), np.float64)
    c = _ocam(cam)
    lib.oracle_project_f64(n, _p(m), _p(s), _p(q), _p(o), ctypes.byref(c), _p(out))
    keys = ["mx", "my", "A", "B", "C", "op", "c00", "c01", "c11", "depth"]
    return {k: out[:, i].copy() for i, k in enumerate(keys)}


# ----------------------------------------------------------------------------
# compositing + aggregation
# ----------------------------------------------------------------------------

def view_weights(g, view, weight_mode=ALPHA_T, sub_ids=None, per_pixel=False, lib=None, tile_rows=None):
    """B (n_sub x M) of one view, plus optional per-pixel T_final / sum w / count.

    tile_rows = (ty0, ty1) composites only the pixels of those tile rows (a bounded sample of
    the view; each of its pixels gets the whole view's result); per-pixel outputs of the other
    rows are left unset."""
    lib = lib or load()
    m, s, q, o = _garr(g)
    n = m.shape[0]
    cam = view.camera
    seg = np.ascontiguousarray(view.seg, np.int32)
    M = int(view.table.shape[0])
    sub = None if sub_ids is None else np.ascontiguousarray(sub_ids, np.int64)
    n_sub = n if sub is None else sub.shape[0]
    B = np.zeros((n_sub, M), np.float64)
    H, W = cam.height, cam.width
    Tf = np.empty((H, W), np.float64) if per_pixel else None
    ws = np.empty((H, W), np.float64) if per_pixel else None
    cnt = np.empty((H, W), np.int32) if per_pixel else None
    stats = np.zeros(2, np.int64)
    c = _ocam(cam)
    if tile_rows is None:
        rc = lib.oracle_view_weights(n, _p(m), _p(s), _p(q), _p(o), ctypes.byref(c), _p(seg), M,
                                     weight_mode, n_sub, _p(sub), _p(B), _p(Tf), _p(ws), _p(cnt), _p(stats))
    else:
        rc = lib.oracle_view_weights_rows(n, _p(m), _p(s), _p(q), _p(o), ctypes.byref(c), _p(seg), M,
                                          weight_mode, n_sub, _p(sub), _p(B), _p(Tf), _p(ws), _p(cnt), _p(stats),
                                          int(tile_rows[0]), int(tile_rows[1]))
    if rc == -2:
        raise ValueError("segment id outside [-1, M)")
    if rc != 0:
        raise MemoryError("oracle_view_weights")
    out = dict(B=B, P=int(stats[0]), contributions=int(stats[1]))
    if per_pixel:
        out.update(T_final=Tf, wsum_px=ws, count_px=cnt)
    return out


def view_literal(g, view, weight_mode=ALPHA_T, num=None, den=None, lib=None):
    """Literal form: num += sum_p w E_seg(p), den += sum_p w, one contribution at a time."""
    lib = lib or load()
    m, s, q, o = _garr(g)
    n = m.shape[0]
    table = np.ascontiguousarray(view.table, np.float32)
    D = table.shape[1]
    num = np.zeros((n, D), np.float64) if num is None else num
    den = np.zeros(n, np.float64) if den is None else den
    c = _ocam(view.camera)
    seg = np.ascontiguousarray(view.seg, np.int32)
    rc = lib.oracle_view_literal(n, _p(m), _p(s), _p(q), _p(o), ctypes.byref(c), _p(seg),
                                 table.shape[0], _p(table), D, weight_mode, _p(num), _p(den))
    if rc != 0:
        raise RuntimeError("oracle_view_literal rc=%d" % rc)
    return num, den


def lift(g, views, weight_mode=ALPHA_T, sub_ids=None, threads=1, lib=None, tile_rows=None):
    """Factored aggregation over `views` (an iterable of View).

    Returns (num, den, info): num (n_sub x D) = sum_v B_v . E_v, den (n_sub) =
    sum_v sum_j B_v, info = per-view P and contribution counts. Views are
    spread over `threads` host threads (the C oracle runs without the GIL),
    one accumulator per thread, summed at the end. tile_rows = (ty0, ty1)
    limits every view to the pixels of those tile rows (a bounded sample).
    """
    lib = lib or load()
    views = list(views)
    n_sub = g.n if sub_ids is None else len(sub_ids)
    D = views[0].table.shape[1] if views else 0

    def work(chunk):
        num = np.zeros((n_sub, D), np.float64)
        den = np.zeros(n_sub, np.float64)
        info = []
        for v in chunk:
            r = view_weights(g, v, weight_mode, sub_ids, lib=lib, tile_rows=tile_rows)
            num += r["B"] @ v.table.astype(np.float64)
            den += r["B"].sum(axis=1)
            info.append((r["P"], r["contributions"]))
        return num, den, info

    threads = max(1, min(threads, len(views)))
    chunks = [views[i::threads] for i in range(threads)]
    if threads == 1:
        parts = [work(chunks[0])]
    else:
        with cf.ThreadPoolExecutor(threads) as ex:
            parts = list(ex.map(work, chunks))
    num = sum(p[0] for p in parts)
    den = sum(p[1] for p in parts)
    info = [x for p in parts for x in p[2]]
    return num, den, info


def normalise(num, den):
    """E_k = num_k / den_k; Gaussians no view touched (den = 0) get the zero vector."""
    E = np.zeros_like(num)
    ok = den > 0
    E[ok] = num[ok] / den[ok, None]
    return E


def topk(E, den, q, k):
    """Top-k Gaussians by cosine with q (descending, ties to the lower index).

    Gaussians with den = 0 or a zero embedding are not candidates.
    """
    E = np.asarray(E, np.float64)
    nrm = np.linalg.norm(E, axis=1)
    ok = (np.asarray(den) > 0) & (nrm > 0)
    idx = np.nonzero(ok)[0]
    sc = (E[idx] @ np.asarray(q, np.float64)) / nrm[idx]
    order = np.lexsort((idx, -sc))[:k]
    return idx[order], sc[order]
