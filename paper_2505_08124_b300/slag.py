"""Thin Python binding of libslag (ctypes; argument marshalling only).

Every step of the lifting path runs in the library's CUDA kernels; this
module only converts arguments. Host inputs are numpy arrays; device inputs
are torch CUDA tensors (passed by data pointer). There is no fallback: when
libslag.so is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libslag.so")
CHECKED_LIB_PATH = os.path.join(_HERE, "libslag_checks.so")   # compiled with -DSLAG_CHECKS

OK = 0
ERR_INVALID_ARG, ERR_STATE, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_CAPACITY = 1, 2, 3, 4, 5, 6
_NAMES = {1: "INVALID_ARG", 2: "STATE", 3: "OOM", 4: "CUDA", 5: "TIMEOUT", 6: "CAPACITY"}
WEIGHT_ALPHA_T, WEIGHT_KERNEL = 0, 1
PREC_FP32 = 0
PREC_BF16 = 1
PREC_LATENT32 = 2
PREC_LINEAR32 = 3
FLAG_EMBEDDINGS_ON_HOST = 1


class SlagError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("slag error %s (%d): %s" % (_NAMES.get(status, "?"), status, msg))
        self.status = status


class CCamera(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float),
                ("cy", ctypes.c_float), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3),
                ("near_z", ctypes.c_float), ("far_z", ctypes.c_float)]


class CGaussians(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("means", ctypes.c_void_p), ("scales", ctypes.c_void_p),
                ("quats", ctypes.c_void_p), ("opacities", ctypes.c_void_p), ("on_device", ctypes.c_int32)]


class COptions(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("precision", ctypes.c_int32), ("weight_mode", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("cuda_stream", ctypes.c_void_p)]


class CView(ctypes.Structure):
    _fields_ = [("camera", ctypes.c_void_p), ("seg_ids", ctypes.c_void_p), ("seg_table", ctypes.c_void_p),
                ("M", ctypes.c_int32), ("on_device", ctypes.c_int32)]


class CStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("views", "pairs", "contributions", "triples", "columns",
                                               "last_pairs", "last_contributions", "touched",
                                               "evaluations", "executed", "resized_views",
                                               "recomposited_views")]


_lib = None

EXPORTS = ("slag_create", "slag_add_view", "slag_finalize", "slag_query", "slag_query_batch", "slag_reset",
           "slag_get_stats", "slag_last_error", "slag_destroy", "slag_bin_view", "slag_render_debug",
           "slag_set_profiling", "slag_get_profile", "slag_noalloc_query_topk", "slag_kernel_launches",
           "slag_export_partitions", "slag_latent_param_count", "slag_latent_train", "slag_latent_apply",
           "slag_set_latent", "slag_add_views_batched", "slag_set_autotune", "slag_finalize_async",
           "slag_wait_outputs", "slag_set_profiling_stages", "slag_bin_view_bins", "slag_composite_trace",
           "slag_save_state", "slag_load_state", "slag_merge_state", "slag_state_merge_host",
           "slag_check_wait_timeout", "slag_is_checked_build", "slag_debug_force_pair_capacity",
           "slag_linear_param_count", "slag_linear_code_fit", "slag_set_linear_code", "slag_query_threshold",
           "slag_set_device_budget", "slag_set_graphs")
STAGES = ("project", "bin", "composite", "consume", "log_sort", "aggregate", "query")


class CProfile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * len(STAGES)), ("spans", ctypes.c_int64 * len(STAGES)),
                ("busy_ms", ctypes.c_double * len(STAGES))]


def load_library(path: str = LIB_PATH):
    """Load libslag.so (once). Raises if it is missing: there is no other implementation."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libslag.so not found at %s: build it with `python -m paper_2505_08124_b300.build`"
                           % path)
    lib = ctypes.CDLL(path)
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.slag_create.argtypes = [ctypes.POINTER(CGaussians), ctypes.POINTER(COptions), ctypes.POINTER(P)]
    lib.slag_add_view.argtypes = [P, ctypes.POINTER(CCamera), P, P, i32, i32]
    lib.slag_finalize.argtypes = [P, P, P, i32]
    lib.slag_finalize_async.argtypes = [P, P, P, i32]
    lib.slag_wait_outputs.argtypes = [P]
    lib.slag_query.argtypes = [P, P, i32, P, P, P]
    lib.slag_query_batch.argtypes = [P, P, i32, i32, P, P, P, i32]
    lib.slag_query_threshold.argtypes = [P, P, ctypes.c_float, P, i64, ctypes.POINTER(i64), i32]
    lib.slag_reset.argtypes = [P]
    lib.slag_get_stats.argtypes = [P, ctypes.POINTER(CStats)]
    lib.slag_last_error.argtypes = [P]
    lib.slag_last_error.restype = ctypes.c_char_p
    lib.slag_destroy.argtypes = [P]
    lib.slag_destroy.restype = None
    lib.slag_bin_view.argtypes = [P, ctypes.POINTER(CCamera), P, P, P, i64, P]
    lib.slag_render_debug.argtypes = [P, ctypes.POINTER(CCamera), P, P, P]
    lib.slag_check_wait_timeout.argtypes = [P, i32, i32]
    lib.slag_is_checked_build.argtypes = []
    lib.slag_debug_force_pair_capacity.argtypes = [P, i64]
    lib.slag_save_state.argtypes = [P, P, i64, ctypes.POINTER(i64)]
    lib.slag_load_state.argtypes = [P, P, i64]
    lib.slag_merge_state.argtypes = [P, P, i64]
    lib.slag_state_merge_host.argtypes = [P, i64, P, i64, P, i64, ctypes.POINTER(i64)]
    lib.slag_bin_view_bins.argtypes = [P, ctypes.POINTER(CCamera), i32, P, P, i64, P]
    lib.slag_composite_trace.argtypes = [P, ctypes.POINTER(CCamera), P, P, i64, P]
    lib.slag_set_profiling.argtypes = [P, i32]
    lib.slag_set_profiling_stages.argtypes = [P, ctypes.c_uint32]
    lib.slag_get_profile.argtypes = [P, ctypes.POINTER(CProfile), i32]
    lib.slag_export_partitions.argtypes = [P, ctypes.c_char_p, i32, i32, i64, ctypes.POINTER(i64)]
    lib.slag_latent_param_count.argtypes = [i32]
    lib.slag_latent_param_count.restype = i64
    lib.slag_latent_train.argtypes = [P, i64, i32, i32, i32, ctypes.c_float, ctypes.c_uint64, i32, P, P, P]
    lib.slag_latent_apply.argtypes = [P, i32, P, i64, i32, P, P]
    lib.slag_set_latent.argtypes = [P, P]
    lib.slag_linear_param_count.argtypes = [i32]
    lib.slag_linear_param_count.restype = i64
    lib.slag_linear_code_fit.argtypes = [P, i64, i32, i32, P, P, P]
    lib.slag_set_linear_code.argtypes = [P, P]
    lib.slag_set_device_budget.argtypes = [P, i64]
    lib.slag_add_views_batched.argtypes = [i32, P, P, P, ctypes.POINTER(i32)]
    lib.slag_set_autotune.argtypes = [P, i32]
    lib.slag_set_graphs.argtypes = [P, i32]
    lib.slag_kernel_launches.argtypes = []
    lib.slag_kernel_launches.restype = ctypes.c_uint64
    lib.slag_noalloc_query_topk.argtypes = [P, i64, i32, P, P, i32, i32, P, P, P, P]
    for name in EXPORTS:
        f = getattr(lib, name)
        if f.restype is ctypes.c_int:   # default
            f.restype = ctypes.c_int
    _lib = lib
    return lib


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype):
    """(pointer, on_device, keepalive) of a numpy array or a torch CUDA tensor."""
    if x is None:
        return None, 0, None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("torch tensors must be contiguous")
        want = {np.float32: "torch.float32", np.int32: "torch.int32", np.int64: "torch.int64"}[dtype]
        if str(x.dtype) != want:
            raise TypeError("expected %s, got %s" % (want, x.dtype))
        return ctypes.c_void_p(x.data_ptr()), 1 if x.is_cuda else 0, x
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data_as(ctypes.c_void_p), 0, a


def camera_struct(cam) -> CCamera:
    c = CCamera()
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    c.R[:] = [float(v) for v in np.asarray(cam.R, np.float32).reshape(9)]
    c.t[:] = [float(v) for v in np.asarray(cam.t, np.float32).reshape(3)]
    c.near_z, c.far_z = float(getattr(cam, "near", 0.01)), float(getattr(cam, "far", 100.0))
    return c


def noalloc_query_topk(E, wsum, Q, k: int, out_ids, out_scores, out_count=None, stream: Optional[int] = None):
    """Allocation-free cosine top-k on torch CUDA tensors (see slag_noalloc_query_topk).

    Fills out_ids (B x k int64), out_scores (B x k float32) and out_count (B int32, optional)
    asynchronously in `stream`; returns the status code. Every array must be a contiguous CUDA
    tensor on the current device with the shape the call implies (E: n x dim, wsum: n, Q:
    B x dim); anything else raises before the library is called."""
    lib = load_library()
    import torch
    dev = torch.cuda.current_device()

    def dev_tensor(x, name, dtype, shape):
        if not (_is_torch(x) and x.is_cuda and x.device.index == dev):
            raise ValueError("%s must be a CUDA tensor on the current device (cuda:%d)" % (name, dev))
        if tuple(x.shape) != tuple(shape):
            raise ValueError("%s has shape %s, expected %s" % (name, tuple(x.shape), tuple(shape)))
        return _ptr(x, dtype)[0]

    if not (_is_torch(E) and E.dim() == 2) or not (_is_torch(Q) and Q.dim() == 2):
        raise ValueError("E and Q must be 2-d torch CUDA tensors")
    n, dim = int(E.shape[0]), int(E.shape[1])
    B = int(Q.shape[0])
    k = int(k)
    ep = dev_tensor(E, "E", np.float32, (n, dim))
    wp = None if wsum is None else dev_tensor(wsum, "wsum", np.float32, (n,))
    qp = dev_tensor(Q, "Q", np.float32, (B, dim))
    ip = dev_tensor(out_ids, "out_ids", np.int64, (B, k))
    sp = dev_tensor(out_scores, "out_scores", np.float32, (B, k))
    cp = None if out_count is None else dev_tensor(out_count, "out_count", np.int32, (B,))
    return lib.slag_noalloc_query_topk(ep, n, dim, wp, qp, B, k, ip, sp, cp,
                                       ctypes.c_void_p(stream) if stream else None)


class Lifter:
    """One lifting context: a fixed Gaussian set, views added one at a time."""

    def __init__(self, gaussians, dim: int = 512, weight_mode: int = WEIGHT_ALPHA_T,
                 stream: Optional[int] = None, precision: int = PREC_FP32, embeddings_on_host: bool = False,
                 latent_params=None, linear_code=None):
        self._lib = load_library()
        self.n = int(gaussians.means.shape[0])
        self.dim = int(dim)
        ptrs = [_ptr(getattr(gaussians, k), np.float32) for k in ("means", "scales", "quats", "opacities")]
        dev = {p[1] for p in ptrs}
        if len(dev) != 1:
            raise ValueError("Gaussian arrays must all be on the host or all on the device")
        g = CGaussians(self.n, ptrs[0][0], ptrs[1][0], ptrs[2][0], ptrs[3][0], dev.pop())
        flags = FLAG_EMBEDDINGS_ON_HOST if embeddings_on_host else 0
        o = COptions(self.dim, int(precision), int(weight_mode), flags, ctypes.c_void_p(stream) if stream else None)
        h = ctypes.c_void_p()
        rc = self._lib.slag_create(ctypes.byref(g), ctypes.byref(o), ctypes.byref(h))
        if rc != OK:
            raise SlagError(rc, "slag_create")
        self._h = h
        if latent_params is not None:
            lp = np.ascontiguousarray(latent_params, np.float32)
            self._check(self._lib.slag_set_latent(self._h, lp.ctypes.data_as(ctypes.c_void_p)), "slag_set_latent")
        if linear_code is not None:
            lc = np.ascontiguousarray(linear_code, np.float32)
            if lc.size != linear_param_count(self.dim):
                raise ValueError("linear code has %d parameters, expected %d" % (lc.size, linear_param_count(self.dim)))
            self._check(self._lib.slag_set_linear_code(self._h, lc.ctypes.data_as(ctypes.c_void_p)),
                        "slag_set_linear_code")

    # -- helpers --------------------------------------------------------------
    def _check(self, rc: int, what: str):
        if rc != OK:
            raise SlagError(rc, "%s: %s" % (what, self._lib.slag_last_error(self._h).decode()))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.slag_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- the path -------------------------------------------------------------
    def add_view(self, camera, seg, table):
        sp, sdev, sk = _ptr(seg, np.int32)
        tp, tdev, tk = _ptr(table, np.float32)
        if sdev != tdev:
            raise ValueError("segment map and table must both be host or both device")
        M = int(table.shape[0])
        if int(table.shape[1]) != self.dim:
            raise ValueError("table has %d columns, context dim is %d" % (table.shape[1], self.dim))
        if tuple(seg.shape) != (int(camera.height), int(camera.width)):
            raise ValueError("segment map shape %s does not match the camera" % (tuple(seg.shape),))
        c = camera_struct(camera)
        self._check(self._lib.slag_add_view(self._h, ctypes.byref(c), sp, tp, M, sdev), "slag_add_view")
        del sk, tk

    def finalize(self, out_emb=None, out_wsum=None, want_emb: bool = True):
        """Returns (E, wsum). With torch CUDA outputs given, fills them; else returns numpy arrays."""
        if out_emb is None and out_wsum is None:
            E = np.empty((self.n, self.dim), np.float32) if want_emb else None
            w = np.empty(self.n, np.float32)
            ep = E.ctypes.data_as(ctypes.c_void_p) if E is not None else None
            self._check(self._lib.slag_finalize(self._h, ep, w.ctypes.data_as(ctypes.c_void_p), 0), "slag_finalize")
            return E, w
        ep, edev, _ = _ptr(out_emb, np.float32)
        wp, wdev, _ = _ptr(out_wsum, np.float32)
        dev = edev if out_emb is not None else wdev
        self._check(self._lib.slag_finalize(self._h, ep, wp, dev), "slag_finalize")
        return out_emb, out_wsum

    def finalize_async(self, out_emb=None, out_wsum=None):
        """slag_finalize_async: fills out_emb / out_wsum (numpy arrays, pinned for overlap, or torch
        tensors) once wait_outputs() returns; the embeddings are queryable on return."""
        for x in (out_emb, out_wsum):
            # the copies land later: a converted temporary would be written after it is gone
            if isinstance(x, np.ndarray) and not (x.dtype == np.float32 and x.flags.c_contiguous):
                raise ValueError("asynchronous outputs must be C-contiguous float32 arrays")
        ep, edev, _ = _ptr(out_emb, np.float32)
        wp, wdev, _ = _ptr(out_wsum, np.float32)
        dev = edev if out_emb is not None else wdev
        self._check(self._lib.slag_finalize_async(self._h, ep, wp, dev), "slag_finalize_async")

    def wait_outputs(self):
        self._check(self._lib.slag_wait_outputs(self._h), "slag_wait_outputs")

    def query(self, q, k: int):
        q = np.ascontiguousarray(q, np.float32)
        ids = np.empty(k, np.int64)
        sc = np.empty(k, np.float32)
        cnt = ctypes.c_int32()
        self._check(self._lib.slag_query(self._h, q.ctypes.data_as(ctypes.c_void_p), k,
                                         ids.ctypes.data_as(ctypes.c_void_p), sc.ctypes.data_as(ctypes.c_void_p),
                                         ctypes.byref(cnt)), "slag_query")
        return ids[:cnt.value], sc[:cnt.value]

    def query_threshold(self, q, threshold: float = 0.28):
        """Ids (increasing) of the Gaussians whose cosine with q is at least `threshold`."""
        qa = np.ascontiguousarray(q, np.float32)
        qp = qa.ctypes.data_as(ctypes.c_void_p)
        cnt = ctypes.c_int64()
        self._check(self._lib.slag_query_threshold(self._h, qp, float(threshold), None, 0, ctypes.byref(cnt), 0),
                    "slag_query_threshold")
        ids = np.empty(max(cnt.value, 1), np.int64)
        self._check(self._lib.slag_query_threshold(self._h, qp, float(threshold), ids.ctypes.data_as(ctypes.c_void_p),
                                                   ids.size, ctypes.byref(cnt), 0), "slag_query_threshold")
        return ids[:cnt.value]

    def query_batch(self, Q, k: int, out_ids=None, out_scores=None, out_count=None):
        """Host numpy Q -> (ids, scores, count) numpy; torch CUDA Q -> fills the given torch outputs."""
        B = int(Q.shape[0])
        if _is_torch(Q) and Q.is_cuda:
            qp, _, _ = _ptr(Q, np.float32)
            ip, _, _ = _ptr(out_ids, np.int64)
            sp, _, _ = _ptr(out_scores, np.float32)
            cp, _, _ = _ptr(out_count, np.int32)
            self._check(self._lib.slag_query_batch(self._h, qp, B, k, ip, sp, cp, 1), "slag_query_batch")
            return out_ids, out_scores, out_count
        Qa = np.ascontiguousarray(Q, np.float32)
        ids = np.empty((B, k), np.int64)
        sc = np.empty((B, k), np.float32)
        cnt = np.empty(B, np.int32)
        self._check(self._lib.slag_query_batch(self._h, Qa.ctypes.data_as(ctypes.c_void_p), B, k,
                                               ids.ctypes.data_as(ctypes.c_void_p),
                                               sc.ctypes.data_as(ctypes.c_void_p),
                                               cnt.ctypes.data_as(ctypes.c_void_p), 0), "slag_query_batch")
        return ids, sc, cnt

    def reset(self):
        self._check(self._lib.slag_reset(self._h), "slag_reset")

    def set_device_budget(self, nbytes: int):
        """Device bytes the out-of-core finalize may hold for output rows at a time (0 = default)."""
        self._check(self._lib.slag_set_device_budget(self._h, int(nbytes)), "slag_set_device_budget")

    def set_autotune(self, on: bool = True):
        self._check(self._lib.slag_set_autotune(self._h, 1 if on else 0), "slag_set_autotune")

    def set_graphs(self, on: bool = True):
        """Replay captured CUDA graphs for views sized on the device (on by default)."""
        self._check(self._lib.slag_set_graphs(self._h, 1 if on else 0), "slag_set_graphs")

    def export_partitions(self, directory: str, cells_x: int, cells_y: int, chunk_gaussians: int = 0) -> int:
        """Per-area embedding files of the touched Gaussians (see slag_export_partitions); returns
        the number of records written."""
        written = ctypes.c_int64()
        self._check(self._lib.slag_export_partitions(self._h, os.fsencode(directory), int(cells_x), int(cells_y),
                                                     int(chunk_gaussians), ctypes.byref(written)),
                    "slag_export_partitions")
        return int(written.value)

    def check_wait_timeout(self, limit_us: int, complete: bool = False) -> int:
        """Runs the bounded-wait check (slag_check_wait_timeout); returns the status code."""
        return int(self._lib.slag_check_wait_timeout(self._h, int(limit_us), 1 if complete else 0))

    def debug_force_pair_capacity(self, cap: int) -> int:
        """Checked build only (slag_debug_force_pair_capacity); returns the status code."""
        return int(self._lib.slag_debug_force_pair_capacity(self._h, int(cap)))

    def save_state(self) -> np.ndarray:
        """The accumulated state (slag_save_state) as a uint8 array."""
        size = ctypes.c_int64()
        self._check(self._lib.slag_save_state(self._h, None, 0, ctypes.byref(size)), "slag_save_state")
        buf = np.empty(size.value, np.uint8)
        self._check(self._lib.slag_save_state(self._h, buf.ctypes.data_as(ctypes.c_void_p), buf.size,
                                              ctypes.byref(size)), "slag_save_state")
        return buf

    def load_state(self, state):
        buf = np.ascontiguousarray(np.frombuffer(state, np.uint8) if isinstance(state, (bytes, bytearray)) else state,
                                   np.uint8)
        self._check(self._lib.slag_load_state(self._h, buf.ctypes.data_as(ctypes.c_void_p), buf.size),
                    "slag_load_state")

    def merge_state(self, state):
        buf = np.ascontiguousarray(np.frombuffer(state, np.uint8) if isinstance(state, (bytes, bytearray)) else state,
                                   np.uint8)
        self._check(self._lib.slag_merge_state(self._h, buf.ctypes.data_as(ctypes.c_void_p), buf.size),
                    "slag_merge_state")

    def stats(self) -> dict:
        s = CStats()
        self._check(self._lib.slag_get_stats(self._h, ctypes.byref(s)), "slag_get_stats")
        return {k: int(getattr(s, k)) for k, _ in CStats._fields_}

    # -- diagnostics ----------------------------------------------------------
    def set_profiling(self, on: bool = True, stages=None):
        """Per-stage timing on or off; `stages` (names from STAGES) limits it to those stages."""
        if stages is None:
            self._check(self._lib.slag_set_profiling(self._h, 1 if on else 0), "slag_set_profiling")
            return
        mask = 0
        for name in stages:
            mask |= 1 << STAGES.index(name)
        self._check(self._lib.slag_set_profiling_stages(self._h, mask if on else 0), "slag_set_profiling_stages")

    def profile(self, reset: bool = False) -> dict:
        """{stage: (summed span ms, spans)} from events recorded in the streams that run each stage."""
        return {k: v[:2] for k, v in self.profile_busy(reset).items()}

    def profile_busy(self, reset: bool = False) -> dict:
        """{stage: (summed span ms, spans, busy ms)}; busy ms is the union of the stage's spans
        (overlapping views make the summed ms larger than it)."""
        p = CProfile()
        self._check(self._lib.slag_get_profile(self._h, ctypes.byref(p), 1 if reset else 0), "slag_get_profile")
        return {name: (float(p.ms[i]), int(p.spans[i]), float(p.busy_ms[i])) for i, name in enumerate(STAGES)}

    def bin_view(self, camera):
        """(tiles_touched[n], list[P] caller ids grouped by tile, ranges[tiles, 2])."""
        c = camera_struct(camera)
        P = ctypes.c_int64()
        self._check(self._lib.slag_bin_view(self._h, ctypes.byref(c), None, ctypes.byref(P), None, 0, None),
                    "slag_bin_view")
        tiles = ((int(camera.width) + 15) // 16) * ((int(camera.height) + 15) // 16)
        touched = np.empty(self.n, np.uint32)
        lst = np.empty(max(P.value, 1), np.int32)
        rng = np.empty((tiles, 2), np.int64)
        self._check(self._lib.slag_bin_view(self._h, ctypes.byref(c), touched.ctypes.data_as(ctypes.c_void_p),
                                            ctypes.byref(P), lst.ctypes.data_as(ctypes.c_void_p), lst.shape[0],
                                            rng.ctypes.data_as(ctypes.c_void_p)), "slag_bin_view")
        return touched, lst[:P.value], rng

    def bin_view_bins(self, camera, bin_shift: int):
        """(list[P] caller ids grouped by bin, ranges[bins, 2]) of 2^bin_shift x 2^bin_shift-tile bins."""
        c = camera_struct(camera)
        P = ctypes.c_int64()
        self._check(self._lib.slag_bin_view_bins(self._h, ctypes.byref(c), int(bin_shift), ctypes.byref(P), None, 0,
                                                 None), "slag_bin_view_bins")
        tx, ty = (int(camera.width) + 15) // 16, (int(camera.height) + 15) // 16
        bins = (((tx - 1) >> bin_shift) + 1) * (((ty - 1) >> bin_shift) + 1)
        lst = np.empty(max(P.value, 1), np.int32)
        rng = np.empty((bins, 2), np.int64)
        self._check(self._lib.slag_bin_view_bins(self._h, ctypes.byref(c), int(bin_shift), ctypes.byref(P),
                                                 lst.ctypes.data_as(ctypes.c_void_p), lst.shape[0],
                                                 rng.ctypes.data_as(ctypes.c_void_p)), "slag_bin_view_bins")
        return lst[:P.value], rng

    def composite_trace(self, camera):
        """(list[P] caller ids staged per tile by the compositing kernel, ranges[tiles, 2])."""
        c = camera_struct(camera)
        P = ctypes.c_int64()
        self._check(self._lib.slag_composite_trace(self._h, ctypes.byref(c), ctypes.byref(P), None, 0, None),
                    "slag_composite_trace")
        tiles = ((int(camera.width) + 15) // 16) * ((int(camera.height) + 15) // 16)
        lst = np.full(max(P.value, 1), -1, np.int32)
        rng = np.empty((tiles, 2), np.int64)
        self._check(self._lib.slag_composite_trace(self._h, ctypes.byref(c), ctypes.byref(P),
                                                   lst.ctypes.data_as(ctypes.c_void_p), lst.shape[0],
                                                   rng.ctypes.data_as(ctypes.c_void_p)), "slag_composite_trace")
        return lst[:P.value], rng

    def render_debug(self, camera):
        """Per pixel (final transmittance, sum of weights, contributor count)."""
        c = camera_struct(camera)
        H, W = int(camera.height), int(camera.width)
        T = np.empty((H, W), np.float32)
        ws = np.empty((H, W), np.float32)
        cnt = np.empty((H, W), np.int32)
        self._check(self._lib.slag_render_debug(self._h, ctypes.byref(c), T.ctypes.data_as(ctypes.c_void_p),
                                                ws.ctypes.data_as(ctypes.c_void_p),
                                                cnt.ctypes.data_as(ctypes.c_void_p)), "slag_render_debug")
        return T, ws, cnt


def kernel_launches() -> int:
    """Kernel launches issued by libslag so far (process-wide running count)."""
    return int(load_library().slag_kernel_launches())


def read_partitions(directory: str) -> dict:
    """Reads the files of slag_export_partitions: {(cx, cy): {"bounds": (x0, x1, y0, y1),
    "ids": int64[count], "wsum": float32[count], "E": float32[count, D]}}."""
    out = {}
    with open(os.path.join(directory, "index.txt")) as f:
        lines = [ln.split() for ln in f if ln.strip()]
    for cx, cy, count, x0, x1, y0, y1, name in lines:
        with open(os.path.join(directory, name), "rb") as f:
            raw = f.read()
        if raw[:8] != b"SLAGPART":
            raise ValueError("%s: not a partition file" % name)
        ver, D = np.frombuffer(raw, np.uint32, 2, 8)
        cnt = int(np.frombuffer(raw, np.int64, 1, 16)[0])
        bounds = tuple(float(x) for x in np.frombuffer(raw, np.float32, 4, 24))
        if ver != 1 or cnt != int(count):
            raise ValueError("%s: version %d, count %d (index says %s)" % (name, ver, cnt, count))
        rec = np.dtype([("id", "<i8"), ("wsum", "<f4"), ("E", "<f4", (int(D),))])
        r = np.frombuffer(raw, rec, cnt, 40)
        out[(int(cx), int(cy))] = {"bounds": bounds, "ids": r["id"].copy(), "wsum": r["wsum"].copy(),
                                   "E": r["E"].copy()}
    return out


def state_merge_host(a, b) -> np.ndarray:
    """Merges two saved states on the host (slag_state_merge_host); no GPU is needed."""
    lib = load_library()
    A = np.ascontiguousarray(np.frombuffer(a, np.uint8) if isinstance(a, (bytes, bytearray)) else a, np.uint8)
    B = np.ascontiguousarray(np.frombuffer(b, np.uint8) if isinstance(b, (bytes, bytearray)) else b, np.uint8)
    size = ctypes.c_int64()
    pa, pb = A.ctypes.data_as(ctypes.c_void_p), B.ctypes.data_as(ctypes.c_void_p)
    rc = lib.slag_state_merge_host(pa, A.size, pb, B.size, None, 0, ctypes.byref(size))
    if rc != OK:
        raise SlagError(rc, "slag_state_merge_host")
    out = np.empty(size.value, np.uint8)
    rc = lib.slag_state_merge_host(pa, A.size, pb, B.size, out.ctypes.data_as(ctypes.c_void_p), out.size,
                                   ctypes.byref(size))
    if rc != OK:
        raise SlagError(rc, "slag_state_merge_host")
    return out


STATE_HEADER = np.dtype([("magic", "S8"), ("version", "<u4"), ("dim", "<u4"), ("n", "<i8"), ("columns", "<i8"),
                         ("triples", "<i8"), ("fingerprint", "<u8"), ("views", "<i8"), ("pairs", "<i8"),
                         ("contributions", "<i8"), ("evaluations", "<i8"), ("executed", "<i8"),
                         ("weight_mode", "<i4"), ("reserved", "<i4")])


def read_state(state) -> dict:
    """The parts of a saved state as numpy arrays (the format of slag_save_state)."""
    buf = np.frombuffer(state, np.uint8) if isinstance(state, (bytes, bytearray)) else np.asarray(state, np.uint8)
    h = np.frombuffer(buf, STATE_HEADER, 1, 0)[0]
    if h["magic"] != b"SLAGSTAT" or h["version"] != 1:
        raise ValueError("not a state of this library")
    n, D, C, Z = int(h["n"]), int(h["dim"]), int(h["columns"]), int(h["triples"])
    o = STATE_HEADER.itemsize
    table = np.frombuffer(buf, np.float32, C * D, o).reshape(C, D)
    o += 4 * C * D
    sums = np.frombuffer(buf, np.float32, 3 * n, o).reshape(3, n)
    o += 12 * n
    g = np.frombuffer(buf, np.uint32, Z, o)
    c = np.frombuffer(buf, np.uint32, Z, o + 4 * Z)
    w = np.frombuffer(buf, np.float32, Z, o + 8 * Z)
    return {"header": {k: h[k] for k in STATE_HEADER.names}, "table": table, "w_hi": sums[0], "w_lo": sums[1],
            "w_ovf": sums[2], "gauss": g, "column": c, "w": w}


def linear_param_count(dim: int) -> int:
    return int(load_library().slag_linear_param_count(int(dim)))


def linear_code_fit(samples):
    """The linear 32-d code of host samples (n x dim float32): (parameters U then mu, fraction of
    the variance kept)."""
    lib = load_library()
    X = np.ascontiguousarray(samples, np.float32)
    n, dim = X.shape
    params = np.empty(linear_param_count(dim), np.float32)
    kept = ctypes.c_float()
    rc = lib.slag_linear_code_fit(X.ctypes.data_as(ctypes.c_void_p), n, dim, 0, params.ctypes.data_as(ctypes.c_void_p),
                                  ctypes.byref(kept), None)
    if rc != OK:
        raise SlagError(rc, "slag_linear_code_fit")
    return params, float(kept.value)


def latent_param_count(dim: int) -> int:
    return int(load_library().slag_latent_param_count(int(dim)))


def latent_train(samples, epochs: int = 4, batch: int = 1024, lr: float = 1e-3, seed: int = 0):
    """Trains the latent form's autoencoder on host samples (n x dim float32); returns
    (parameters, mean loss per epoch)."""
    lib = load_library()
    X = np.ascontiguousarray(samples, np.float32)
    n, dim = X.shape
    params = np.empty(latent_param_count(dim), np.float32)
    losses = np.empty(int(epochs), np.float32)
    rc = lib.slag_latent_train(X.ctypes.data_as(ctypes.c_void_p), n, dim, int(epochs), int(batch), float(lr),
                               int(seed), 0, params.ctypes.data_as(ctypes.c_void_p),
                               losses.ctypes.data_as(ctypes.c_void_p), None)
    if rc != OK:
        raise SlagError(rc, "slag_latent_train")
    return params, losses


def latent_apply(params, X, mode: int):
    """mode 0: encode (rows x dim -> rows x 32); 1: decode (rows x 32 -> rows x dim); 2: both."""
    lib = load_library()
    p = np.ascontiguousarray(params, np.float32)
    X = np.ascontiguousarray(X, np.float32)
    rows = X.shape[0]
    dim = X.shape[1] if mode != 1 else (p.size - 2 * 32 * 256 - 256 - 32 - 256) // (2 * 256 + 1)
    out = np.empty((rows, 32 if mode == 0 else dim), np.float32)
    rc = lib.slag_latent_apply(p.ctypes.data_as(ctypes.c_void_p), int(dim), X.ctypes.data_as(ctypes.c_void_p), rows,
                               int(mode), out.ctypes.data_as(ctypes.c_void_p), None)
    if rc != OK:
        raise SlagError(rc, "slag_latent_apply")
    return out


def add_views_batched(lifters, view_lists):
    """Adds view_lists[i] (lists of (camera, seg_ids, table) with host numpy or CUDA torch arrays)
    to lifters[i], scene after scene, in one call (slag_add_views_batched)."""
    lib = load_library()
    keep = []
    arrays = []
    counts = (ctypes.c_int32 * len(lifters))()
    for i, (L, views) in enumerate(zip(lifters, view_lists)):
        arr = (CView * max(1, len(views)))()
        for j, (cam, seg, tab) in enumerate(views):
            c = camera_struct(cam)
            sp, sdev, s_keep = _ptr(seg, np.int32)
            tp, tdev, t_keep = _ptr(tab, np.float32)
            keep += [c, s_keep, t_keep]
            arr[j] = CView(ctypes.addressof(c), sp.value, tp.value, int(tab.shape[0]), 1 if sdev else 0)
        counts[i] = len(views)
        arrays.append(arr)
    ctxs = (ctypes.c_void_p * len(lifters))(*[L._h for L in lifters])
    vptrs = (ctypes.c_void_p * len(lifters))(*[ctypes.addressof(a) for a in arrays])
    failed = ctypes.c_int32(-1)
    rc = lib.slag_add_views_batched(len(lifters), ctxs, vptrs, counts, ctypes.byref(failed))
    if rc != OK:
        raise SlagError(rc, "slag_add_views_batched (scene %d)" % failed.value)
