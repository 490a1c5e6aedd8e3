#!/usr/bin/env python
"""Benchmark of the lifting path on one B300 (or N replicas under torchrun).

One step = one whole lifting job, through slag_reset -> one slag_add_view per
view -> slag_finalize -> 1,000 top-10 cosine queries. The default workload is
the precision configuration at full size: 2,000,000 Gaussians on 60
ellipsoid surfaces, 300 views of 1920x1080 on a jittered orbit, 128 Voronoi
segments per view, 512-d segment embeddings from 64 prototypes (seed 2).
Inputs are seeded synthetic data of that shape (the paper's datasets are not
available); every view is generated on the host cores before the first CUDA
call.

Reported (one JSON line):
  value     Gaussian-pixel contributions per second of the float32 path (whole
            job, device-resident inputs); views_per_s beside it
  e2e       the same job through host buffers: per step the segment maps and
            tables are copied host->device, the embeddings, weight sums and
            query results device->host, all inside the timed region
  roofline  the compositing kernel (the largest share of device time), bound
            by its arithmetic: executed (Gaussian, pixel) evaluations x the
            operations of one, over the time at least one composite ran
  roofline_step_hbm  the whole step against the algorithmic bytes and flops
            of the method (per view: Gaussians, segment ids, table, sort
            pairs, records, sparse triples; per step: the output)
  forms     the BF16 form on the same job, and the latent form on the learned
            workload (its embeddings follow the mid-scale law the autoencoder
            is trained on); each with views/s and its error against the float32
            path of the same job
  oracle_error  the float32 path and the BF16 form against the float64 oracle
            on a 10,000-Gaussian subsample of the first 8 views
  cpu_baseline  the oracle's own time on that sample (per view)
  mid       the mid-scale workload (300k Gaussians, 64 views 960x540) as a
            secondary line

`--impl reference` times the CPU oracle alone (the reference arm), on bands
of tile rows of the same views. Under torchrun each rank runs its own replica
of the job (weak scaling).
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import hashlib
import json
import multiprocessing as mp
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gaussian-pixel contribs/s & views/s, D=512: BF16/latent vs FP32 plain at stated cos err"
UNIT = "contribs/s"
WORKLOAD_DESC = {
    "precision": ("precision form at full size: 2,000,000 Gaussians on 60 ellipsoids, 300 views 1920x1080, "
                  "128 Voronoi segments per view, D=512 from 64 prototypes (seed 2), +1000 top-10 queries"),
    "mid": ("plain FP32 mid scale: 300,000 Gaussians on 20 ellipsoids, 64 views 960x540, 64 segments, "
            "D=512 from 32 prototypes (seed 1), +1000 top-10 queries"),
}
LEARNED_DESC = ("learned form: 2,000,000 Gaussians on 60 ellipsoids, 300 views 1920x1080, 128 segments, "
                "embeddings of the mid-scale law (its 32 prototypes), seed 4; autoencoder trained on 1M "
                "samples of that law")

# Compositing kernel's arithmetic roofline: 148 SMs x 128 FP32 lanes x the maximum SM clock. The
# packed FP32 instructions (f32x2) the kernel uses halve its instruction count but not the lane
# rate: independent chains of fma.rn.f32x2 ran at the scalar FFMA's 37-38 T lane-FMA/s on a B300.
N_SM = 148
FP32_LANES = 128
F32X2_LANE_FACTOR = 1
# FP32 and integer/select operations per executed (Gaussian, pixel) evaluation in the compositing
# loop: offsets and quadratic form (5 multiply-adds), floor test (1), opacity cap (1),
# transmittance update and weight (2), stop test (1), selects of T, weight and stop position (3),
# contribution count (2), the two pixels' weight sum (1) and the record bookkeeping (2); plus one
# exp2 on the SFU.
OPS_PER_EVAL = 18
# DRAM bytes (read + write) per launch of composite_k from one ncu capture, valid while the kernel
# source has the recorded SHA-256 (otherwise the roofline reports traffic: null).
COMPOSITE_TRAFFIC = {"bytes_per_launch": 36.27e6,
                     "source_sha256": "e3398ed48afaf888d9606eb7b288e9f7d3f81e2cc31ed0f4efd9739cad3c1d74",
                     "workload": "precision workload, 1920x1080 views 4-6 of the third step of an 8-view run: "
                                 "mean of 3 launches (profiles/composite_k_traffic_precision_1080p.md)"}
# Nominal TF32 : BF16 dense tensor rate (1.1 : 2.25 PFLOP/s); the float32 path's contraction is a
# three-term TF32 split (three MMAs per product).
TF32_OVER_BF16 = 1.1 / 2.25
TF32_TERMS = 3
CPU_VIEWS = 8
CPU_SUBSAMPLE = 10_000


def _args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="slag", choices=["slag", "reference"])
    p.add_argument("--queries", type=int, default=1000)
    p.add_argument("--k", type=int, default=10)
    p.add_argument("--views", type=int, default=0, help="use only the first V views (0 = all)")
    p.add_argument("--workload", default="precision", choices=["precision", "mid", "batched"],
                   help="precision: the headline workload (2M Gaussians, 300 views 1920x1080); mid: 300k "
                        "Gaussians, 64 views 960x540; batched: 16 uneven scenes, their first --views views each")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-forms", action="store_true", help="skip the BF16 and latent forms")
    p.add_argument("--no-mid", action="store_true", help="skip the secondary mid-scale line")
    p.add_argument("--no-cpu", action="store_true", help="skip the oracle (cpu_baseline and oracle_error)")
    p.add_argument("--form-steps", type=int, default=5, help="timed steps of each form (at most --steps)")
    p.add_argument("--stage-steps", type=int, default=3, help="untimed steps of the per-stage breakdown")
    p.add_argument("--cpu-views", type=int, default=CPU_VIEWS)
    p.add_argument("--band-rows", type=int, default=4, help="reference arm: tile rows per view and step")
    return p.parse_args(argv)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, dist=None, device=None):
    """Max of x over the ranks of the default process group (x itself without one)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world_size, seconds):
    """Whole-job throughput: every rank processed units_per_rank in the (max-over-ranks) time."""
    return units_per_rank * world_size / seconds


# ----------------------------------------------------------------------------
# workloads: scenes and their views, generated on the host cores
# ----------------------------------------------------------------------------

def make_scene(key):
    import synth
    if key == "precision":
        return synth.config_precision()
    if key == "mid":
        return synth.config_mid()
    if key == "learned":
        return synth.config_learned()
    if key == "learned_scaled":
        return synth.config_learned(noise_sigma=0.1 / np.sqrt(512))
    raise KeyError(key)


_WORKER_SCENES = {}


def _view_job(job):
    key, i, table_only = job
    if key not in _WORKER_SCENES:
        _WORKER_SCENES[key] = make_scene(key)
    v = _WORKER_SCENES[key].view(i)
    return key, i, v.camera, (None if table_only else v.seg), v.table


def generate_views(jobs):
    """{(key, i): (camera, seg or None, table)} for jobs (key, view index, table only), on a
    spawned process pool (started before any CUDA call)."""
    if not jobs:
        return {}
    workers = max(1, min(32, len(os.sched_getaffinity(0)), len(jobs)))
    if workers == 1:
        got = [_view_job(j) for j in jobs]
    else:
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            got = list(ex.map(_view_job, jobs, chunksize=max(1, len(jobs) // (4 * workers))))
    return {(k, i): (cam, seg, tab) for k, i, cam, seg, tab in got}


def _config(a, scene, cams, parallelism, l2):
    c0 = cams[0]
    return {"workload": WORKLOAD_DESC[a.workload], "gaussians": scene.gaussians.n, "views": len(cams),
            "resolution": "%dx%d" % (c0.width, c0.height), "segments": int(scene.meta["n_segments"]),
            "dim": scene.dim, "queries": a.queries, "k": a.k, "parallelism": parallelism, "l2": l2}


def _queries(dim, B, seed=4):
    rng = np.random.default_rng(seed)
    Q = rng.standard_normal((B, dim)).astype(np.float32)
    Q /= np.linalg.norm(Q, axis=1, keepdims=True)
    return Q


# ----------------------------------------------------------------------------
# clocks
# ----------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id: str):
        self.device_id = device_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.device_id, "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def _device_id(torch, local):
    try:
        u = str(torch.cuda.get_device_properties(local).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(local)


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return json.load(open(path)), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0, "sm_max_mhz": 2032.0}, \
        "fallback"


# ----------------------------------------------------------------------------
# roofline arithmetic
# ----------------------------------------------------------------------------

def algorithmic_work(n, dim, cams, segments_per_view, pairs, triples):
    """The method's bytes and flops for one whole job: per view 44 B per Gaussian in, 4 B per
    pixel of segment ids, the M x D table, 24 B per Gaussian-tile pair (sort pairs written and
    read once), 40 B per Gaussian of records (written and read once), 12 B per sparse
    (Gaussian, view-segment, W) triple; per job the n x (D + 1) float32 output. Flops: 2 D per
    triple (the contraction of the weights with the segment embeddings)."""
    V = len(cams)
    hw = sum(int(c.width) * int(c.height) for c in cams)
    b = (V * (44 + 40) * n + 4 * hw + 4 * segments_per_view * dim * V + 24 * pairs + 12 * triples
         + 4 * n * (dim + 1))
    f = 2 * dim * triples
    return float(b), float(f)


def step_roofline(bytes_alg, flops_alg, ms_per_step, peaks, source):
    bw = peaks["hbm_gbs"] * 1e9
    tf = peaks["bf16_tflops"] * 1e12 * TF32_OVER_BF16 / TF32_TERMS
    t_b, t_f = bytes_alg / bw, flops_alg / tf
    t = ms_per_step / 1e3
    bound = "hbm" if t_b >= t_f else "tensor"
    return {"bound": bound, "achieved": bytes_alg / t / 1e9 if bound == "hbm" else flops_alg / t / 1e12,
            "peak": peaks["hbm_gbs"] if bound == "hbm" else tf / 1e12,
            "unit": "GB/s" if bound == "hbm" else "TFLOP/s", "frac": max(t_b, t_f) / t, "traffic": None,
            "bytes_alg_per_step": bytes_alg, "flops_alg_per_step": flops_alg,
            "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs; float32 contraction at bf16_tflops x %.3f / %d)"
                           % (source, TF32_OVER_BF16, TF32_TERMS)}


def composite_roofline(executed_per_launch, busy_ms_per_launch, span_ms_per_launch, peaks, source,
                       f32x2=F32X2_LANE_FACTOR, dominant=None, evaluations_per_launch=None):
    sm_max = peaks.get("sm_max_mhz", 2032.0)
    peak = N_SM * FP32_LANES * f32x2 * sm_max * 1e6 / 1e12
    achieved = executed_per_launch * OPS_PER_EVAL / (busy_ms_per_launch / 1e3) / 1e12
    traffic = None
    if COMPOSITE_TRAFFIC["bytes_per_launch"] is not None:
        src = open(os.path.join(ROOT, "paper_2505_08124_b300", "csrc", "k_composite.cu"), "rb").read()
        if hashlib.sha256(src).hexdigest() == COMPOSITE_TRAFFIC["source_sha256"]:
            traffic = COMPOSITE_TRAFFIC["bytes_per_launch"]
    return {"kernel": "composite_k", "bound": "alu", "achieved": achieved, "peak": peak,
            "unit": "T ops/s (fp32 lanes)", "frac": achieved / peak, "traffic": traffic,
            "executed_evaluations_per_launch": executed_per_launch,
            "visited_evaluations_per_launch": evaluations_per_launch,
            "ops_per_evaluation": OPS_PER_EVAL,
            "busy_ms_per_launch": busy_ms_per_launch, "span_ms_per_launch": span_ms_per_launch,
            "peak_source": "derived: %d SMs x %d FP32 lanes x %.0f MHz (sm_max_mhz, %s); packed f32x2 runs at "
                           "the same lane rate (x%d)" % (N_SM, FP32_LANES, sm_max, source, f32x2),
            "dominant_stage": dominant}


# ----------------------------------------------------------------------------
# CPU oracle (baseline, error and reference arm)
# ----------------------------------------------------------------------------

def _cores():
    return len(os.sched_getaffinity(0))


def oracle_subsample(scene, views, sub):
    """The oracle on whole views for the Gaussians `sub` (every Gaussian still takes part in the
    compositing), views spread over the host cores; returns (E, den, seconds, info)."""
    from oracle import oracle as O
    O.build()
    threads = max(1, min(len(views), _cores()))
    t0 = time.perf_counter()
    num, den, info = O.lift(scene.gaussians, views, sub_ids=sub, threads=threads)
    dt = time.perf_counter() - t0
    return O.normalise(num, den), den, dt, info, threads


def run_reference(a):
    """The reference arm: the float64 oracle as it stands, on the host cores. Each step is a
    bounded sample of the workload: a band of a.band_rows tile rows of each of `cores` views
    (whole rows of the view: each of their pixels gets the whole view's result), accumulated
    for the seeded 10,000-Gaussian subsample of the cpu_baseline leg (every Gaussian is still
    composited; the accumulators of all n Gaussians would take ~10 GB per thread)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    scene = make_scene(a.workload)
    nv = scene.n_views if not a.views else min(a.views, scene.n_views)
    cores = _cores()
    per_step = min(cores, nv)
    views = {}
    tiles_y = None
    samples = []
    sub = np.sort(np.random.default_rng(7).choice(scene.gaussians.n, min(CPU_SUBSAMPLE, scene.gaussians.n),
                                                  replace=False))
    for it in range(a.warmup + a.steps):
        idx = [(it * per_step + j) % nv for j in range(per_step)]
        for i in idx:
            if i not in views:
                views[i] = scene.view(i)
        tiles_y = (views[idx[0]].camera.height + 15) // 16
        rows = min(a.band_rows, tiles_y)
        ty0 = (it * 7) % max(1, tiles_y - rows + 1)
        t0 = time.perf_counter()
        _, _, info = O.lift(scene.gaussians, [views[i] for i in idx], sub_ids=sub, threads=per_step,
                            tile_rows=(ty0, ty0 + rows))
        dt = time.perf_counter() - t0
        if it >= a.warmup:
            samples.append((sum(c for _, c in info), dt, ty0, rows))
    contrib = sum(s[0] for s in samples)
    secs = sum(s[1] for s in samples)
    value = contrib / secs
    rows = samples[0][3]
    cam = views[0].camera if 0 in views else next(iter(views.values())).camera
    cfg = _config(a, scene, [cam] * nv, "rank 0 on host cores", "n/a (host)")
    sample = ("per step, %d views of the %d (threads: one view each), tile rows [r, r + %d) of each (r moves from "
              "step to step; %d tile rows per view), accumulated for a seeded %d-Gaussian subsample (all "
              "Gaussians composited), float64 factored oracle; %d steps, %.1f s"
              % (per_step, nv, rows, tiles_y, len(sub), a.steps, secs))
    out = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": a.gpus,
           "steps": a.steps, "warmup": a.warmup, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": per_step, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------

class Job:
    """One scene's inputs on the device (and pinned on the host for the end-to-end leg)."""

    def __init__(self, torch, dev, scene, views, queries, k, pinned=False):
        self.scene = scene
        self.cams = [v[0] for v in views]
        self.d_seg = [torch.from_numpy(v[1]).to(dev) for v in views]
        self.d_tab = [torch.from_numpy(v[2]).to(dev) for v in views]
        self.Q = _queries(scene.dim, queries)
        self.d_Q = torch.from_numpy(self.Q).to(dev)
        self.k = k
        n = scene.gaussians.n
        self.d_ids = torch.empty((queries, k), dtype=torch.int64, device=dev)
        self.d_sc = torch.empty((queries, k), dtype=torch.float32, device=dev)
        self.d_cnt = torch.empty(queries, dtype=torch.int32, device=dev)
        self.d_w = torch.empty(n, dtype=torch.float32, device=dev)
        self.views = views if pinned else None

    def run(self, L, E_out=None, w_out=None, ids=None):
        L.reset()
        for c, sg, tb in zip(self.cams, self.d_seg, self.d_tab):
            L.add_view(c, sg, tb)
        L.finalize(E_out, self.d_w if w_out is None else w_out)
        L.query_batch(self.d_Q, self.k, self.d_ids if ids is None else ids, self.d_sc, self.d_cnt)


def _timed(torch, stream, fn, steps, warmup, barrier=None):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    if barrier:
        barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    if barrier:
        barrier()
    return e0.elapsed_time(e1)


def _compare(torch, E_a, E_f, w_f, ids_a, ids_f, Q, k, tie_eps):
    """Error of E_a against E_f (1 - cos per Gaussian with sum w >= 1e-3, in row chunks) and the
    agreement of the two top-k lists (strict overlap; tie-tolerant: an id of ids_a counts when
    its E_f cosine is within tie_eps of E_f's k-th best)."""
    n = E_f.shape[0]
    ok = w_f >= 1e-3
    mx, tot, cnt = 0.0, 0.0, 0
    for r0 in range(0, n, 1 << 18):
        sl = slice(r0, min(n, r0 + (1 << 18)))
        m = ok[sl]
        a, b = E_a[sl][m].double(), E_f[sl][m].double()
        if a.shape[0] == 0:
            continue
        c = 1.0 - (a * b).sum(1) / (a.norm(dim=1) * b.norm(dim=1)).clamp_min(1e-300)
        mx = max(mx, float(c.max().item()))
        tot += float(c.sum().item())
        cnt += int(c.shape[0])
    Qd = Q.double()

    def scores(ids):
        rows = E_f[ids.clamp_min(0).reshape(-1)].double().reshape(ids.shape[0], ids.shape[1], -1)
        rows = rows / rows.norm(dim=2, keepdim=True).clamp_min(1e-300)
        return torch.einsum("qkd,qd->qk", rows, Qd)

    sa, sf = scores(ids_a), scores(ids_f)
    tie = float((sa >= sf.min(dim=1, keepdim=True).values - tie_eps).double().mean().item())
    strict = float(np.mean([len(set(x) & set(y)) / k for x, y in zip(ids_a.tolist(), ids_f.tolist())]))
    return {"cos_err_vs_fp32": {"max": mx, "mean": tot / max(1, cnt), "gaussians": cnt},
            "top10_agree_vs_fp32": {"tie_tolerant": tie, "tie_eps": tie_eps, "strict": strict}}


def run_form(S, torch, dev, stream, job, L_f32, precision, steps, warmup, ws, rank_max, latent=None,
             tie_eps=1e-3, time_plain=False, linear=None):
    """A form on `job`: views/s over `steps` timed steps, and its error against the float32 path
    of the same job."""
    n, D = job.scene.gaussians.n, job.scene.dim
    out = {}
    Lb = S.Lifter(job.scene.gaussians, dim=D, stream=stream.cuda_stream, precision=precision, latent_params=latent,
                  linear_code=linear)
    ms = rank_max(_timed(torch, stream, lambda: job.run(Lb), steps, warmup))
    contrib = Lb.stats()["contributions"]
    out.update(value=job_rate(contrib * steps, ws, ms / 1e3), unit=UNIT, ms_per_step=ms / steps,
               views_per_s=job_rate(len(job.cams) * steps, ws, ms / 1e3))
    if time_plain:
        msp = rank_max(_timed(torch, stream, lambda: job.run(L_f32), steps, warmup))
        out["fp32_same_workload"] = {"ms_per_step": msp / steps,
                                     "views_per_s": job_rate(len(job.cams) * steps, ws, msp / 1e3)}
    E_b = torch.empty((n, D), dtype=torch.float32, device=dev)
    ids_b = torch.empty((job.Q.shape[0], job.k), dtype=torch.int64, device=dev)
    job.run(Lb, E_b, None, ids_b)
    torch.cuda.synchronize()
    Lb.close()
    E_f = torch.empty((n, D), dtype=torch.float32, device=dev)
    w_f = torch.empty(n, dtype=torch.float32, device=dev)
    ids_f = torch.empty_like(ids_b)
    job.run(L_f32, E_f, w_f, ids_f)
    torch.cuda.synchronize()
    out.update(_compare(torch, E_b, E_f, w_f, ids_b, ids_f, job.d_Q, job.k, tie_eps))
    del E_b, E_f
    return out


def run_slag(a):
    ws, rank, local = _dist()
    key = a.workload
    scene = make_scene(key)
    nv = scene.n_views if not a.views else min(a.views, scene.n_views)
    # every view generated on the host cores before the first CUDA call
    jobs = [(key, i, False) for i in range(nv)]
    want_forms = not a.no_forms and key == "precision"
    want_mid = not a.no_mid and key == "precision"
    if want_forms:
        jobs += [("learned", i, False) for i in range(nv)] + [("learned_scaled", i, True) for i in range(nv)]
    if want_mid:
        jobs += [("mid", i, False) for i in range(64)]
    t_gen = time.perf_counter()
    got = generate_views(jobs)
    t_gen = time.perf_counter() - t_gen
    views = [got[(key, i)] for i in range(nv)]

    import torch
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2505_08124_b300 import slag as S
    S.load_library()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    g = scene.gaussians
    D = scene.dim
    peaks, peak_source = _peaks()

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()

    def rank_max(x):
        return max_over_ranks(x, dist, dev)

    job = Job(torch, dev, scene, views, a.queries, a.k)
    L = S.Lifter(g, dim=D, stream=stream.cuda_stream)

    # ---- the headline: float32 path, device-resident inputs ---------------------------
    for _ in range(a.warmup):
        job.run(L)
    barrier()
    # timed steps without stage timing: the views sized on the device replay captured graphs
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(_device_id(torch, local)) as clk:
        barrier()
        n_launch0 = S.kernel_launches()
        e0.record(stream)
        for _ in range(a.steps):
            job.run(L)
        e1.record(stream)
        barrier()
        gpu_launches = S.kernel_launches() - n_launch0
    ms = rank_max(e0.elapsed_time(e1))
    stats = L.stats()                       # one step's counters (reset() clears them every step)
    # the compositing kernel's busy time: untimed steps with events around the composites only
    c_steps = max(1, min(2, a.steps))
    L.set_profiling(True, stages=("composite",))
    L.profile(reset=True)
    for _ in range(c_steps):
        job.run(L)
    prof_timed = L.profile_busy(reset=True)
    L.set_profiling(False)
    # per-stage breakdown: a few more steps, untimed, with every stage's spans recorded
    L.set_profiling(True)
    L.profile(reset=True)
    st_steps = max(1, min(a.stage_steps, a.steps))
    for _ in range(st_steps):
        job.run(L)
    prof = L.profile_busy(reset=True)
    L.set_profiling(False)
    contrib_per_step = stats["contributions"]
    value = job_rate(contrib_per_step * a.steps, ws, ms / 1e3)
    views_per_s = job_rate(nv * a.steps, ws, ms / 1e3)

    # ---- end to end through host buffers --------------------------------------------------
    e2e = None
    if not a.no_e2e:
        h_seg = [torch.from_numpy(v[1]).pin_memory().numpy() for v in views]
        h_tab = [torch.from_numpy(v[2]).pin_memory().numpy() for v in views]
        h_E = torch.empty((g.n, D), dtype=torch.float32).pin_memory().numpy()
        h_w = torch.empty(g.n, dtype=torch.float32).pin_memory().numpy()
        h_Q = torch.from_numpy(job.Q).pin_memory().numpy()

        def step_host():
            L.reset()
            for c, sg, tb in zip(job.cams, h_seg, h_tab):
                L.add_view(c, sg, tb)
            # the download of E and sum w is queued on the library's copy stream and overlaps the
            # next step; every step's copy is complete before the clock stops (wait_outputs)
            L.finalize_async(h_E, h_w)
            L.query_batch(h_Q, a.k)

        step_host()
        L.wait_outputs()
        barrier()
        t0 = time.perf_counter()
        for _ in range(a.steps):
            step_host()
        L.wait_outputs()
        barrier()
        dt = rank_max(time.perf_counter() - t0)
        h2d = sum(x.nbytes for x in h_seg) + sum(x.nbytes for x in h_tab) + h_Q.nbytes
        d2h = h_E.nbytes + h_w.nbytes + a.queries * a.k * (8 + 4) + a.queries * 4
        e2e = {"value": job_rate(contrib_per_step * a.steps, ws, dt), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "views_per_s": job_rate(nv * a.steps, ws, dt), "ms_per_step": dt * 1e3 / a.steps,
               "outputs": "slag_finalize_async into pinned host buffers: a step's download overlaps the next step"}
        del h_seg, h_tab, h_E

    # ---- rooflines -------------------------------------------------------------------------
    dominant = max(prof, key=lambda s: prof[s][2])
    comp_ms, comp_spans, comp_busy = prof_timed["composite"]
    launches = max(1, comp_spans)
    roofline = composite_roofline(stats["executed"] * c_steps / launches, comp_busy / launches,
                                  comp_ms / launches, peaks, peak_source, dominant=dominant,
                                  evaluations_per_launch=stats["evaluations"] * c_steps / launches)
    b_alg, f_alg = algorithmic_work(g.n, D, job.cams, int(scene.meta["n_segments"]), stats["pairs"],
                                    stats["triples"])
    roof_step = step_roofline(b_alg, f_alg, ms / a.steps, peaks, peak_source)

    # ---- forms -------------------------------------------------------------------------------
    forms = None
    fsteps = max(1, min(a.form_steps, a.steps))
    fwarm = max(1, min(a.warmup, 3))
    if want_forms:
        forms = {"bf16": dict(run_form(S, torch, dev, stream, job, L, S.PREC_BF16, fsteps, fwarm, ws, rank_max),
                              dtype="bf16 operands, f32 accumulate", workload=WORKLOAD_DESC[key])}
        forms["latent32"] = latent_forms(S, torch, dev, stream, got, nv, a, fsteps, fwarm, ws, rank_max)

    # ---- the oracle: float64 error on a subsample, and its own time ------------------------
    cpu, oracle_err = None, None
    if rank == 0 and not a.no_cpu:
        cpu, oracle_err = oracle_leg(S, torch, dev, stream, scene, views, a)

    # ---- the mid-scale workload as a secondary line ----------------------------------------
    mid = None
    if want_mid:
        ms_scene = make_scene("mid")
        mviews = [got[("mid", i)] for i in range(ms_scene.n_views)]
        mjob = Job(torch, dev, ms_scene, mviews, a.queries, a.k)
        Lm = S.Lifter(ms_scene.gaussians, dim=ms_scene.dim, stream=stream.cuda_stream)
        mms = rank_max(_timed(torch, stream, lambda: mjob.run(Lm), a.steps, a.warmup, barrier))
        mst = Lm.stats()
        Lm.close()
        mid = {"workload": WORKLOAD_DESC["mid"], "value": job_rate(mst["contributions"] * a.steps, ws, mms / 1e3),
               "unit": UNIT, "ms_per_step": mms / a.steps,
               "views_per_s": job_rate(len(mviews) * a.steps, ws, mms / 1e3), "stats_per_step": mst}
        del mjob

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": a.steps,
               "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "views_per_s": views_per_s,
               "config": _config(a, scene, job.cams, "replicas x%d" % ws,
                                 "inputs larger than L2 (%d MB of segment maps + %d MB tables per step; %d MB "
                                 "embeddings written per step)" % (sum(v[1].nbytes for v in views) >> 20,
                                                                   sum(v[2].nbytes for v in views) >> 20,
                                                                   (g.n * D * 4) >> 20)),
               "clocks": clk.summary(),
               "e2e": e2e,
               "roofline": roofline,
               "roofline_step_hbm": roof_step,
               "cpu_baseline": cpu,
               "oracle_error": oracle_err,
               "gpu_launches": gpu_launches,
               "forms": forms,
               "mid": mid,
               "host_view_generation_s": t_gen,
               "stages_note": "per-stage CUDA-event spans from %d untimed steps after the timed ones (stage "
                              "timing launches kernel by kernel; the timed steps replay graphs and record "
                              "nothing; the compositing roofline's busy time comes from %d more untimed steps "
                              "that record the composite's spans only)" % (st_steps, c_steps),
               "stages_busy_ms_per_step": {s: v[2] / st_steps for s, v in prof.items()},
               "stages_span_ms_per_step": {s: v[0] / st_steps for s, v in prof.items()},
               "stats_per_step": stats}
        print(json.dumps(out), flush=True)
    L.close()
    if dist:
        dist.destroy_process_group()


def latent_forms(S, torch, dev, stream, got, nv, a, steps, warmup, ws, rank_max):
    """The latent form on the learned workload, under both readings of the embeddings' noise
    N(0, 0.1): per coordinate (literal) and with norm 0.1 (sigma = 0.1 / sqrt(D)). The
    autoencoder is trained on 1M samples of the mid-scale law (its 32 prototypes); views/s of the
    latent form and of the float32 path on the same job, errors against the float32 path."""
    import synth
    out = {"workload": LEARNED_DESC}
    lscene = make_scene("learned")
    D = lscene.dim
    lviews = [got[("learned", i)] for i in range(nv)]
    mid_seed, mid_protos = 1, 32           # the mid-scale workload's embedding law
    for reading, sigma in (("literal", 0.1), ("scaled", 0.1 / np.sqrt(D))):
        if reading == "scaled":
            lviews = [(c, s, got[("learned_scaled", i)][2]) for i, (c, s, _) in enumerate(lviews)]
        job = Job(torch, dev, lscene, lviews, a.queries, a.k)
        X = synth.segment_samples(mid_seed, 1 << 20, D, mid_protos, noise_sigma=sigma)
        t0 = time.perf_counter()
        params, losses = S.latent_train(X, epochs=4, batch=512, lr=2e-3, seed=5)
        train_s = time.perf_counter() - t0
        Lf = S.Lifter(lscene.gaussians, dim=D, stream=stream.cuda_stream)
        r = run_form(S, torch, dev, stream, job, Lf, S.PREC_LATENT32, steps, warmup, ws, rank_max, latent=params,
                     tie_eps=1e-2, time_plain=(reading == "literal"))
        Lf.close()
        r["noise_sigma"] = float(sigma)
        r["training"] = {"samples": 1 << 20, "epochs": 4, "seconds": train_s,
                         "loss_first_epoch": float(losses[0]), "loss_last_epoch": float(losses[-1])}
        # the linear 32-d code (principal directions of the same samples): exact aggregation of
        # codes, so its error is the part of E_k outside the code's subspace
        t0 = time.perf_counter()
        lin, kept = S.linear_code_fit(X)
        fit_s = time.perf_counter() - t0
        Lf = S.Lifter(lscene.gaussians, dim=D, stream=stream.cuda_stream)
        rl = run_form(S, torch, dev, stream, job, Lf, S.PREC_LINEAR32, steps, warmup, ws, rank_max, linear=lin,
                      tie_eps=1e-2)
        Lf.close()
        rl["fit"] = {"samples": 1 << 20, "seconds": fit_s, "variance_kept": kept}
        r["linear_code"] = rl
        out[reading] = r
        del job, X
    out["dtype"] = "32-d codes, bf16 weights, f32 accumulate (linear code: TF32-rounded basis, f32 accumulate)"
    return out


def oracle_leg(S, torch, dev, stream, scene, views, a):
    """cpu_baseline (the float64 oracle's time on the first a.cpu_views views, reported per view)
    and oracle_error (the float32 path and the BF16 form against it), on a seeded
    10,000-Gaussian subsample: the oracle accumulates only those Gaussians, every Gaussian
    still takes part in the compositing."""
    import synth
    nv = min(a.cpu_views, len(views))
    vs = [synth.View(c, s, t) for c, s, t in views[:nv]]
    g = scene.gaussians
    sub = np.sort(np.random.default_rng(7).choice(g.n, min(CPU_SUBSAMPLE, g.n), replace=False))
    sub_t = torch.from_numpy(sub).to(dev)
    got = {}
    for name, prec in (("fp32", S.PREC_FP32), ("bf16", S.PREC_BF16)):
        with S.Lifter(g, dim=scene.dim, stream=stream.cuda_stream, precision=prec) as L:
            for v in vs:
                L.add_view(v.camera, v.seg, v.table)
            E = torch.empty((g.n, scene.dim), dtype=torch.float32, device=dev)
            w = torch.empty(g.n, dtype=torch.float32, device=dev)
            L.finalize(E, w)
            torch.cuda.synchronize()
            got[name] = (E[sub_t].cpu().numpy().astype(np.float64), w[sub_t].cpu().numpy().astype(np.float64))
            del E, w
    Eo, den, secs, info, threads = oracle_subsample(scene, vs, sub)
    contrib = sum(c for _, c in info)
    cpu = {"value": contrib / secs, "unit": UNIT, "cores": threads, "kind": "oracle",
           "views_per_s": nv / secs, "s_per_view": secs / nv,
           "sample": "the first %d views of the same workload, whole views, accumulated for a seeded %d-Gaussian "
                     "subsample (tiles that touch none of it are skipped); float64 factored oracle, one view per "
                     "thread on %d threads; %.1f s" % (nv, len(sub), threads, secs)}
    ok = den >= 1e-3
    err = {"views": nv, "subsample": int(len(sub)), "touched": int(ok.sum())}
    for name, (E, w) in got.items():
        rel = float(np.linalg.norm(E - Eo) / np.linalg.norm(Eo))
        relw = float(np.linalg.norm(w - den) / np.linalg.norm(den))
        x, y = E[ok], Eo[ok]
        cos = (x * y).sum(1) / (np.linalg.norm(x, axis=1) * np.linalg.norm(y, axis=1))
        err[name] = {"rel_l2": rel, "wsum_rel_l2": relw, "max_1_minus_cos": float((1 - cos).max()),
                     "mean_1_minus_cos": float((1 - cos).mean())}
    return cpu, err


# ----------------------------------------------------------------------------
# batched workload (secondary)
# ----------------------------------------------------------------------------

def _batched_view(job):
    """(scene index, view index) -> (camera, segment map, table) of the batched workload."""
    import synth
    i, j = job
    v = synth.config_batched()[i].view(j)
    return i, j, v.camera, v.seg, v.table


def run_batched(a):
    """16 independent uneven scenes (config_batched, seed 3), their first `views` views each:
    every scene lifted on its own in turn (its views, then its finalize), against all scenes in
    one slag_add_views_batched call and then every finalize; both with device-resident inputs, no
    queries."""
    import synth
    scenes = synth.config_batched()
    cap = a.views or 16
    jobs = [(i, j) for i, s in enumerate(scenes) for j in range(min(cap, s.n_views))]
    # views generated on the host cores before any CUDA call
    with cf.ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 1), mp_context=mp.get_context("spawn")) as ex:
        got = list(ex.map(_batched_view, jobs, chunksize=4))
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2505_08124_b300 import slag as S
    S.load_library()
    stream = torch.cuda.current_stream()
    views = [[] for _ in scenes]
    for i, j, cam, seg, tab in sorted(got, key=lambda t: (t[0], t[1])):
        views[i].append((cam, torch.from_numpy(seg).to(dev), torch.from_numpy(tab).to(dev)))
    lifters = [S.Lifter(s.gaussians, dim=s.dim, stream=stream.cuda_stream) for s in scenes]
    wbuf = [torch.empty(s.gaussians.n, dtype=torch.float32, device=dev) for s in scenes]

    def sequential():
        for L, vs, w in zip(lifters, views, wbuf):
            L.reset()
            for cam, seg, tab in vs:
                L.add_view(cam, seg, tab)
            L.finalize(None, w)

    def batched():
        for L in lifters:
            L.reset()
        S.add_views_batched(lifters, views)
        for L, w in zip(lifters, wbuf):
            L.finalize(None, w)

    ms_seq = _timed(torch, stream, sequential, a.steps, max(1, a.warmup)) / a.steps
    ms_bat = _timed(torch, stream, batched, a.steps, max(1, a.warmup)) / a.steps
    contrib = sum(L.stats()["contributions"] for L in lifters)
    nviews = sum(len(v) for v in views)
    for L in lifters:
        L.close()
    if rank == 0:
        out = {"metric": METRIC, "value": contrib / (ms_bat / 1e3), "unit": UNIT, "n_gpus": ws, "steps": a.steps,
               "warmup": a.warmup, "ms_per_step": ms_bat, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "views_per_s": nviews / (ms_bat / 1e3),
               "sequential": {"ms_per_step": ms_seq, "views_per_s": nviews / (ms_seq / 1e3),
                              "value": contrib / (ms_seq / 1e3)},
               "config": {"workload": "batched form: 16 independent scenes (log-uniform 50k-1.5M Gaussians, "
                                      "640x480 / 960x540 / 1920x1080, 32-128 segments, D=512), the first %d views "
                                      "of each (of 20-200)" % cap,
                          "scenes": len(scenes), "views": nviews,
                          "gaussians": [s.gaussians.n for s in scenes],
                          "parallelism": "replicas x%d" % ws}}
        print(json.dumps(out), flush=True)


def main():
    a = _args()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "batched":
        run_batched(a)
    else:
        run_slag(a)


if __name__ == "__main__":
    main()
