#!/usr/bin/env python
"""Benchmark of the lifting path on one B300 (or N replicas under torchrun).

One step = one whole lifting job on the mid-scale workload: 300,000 Gaussians
on 20 ellipsoid surfaces, 64 views of 960x540 with 64 Voronoi segments each,
512-d float32 segment embeddings from 32 prototypes (seed 1), through
slag_reset -> 64 x slag_add_view -> slag_finalize -> 1,000 top-10 cosine
queries. Inputs are seeded synthetic data of that shape.

Reported:
  value  Gaussian-pixel contributions per second (whole job, device-resident inputs)
  e2e    the same through host buffers: per step the segment maps and tables
         are copied host->device, the embeddings, weight sums and query
         results device->host, all inside the timed region
  roofline  the compositing kernel (the largest share of device time): its
         algorithmic operations over the time at least one composite was
         running, from CUDA events the library records in the streams that
         launch it (views in flight overlap, so summed launch spans would
         count shared time more than once)
  cpu_baseline  the CPU oracle on a bounded sample of the same workload

`--impl reference` times the CPU oracle alone (the reference arm).
Under torchrun each rank runs its own replica of the job (weak scaling).
"""
from __future__ import annotations

import argparse
import json
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
WORKLOAD = "plain FP32 mid scale: 300k Gaussians on 20 ellipsoids, 64 views 960x540, 64 segments, D=512, +1000 top-10 queries"
WORKLOAD_PRECISION = ("precision form at scale (a view subset): 2M Gaussians on 60 ellipsoids, 1920x1080 views, "
                      "128 segments, D=512, +1000 top-10 queries")

# Dense FP32 issue rate used as the compositing kernel's ALU roofline: 148 SMs x 128 FP32 lanes
# x the maximum SM clock, one operation per lane per cycle (most of the work is not FMA).
N_SM = 148
FP32_LANES = 128
# FP32 operations per evaluated (Gaussian, pixel) pair in the compositing loop: offsets (2),
# quadratic form (9), exponent argument check (1), opacity product and cap (2), floor test (1),
# transmittance update, stop test and weight (3), plus the exp itself on the SFU.
OPS_PER_EVAL = 18
# DRAM bytes (read + write) per launch of composite_k from one ncu capture on this workload, valid
# while the kernel source has the recorded SHA-256 (otherwise the roofline reports traffic: null).
COMPOSITE_TRAFFIC = {"bytes_per_launch": 15660544,   # 15.661 MB read + 0.000 MB written
                     "source_sha256": "e53356ef3f9b78baf799fae158c4671a5d1a8432248cd791a078f3977f4ac0b7"}


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="slag", choices=["slag", "reference"])
    p.add_argument("--queries", type=int, default=1000)
    p.add_argument("--k", type=int, default=10)
    p.add_argument("--views", type=int, default=0, help="use only the first V views (0 = all)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-forms", action="store_true", help="skip the BF16 form's line")
    p.add_argument("--workload", default="mid", choices=["mid", "precision", "batched"],
                   help="mid: the headline workload; precision: 2M Gaussians at 1920x1080 on a view subset; "
                        "batched: 16 uneven scenes, their first --views views each (16 by default)")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    return p.parse_args()


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


def _scene(views_limit=0, workload="mid"):
    """The bench's scene: the mid-scale workload (default, every view), or the precision
    configuration on its first `views_limit` views (32 by default)."""
    import synth
    if workload == "precision":
        s = synth.config_precision()
        views_limit = views_limit or 32
    else:
        s = synth.config_mid()
    nv = s.n_views if not views_limit else min(views_limit, s.n_views)
    views = [s.view(i) for i in range(nv)]
    return s, views


def _config(a, scene, views, parallelism, l2):
    v0 = views[0]
    return {"workload": WORKLOAD_PRECISION if a.workload == "precision" else WORKLOAD,
            "gaussians": scene.gaussians.n, "views": len(views),
            "resolution": "%dx%d" % (v0.camera.width, v0.camera.height), "segments": int(v0.table.shape[0]),
            "dim": scene.dim, "queries": a.queries, "k": a.k, "parallelism": parallelism, "l2": l2}


def _queries(views, B, seed=4):
    rng = np.random.default_rng(seed)
    Q = rng.standard_normal((B, views[0].table.shape[1])).astype(np.float32)
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


# ----------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ----------------------------------------------------------------------------

def _cpu_oracle_sample(scene, views, seconds):
    """The oracle as it stands on the host cores, on whole views until `seconds` pass."""
    from oracle import oracle as O
    O.build()
    cores = len(os.sched_getaffinity(0))
    done_views, contrib = 0, 0
    t0 = time.perf_counter()
    i = 0
    while i < len(views) and time.perf_counter() - t0 < seconds:
        batch = views[i:i + cores]
        _, _, info = O.lift(scene.gaussians, batch, threads=cores)
        contrib += sum(c for _, c in info)
        done_views += len(batch)
        i += len(batch)
    dt = time.perf_counter() - t0
    return {"value": contrib / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "views_per_s": done_views / dt,
            "sample": "%d of %d views of the same workload (float64 factored oracle, views spread over %d "
                      "threads, one accumulator per thread); %.1f s" % (done_views, len(views), cores, dt)}


def run_reference(a):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    scene, views = _scene(a.views, a.workload)
    per_step = []
    s = None
    for it in range(a.warmup + a.steps):
        s = _cpu_oracle_sample(scene, views, max(2.0, a.cpu_seconds / 4))
        if it >= a.warmup:
            per_step.append(s)
    value = float(np.mean([x["value"] for x in per_step]))
    vps = float(np.mean([x["views_per_s"] for x in per_step]))
    out = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": a.gpus,
           "steps": a.steps, "warmup": a.warmup, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "views_per_s": vps,
           "config": _config(a, scene, views, "rank 0 on host cores", "n/a (host)"),
           "cpu_baseline": dict(s, value=value),
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------

def run_slag(a):
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2505_08124_b300 import slag as S
    S.load_library()

    scene, views = _scene(a.views, a.workload)
    g = scene.gaussians
    D = scene.dim
    Q = _queries(views, a.queries)
    stream = torch.cuda.current_stream()
    dev = torch.device("cuda", local)

    # device-resident inputs
    d_seg = [torch.from_numpy(v.seg).to(dev) for v in views]
    d_tab = [torch.from_numpy(v.table).to(dev) for v in views]
    d_Q = torch.from_numpy(Q).to(dev)
    d_ids = torch.empty((a.queries, a.k), dtype=torch.int64, device=dev)
    d_sc = torch.empty((a.queries, a.k), dtype=torch.float32, device=dev)
    d_cnt = torch.empty(a.queries, dtype=torch.int32, device=dev)
    d_w = torch.empty(g.n, dtype=torch.float32, device=dev)
    cams = [v.camera for v in views]

    L = S.Lifter(g, dim=D, stream=stream.cuda_stream)

    def step_device():
        L.reset()
        for c, sg, tb in zip(cams, d_seg, d_tab):
            L.add_view(c, sg, tb)
        L.finalize(None, d_w)
        L.query_batch(d_Q, a.k, d_ids, d_sc, d_cnt)

    # host-resident inputs (pinned) for the end-to-end leg
    h_seg = [torch.from_numpy(v.seg).pin_memory().numpy() for v in views]
    h_tab = [torch.from_numpy(v.table).pin_memory().numpy() for v in views]
    h_E = torch.empty((g.n, D), dtype=torch.float32).pin_memory().numpy()
    h_w = torch.empty(g.n, dtype=torch.float32).pin_memory().numpy()
    h_Q = torch.from_numpy(Q).pin_memory().numpy()

    def step_host():
        L.reset()
        for c, sg, tb in zip(cams, h_seg, h_tab):
            L.add_view(c, sg, tb)
        # the download of E and sum w is queued on the library's copy stream and overlaps the
        # next step; every step's copy is complete before the clock stops (wait_outputs)
        L.finalize_async(h_E, h_w)
        ids, sc, cnt = L.query_batch(h_Q, a.k)
        return ids

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()

    def rank_max(x):
        return max_over_ranks(x, dist, dev)

    for _ in range(a.warmup):
        step_device()
    barrier()
    # the timed steps record events around the composite launches only (the roofline's
    # kernel); the other stages' times come from an untimed pass below
    L.set_profiling(True, stages=("composite",))
    L.profile(reset=True)
    st0 = L.stats()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(_device_id(torch, local)) as clk:
        barrier()
        n_launch0 = S.kernel_launches()
        e0.record(stream)
        for _ in range(a.steps):
            step_device()
        e1.record(stream)
        barrier()
        gpu_launches = S.kernel_launches() - n_launch0
    ms = rank_max(e0.elapsed_time(e1))
    prof_timed = L.profile_busy(reset=True)
    L.set_profiling(False)
    stats = L.stats()
    # per-stage breakdown: the same steps, untimed, with every stage's spans recorded
    L.set_profiling(True)
    L.profile(reset=True)
    for _ in range(a.steps):
        step_device()
    prof = L.profile_busy(reset=True)
    L.set_profiling(False)
    contrib_per_step = stats["contributions"]          # reset() clears the counters each step
    evals_per_step = stats["evaluations"]
    views_per_step = len(views)
    value = job_rate(contrib_per_step * a.steps, ws, ms / 1e3)
    views_per_s = job_rate(views_per_step * a.steps, ws, ms / 1e3)

    # end to end through host buffers
    e2e = None
    if not a.no_e2e:
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
        e2e = {"value": job_rate(contrib_per_step * a.steps, ws, dt), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "views_per_s": job_rate(views_per_step * a.steps, ws, dt),
               "ms_per_step": dt * 1e3 / a.steps,
               "outputs": "slag_finalize_async into pinned host buffers: a step's download overlaps the next step"}

    # roofline of the stage with the largest device time
    import json as _j
    peaks = _j.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    dominant = max(prof, key=lambda k: prof[k][2])
    comp_ms, comp_spans, comp_busy = prof_timed["composite"]
    launches = max(1, comp_spans)
    busy_per_launch = comp_busy / launches          # composite-busy time per launch (ms)
    sm_max = peaks.get("sm_max_mhz", 2032.0)
    peak_tops = N_SM * FP32_LANES * sm_max * 1e6 / 1e12
    evals_per_launch = evals_per_step * a.steps / launches
    achieved = evals_per_launch * OPS_PER_EVAL / (busy_per_launch / 1e3) / 1e12
    traffic = None
    if COMPOSITE_TRAFFIC["bytes_per_launch"] is not None:
        import hashlib
        src = open(os.path.join(ROOT, "paper_2505_08124_b300", "csrc", "k_composite.cu"), "rb").read()
        if hashlib.sha256(src).hexdigest() == COMPOSITE_TRAFFIC["source_sha256"]:
            traffic = COMPOSITE_TRAFFIC["bytes_per_launch"]
    roofline = {"kernel": "composite_k", "bound": "alu", "achieved": achieved, "peak": peak_tops,
                "unit": "TOPS (fp32 issue)", "frac": achieved / peak_tops, "traffic": traffic,
                "evaluations_per_launch": evals_per_launch,
                "busy_ms_per_launch": busy_per_launch, "span_ms_per_launch": comp_ms / launches,
                "peak_source": "derived: %d SMs x %d FP32 lanes x %.0f MHz (sm_max_mhz of MEASURED_PEAKS.json)"
                               % (N_SM, FP32_LANES, sm_max),
                "dominant_stage": dominant}

    forms = None
    if not a.no_forms:
        fargs = (L, g, D, cams, d_seg, d_tab, d_Q, a, stream, dev, rank_max, ws)
        forms = {"bf16": dict(_form(S, torch, *fargs, precision=S.PREC_BF16), dtype="bf16 operands, f32 accumulate"),
                 "latent32": _latent_form(S, torch, scene, *fargs)}

    cpu = None
    if rank == 0 and not a.no_cpu:
        cpu = _cpu_oracle_sample(scene, views, a.cpu_seconds)

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": a.steps,
               "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "views_per_s": views_per_s,
               "config": _config(a, scene, views, "replicas x%d" % ws,
                                 "inputs larger than L2 (%d MB of segment maps + %d MB tables per step; %d MB embeddings "
                                 "written per step)" % (sum(v.seg.nbytes for v in views) >> 20,
                                                        sum(v.table.nbytes for v in views) >> 20,
                                                        (g.n * D * 4) >> 20)),
               "clocks": clk.summary(),
               "e2e": e2e,
               "roofline": roofline,
               "cpu_baseline": cpu,
               "gpu_launches": gpu_launches,
               "forms": forms,
               "stages_note": "per-stage CUDA-event spans from an untimed pass of the same steps; the timed "
                              "steps record the composite's spans only",
               "stages_busy_ms_per_step": {k: v[2] / a.steps for k, v in prof.items()},
               "stages_span_ms_per_step": {k: v[0] / a.steps for k, v in prof.items()},
               "stats_per_step": stats}
        print(json.dumps(out), flush=True)
    L.close()
    if dist:
        dist.destroy_process_group()


def _form(S, torch, L, g, D, cams, d_seg, d_tab, d_Q, a, stream, dev, rank_max, ws, precision, latent=None,
          tie_eps=1e-3):
    """A form of the aggregation on the same workload: the same step with another precision;
    its error is stated against the float32 path's embeddings of the same job (1 - cosine per
    Gaussian with sum w >= 1e-3) and its top-10 answers against the float32 path's (strict
    overlap, and tie-tolerant: an id counts when its float32 cosine is within tie_eps of the
    float32 10th best)."""
    n = g.n
    Lb = S.Lifter(g, dim=D, stream=stream.cuda_stream, precision=precision, latent_params=latent)
    ids_b = torch.empty((a.queries, a.k), dtype=torch.int64, device=dev)
    sc_b = torch.empty((a.queries, a.k), dtype=torch.float32, device=dev)
    cnt_b = torch.empty(a.queries, dtype=torch.int32, device=dev)
    w_b = torch.empty(n, dtype=torch.float32, device=dev)

    def step(lift, E_out, w_out, ids, sc, cnt):
        lift.reset()
        for c, sg, tb in zip(cams, d_seg, d_tab):
            lift.add_view(c, sg, tb)
        lift.finalize(E_out, w_out)
        lift.query_batch(d_Q, a.k, ids, sc, cnt)

    for _ in range(max(1, a.warmup)):
        step(Lb, None, w_b, ids_b, sc_b, cnt_b)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        step(Lb, None, w_b, ids_b, sc_b, cnt_b)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = rank_max(e0.elapsed_time(e1))
    contrib = Lb.stats()["contributions"]

    # error against the float32 path on this job
    E_b = torch.empty((n, D), dtype=torch.float32, device=dev)
    E_f = torch.empty((n, D), dtype=torch.float32, device=dev)
    w_f = torch.empty(n, dtype=torch.float32, device=dev)
    ids_f = torch.empty_like(ids_b)
    step(Lb, E_b, w_b, ids_b, sc_b, cnt_b)
    step(L, E_f, w_f, ids_f, torch.empty_like(sc_b), torch.empty_like(cnt_b))
    torch.cuda.synchronize()
    Lb.close()
    ok = w_f >= 1e-3
    Eb, Ef = E_b[ok].double(), E_f[ok].double()
    cos = (Eb * Ef).sum(1) / (Eb.norm(dim=1) * Ef.norm(dim=1))
    En = E_f.double() / E_f.double().norm(dim=1, keepdim=True).clamp_min(1e-300)
    Qd = d_Q.double()
    sb = torch.einsum("qkd,qd->qk", En[ids_b.clamp_min(0)], Qd)
    sf = torch.einsum("qkd,qd->qk", En[ids_f.clamp_min(0)], Qd)
    tie = (sb >= sf.min(dim=1, keepdim=True).values - tie_eps).double().mean().item()
    strict = float(np.mean([len(set(x) & set(y)) / a.k for x, y in zip(ids_b.tolist(), ids_f.tolist())]))
    return {"value": job_rate(contrib * a.steps, ws, ms / 1e3), "unit": UNIT, "ms_per_step": ms / a.steps,
            "views_per_s": job_rate(len(cams) * a.steps, ws, ms / 1e3),
            "cos_err_vs_fp32": {"max": float((1 - cos).max().item()), "mean": float((1 - cos).mean().item()),
                                "gaussians": int(ok.sum().item())},
            "top10_agree_vs_fp32": {"tie_tolerant": tie, "tie_eps": tie_eps, "strict": strict}}


def _latent_form(S, torch, scene, *args):
    """The latent form: the autoencoder trained on segment embeddings drawn like the
    workload's tables (same prototypes and noise law), then the same step aggregating codes."""
    import synth
    D = scene.dim
    m = scene.meta
    # training data drawn by the lifted scene's own generator (its seed, prototypes and noise):
    # 1M samples on the 2M-Gaussian configuration, 262k on the mid scale (a short default run)
    n_train, epochs = (1 << 20) if scene.gaussians.n >= 1_000_000 else (1 << 18), 4
    X = synth.segment_samples(m["seed"], n_train, D, m["n_protos"], noise_sigma=m["noise_sigma"])
    t0 = time.perf_counter()
    params, losses = S.latent_train(X, epochs=epochs, batch=512, lr=2e-3, seed=5)
    train_s = time.perf_counter() - t0
    out = _form(S, torch, *args, precision=S.PREC_LATENT32, latent=params, tie_eps=1e-2)
    out["dtype"] = "32-d codes, bf16 weights, f32 accumulate"
    out["training"] = {"samples": n_train, "epochs": epochs, "seconds": train_s,
                       "loss_first_epoch": float(losses[0]), "loss_last_epoch": float(losses[-1])}
    return out


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
    import concurrent.futures as cf
    import multiprocessing as mp
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

    def timed(fn):
        for _ in range(max(1, a.warmup)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(a.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / a.steps

    ms_seq = timed(sequential)
    ms_bat = timed(batched)
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
