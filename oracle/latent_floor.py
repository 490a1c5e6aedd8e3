"""Error floor of a 32-d linear code for the latent form (test infrastructure: oracle and seeded
inputs only).

The latent form aggregates 32-d codes of the segment embeddings and decodes each Gaussian's mean
code. With a linear code -- encode z = U^T (e - mu), decode mu + U z, U the top-32 principal
directions of the training embeddings -- aggregation in code space is exact (the mean of the codes
is the code of the mean), so the decoded embedding is the projection mu + U U^T (E_k - mu) of the
exact E_k of the Aggregation step, and its error is what lies outside that affine subspace. This
script computes that error with the float64 oracle's E_k, for both readings of the embeddings'
noise N(0, 0.1): per coordinate, and with norm 0.1 (sigma = 0.1 / sqrt(D)). The scene is a reduced
version of the learned workload (same law: the mid-scale workload's 32 prototypes, 128 Voronoi
segments per view, a jittered orbit), accumulated for a seeded subsample of Gaussians.

    python -m oracle.latent_floor [--gaussians N] [--views V] [--width W] [--height H]
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pca(X, k):
    mu = X.mean(axis=0)
    C = (X - mu).T @ (X - mu) / X.shape[0]
    w, V = np.linalg.eigh(C)
    return mu, V[:, ::-1][:, :k], w[::-1]


def cos_rows(a, b):
    return (a * b).sum(1) / np.maximum(np.linalg.norm(a, axis=1) * np.linalg.norm(b, axis=1), 1e-300)


def topk_agreement(E_code, E, Q, k, eps):
    """Tie-tolerant agreement (an id of the code's top-k counts when its exact cosine is within
    eps of the exact k-th best) and strict overlap, over the rows of E."""
    En = E / np.linalg.norm(E, axis=1, keepdims=True)
    Cn = E_code / np.linalg.norm(E_code, axis=1, keepdims=True)
    S, Sc = Q @ En.T, Q @ Cn.T
    tie, strict = [], []
    for q in range(Q.shape[0]):
        exact = np.argsort(-S[q], kind="stable")[:k]
        code = np.argsort(-Sc[q], kind="stable")[:k]
        kth = S[q, exact[-1]]
        tie.append(np.mean(S[q, code] >= kth - eps))
        strict.append(len(set(exact) & set(code)) / k)
    return float(np.mean(tie)), float(np.mean(strict))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gaussians", type=int, default=200_000)
    ap.add_argument("--views", type=int, default=300)
    ap.add_argument("--width", type=int, default=480)
    ap.add_argument("--height", type=int, default=270)
    ap.add_argument("--subsample", type=int, default=4000)
    ap.add_argument("--train", type=int, default=200_000)
    ap.add_argument("--queries", type=int, default=1000)
    ap.add_argument("--threads", type=int, default=len(os.sched_getaffinity(0)))
    a = ap.parse_args(argv)
    import synth
    from oracle import oracle as O
    D, code = 512, 32
    g = synth.ellipsoid_gaussians(4, a.gaussians, 60)
    sub = np.sort(np.random.default_rng(7).choice(g.n, a.subsample, replace=False))
    rng = np.random.default_rng(11)
    Q = rng.standard_normal((a.queries, D))
    Q /= np.linalg.norm(Q, axis=1, keepdims=True)
    out = {"scene": {"gaussians": g.n, "views": a.views, "resolution": "%dx%d" % (a.width, a.height),
                     "segments": 128, "subsample": int(len(sub)), "law": "32 prototypes of seed 1"},
           "readings": {}}
    for reading, sigma in (("literal", 0.1), ("scaled", 0.1 / np.sqrt(D))):
        s = synth.make_scene("floor", 4, g, n_views=a.views, width=a.width, height=a.height, n_segments=128,
                             n_protos=32, dim=D, jitter=True, noise_sigma=sigma, proto_seed=1)
        num, den, _ = O.lift(g, s.views(), sub_ids=sub, threads=a.threads)
        ok = den >= 1e-3
        E = num[ok] / den[ok, None]
        X = synth.segment_samples(1, a.train, D, 32, noise_sigma=sigma).astype(np.float64)
        mu, U, ev = pca(X, code)
        P = mu + (E - mu) @ U @ U.T
        err = 1.0 - cos_rows(P, E)
        # the best any 32-d linear code could do on these embeddings: their own top-32 subspace
        mu_e, U_e, _ = pca(E, code)
        P_e = mu_e + (E - mu_e) @ U_e @ U_e.T
        err_e = 1.0 - cos_rows(P_e, E)
        tie, strict = topk_agreement(P, E, Q, 10, 1e-2)
        tie3, _ = topk_agreement(P, E, Q, 10, 1e-3)
        out["readings"][reading] = {
            "noise_sigma": float(sigma), "gaussians": int(ok.sum()),
            "pca_code": {"mean_1_minus_cos": float(err.mean()), "median": float(np.median(err)),
                         "max": float(err.max()), "p99": float(np.quantile(err, 0.99)),
                         "top10_tie_tolerant_eps1e-2": tie, "top10_tie_tolerant_eps1e-3": tie3,
                         "top10_strict": strict,
                         "training_variance_kept": float(ev[:code].sum() / ev.sum())},
            "best_linear_code_on_E": {"mean_1_minus_cos": float(err_e.mean()), "max": float(err_e.max())},
            "mean_norm_E": float(np.linalg.norm(E, axis=1).mean()),
        }
        print(reading, json.dumps(out["readings"][reading]), flush=True)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
