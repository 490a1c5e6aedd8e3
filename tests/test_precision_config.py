"""The precision configuration at scale: 2,000,000 Gaussians on 60 ellipsoids,
1920x1080 views, 128 segments per view, D = 512 (64 prototypes, seed 2).

The CUDA path lifts the first 8 views of the orbit; the float64 oracle
accumulates the same views for a seeded subsample of 10,000 Gaussians (every
Gaussian still takes part in the compositing). The float32 path must meet the
float32 parity bar on the subsample; the BF16 form (bfloat16 contraction on
the tensor cores, float32 accumulation) is held to 1 - cosine <= 1e-3 per
touched Gaussian, and both errors are printed."""
import os

import numpy as np
import pytest

import synth
from oracle import oracle as O

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N_VIEWS = 8
N_SUB = 10_000


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


def test_precision_config_on_a_subsample(slag):
    import torch
    s = synth.config_precision()
    views = [s.view(i) for i in range(N_VIEWS)]
    sub = np.sort(np.random.default_rng(7).choice(s.gaussians.n, N_SUB, replace=False))
    sub_t = torch.from_numpy(sub).cuda()
    got = {}
    for prec in (slag.PREC_FP32, slag.PREC_BF16):
        with slag.Lifter(s.gaussians, dim=s.dim, precision=prec) as L:
            for v in views:
                L.add_view(v.camera, v.seg, v.table)
            E = torch.empty((s.gaussians.n, s.dim), dtype=torch.float32, device="cuda")
            w = torch.empty(s.gaussians.n, dtype=torch.float32, device="cuda")
            L.finalize(E, w)
            torch.cuda.synchronize()
            got[prec] = (E[sub_t].cpu().numpy(), w[sub_t].cpu().numpy())
            del E, w
    num, den, _ = O.lift(s.gaussians, views, sub_ids=sub, threads=max(1, min(N_VIEWS, os.cpu_count() or 1)))
    Eo = O.normalise(num, den)
    ok = den >= 1e-3
    assert ok.sum() > 300   # about 6% of the sample is touched by 8 views of the orbit

    def errors(E, w):
        rel = np.linalg.norm(E.astype(np.float64) - Eo) / np.linalg.norm(Eo)
        relw = np.linalg.norm(w.astype(np.float64) - den) / np.linalg.norm(den)
        a, b = E[ok].astype(np.float64), Eo[ok]
        cos = (a * b).sum(1) / (np.linalg.norm(a, axis=1) * np.linalg.norm(b, axis=1))
        return rel, relw, float((1.0 - cos).max())

    r32, w32, c32 = errors(*got[slag.PREC_FP32])
    rbf, wbf, cbf = errors(*got[slag.PREC_BF16])
    print("precision config, %d views, %d of %d sampled Gaussians touched: "
          "fp32 rel L2 %.2e, sum w rel L2 %.2e, max 1-cos %.2e; "
          "bf16 rel L2 %.2e, max 1-cos %.2e" % (N_VIEWS, ok.sum(), N_SUB, r32, w32, c32, rbf, cbf))
    assert r32 <= 1e-4 and w32 <= 1e-4
    assert c32 <= 1e-5
    assert wbf <= 1e-4
    assert cbf <= 1e-3
