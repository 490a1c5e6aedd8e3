"""The BF16 form of the aggregation (precision SLAG_PREC_BF16).

The per-view weights are composited in float32 exactly as in the plain path;
only the contraction of the weights with the segment embeddings runs with
bfloat16 operands (float32 accumulation) on the tensor cores. The error is
stated against the float64 oracle: per touched Gaussian (sum w >= 1e-3) the
cosine to the oracle's E_k is at least 1 - 1e-3, the weight sums keep the
float32 bar, and top-10 cosine queries agree with the plain float32 path on
at least 99% of the returned ids, an id counting when its float32 score is
within 1e-3 (the bfloat16 score error) of the float32 10th score: neighbouring
Gaussians carry near-identical embeddings, so exact ranks among near-ties are
not a property of either path. The strict overlap is reported beside it."""
import numpy as np
import pytest

import synth
from oracle import oracle as O

pytestmark = pytest.mark.gpu

COS_ERR = 1e-3     # 1 - cosine to the float64 result, per touched Gaussian
W_FLOOR = 1e-3
TOP10_AGREE = 0.99
TIE_EPS = 1e-3


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


def _lift(S, scene, views, precision):
    L = S.Lifter(scene.gaussians, dim=scene.dim, precision=precision)
    for v in views:
        L.add_view(v.camera, v.seg, v.table)
    E, w = L.finalize()
    return L, E, w


@pytest.mark.parametrize("which", ["tiny", "small"])
def test_bf16_error_against_float64(slag, which):
    if which == "tiny":
        s = synth.config_tiny()            # D = 512: 128-dimension passes, 64-column chunks
    else:
        s = synth.small_scene(31, 6000, 3, 200, 120, 9, dim=256, surfaces=5, empty_fraction=0.2)
    views = list(s.views())
    L, E, w = _lift(slag, s, views, slag.PREC_BF16)
    L.close()
    num, den, _ = O.lift(s.gaussians, views, threads=4)
    Eo = O.normalise(num, den)
    relw = np.linalg.norm(w.astype(np.float64) - den) / np.linalg.norm(den)
    assert relw <= 1e-4, relw                        # sum w is the float32 path's
    ok = den >= W_FLOOR
    a, b = E[ok].astype(np.float64), Eo[ok]
    cos = (a * b).sum(1) / (np.linalg.norm(a, axis=1) * np.linalg.norm(b, axis=1))
    rel = np.linalg.norm(E.astype(np.float64) - Eo) / np.linalg.norm(Eo)
    print("bf16 %s: max 1-cos %.3e, mean 1-cos %.3e, rel L2 %.3e over %d Gaussians"
          % (which, (1 - cos).max(), (1 - cos).mean(), rel, ok.sum()))
    assert (1.0 - cos).max() <= COS_ERR
    assert rel <= 1e-2


def test_bf16_top10_agrees_with_plain(slag):
    s = synth.small_scene(32, 8000, 4, 200, 120, 9, dim=256, surfaces=5)
    views = list(s.views())
    Lb, _, _ = _lift(slag, s, views, slag.PREC_BF16)
    Lf, Ef, _ = _lift(slag, s, views, slag.PREC_FP32)
    rng = np.random.default_rng(5)
    Q = rng.standard_normal((200, s.dim)).astype(np.float32)
    Q /= np.linalg.norm(Q, axis=1, keepdims=True)
    ib, _, _ = Lb.query_batch(Q, 10)
    if_, _, _ = Lf.query_batch(Q, 10)
    Lb.close()
    Lf.close()
    strict = np.mean([len(set(x.tolist()) & set(y.tolist())) / 10.0 for x, y in zip(ib, if_)])
    # float32 cosine of every returned id
    E64 = Ef.astype(np.float64)
    En = E64 / np.maximum(np.linalg.norm(E64, axis=1, keepdims=True), 1e-300)
    tol = []
    for q, xb, xf in zip(Q.astype(np.float64), ib, if_):
        tenth = (En[xf] @ q).min()
        tol.append(np.mean(En[xb] @ q >= tenth - TIE_EPS))
    tol = float(np.mean(tol))
    print("bf16 top-10 agreement with the float32 path: tie-tolerant %.4f, strict %.4f" % (tol, strict))
    assert tol >= TOP10_AGREE
    assert strict >= 0.98
