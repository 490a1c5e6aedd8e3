"""Out-of-core aggregation and the spatial partition export.

With SLAG_FLAG_EMBEDDINGS_ON_HOST the context keeps no n x D embeddings on the
device: finalize computes the rows in chunks of spatially adjacent Gaussians
and places them in host memory. slag_export_partitions writes the touched
Gaussians to per-area files of a grid over the means. Both must give the rows
of the resident-embedding path."""
import os

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
    return synth.small_scene(41, 7000, 3, 160, 120, 9, dim=256, surfaces=5, empty_fraction=0.1)


def _lift(S, s, **kw):
    L = S.Lifter(s.gaussians, dim=s.dim, **kw)
    for v in s.views():
        L.add_view(v.camera, v.seg, v.table)
    return L


def test_host_resident_finalize_matches(slag, scene):
    with _lift(slag, scene) as L:
        E, w = L.finalize()
    with _lift(slag, scene, embeddings_on_host=True) as H:
        Eh, wh = H.finalize()
        with pytest.raises(slag.SlagError) as e:
            H.query(np.ones(scene.dim, np.float32) / np.sqrt(scene.dim), 5)
        assert e.value.status == slag.ERR_STATE
    np.testing.assert_allclose(wh, w, rtol=1e-6, atol=0)
    np.testing.assert_allclose(Eh, E, rtol=1e-5, atol=1e-7)


@pytest.mark.parametrize("cells", [(1, 1), (3, 2)])
def test_export_partitions(slag, scene, tmp_path, cells):
    with _lift(slag, scene) as L:
        E, w = L.finalize()
        n_written = L.export_partitions(str(tmp_path), cells[0], cells[1], chunk_gaussians=512)
    parts = slag.read_partitions(str(tmp_path))
    touched = np.flatnonzero(w > 0)
    ids = np.concatenate([p["ids"] for p in parts.values()])
    assert n_written == len(ids) == len(touched)
    np.testing.assert_array_equal(np.sort(ids), touched)          # each touched Gaussian once
    means = scene.gaussians.means
    x0, x1 = means[:, 0].min(), means[:, 0].max()
    y0, y1 = means[:, 1].min(), means[:, 1].max()
    for (cx, cy), p in parts.items():
        assert 0 <= cx < cells[0] and 0 <= cy < cells[1]
        bx0, bx1, by0, by1 = p["bounds"]
        m = means[p["ids"]]
        eps = 1e-4 * max(x1 - x0, y1 - y0)
        assert (m[:, 0] >= bx0 - eps).all() and (m[:, 0] <= bx1 + eps).all()
        assert (m[:, 1] >= by0 - eps).all() and (m[:, 1] <= by1 + eps).all()
        np.testing.assert_allclose(p["E"], E[p["ids"]], rtol=1e-5, atol=1e-7)
        np.testing.assert_allclose(p["wsum"], w[p["ids"]], rtol=1e-6, atol=0)


def test_out_of_core_under_a_device_budget_matches_the_oracle(slag):
    # the mid-scale Gaussians (300k, D = 512: 614 MB of embeddings) with a 24 MB device budget for
    # output rows: the finalize runs ~25 chunks; the rows of a seeded 10k subsample against the
    # float64 oracle (every Gaussian still takes part in the compositing)
    s = synth.config_mid()
    views = [s.view(i) for i in range(4)]
    with slag.Lifter(s.gaussians, dim=s.dim, embeddings_on_host=True) as H:
        H.set_device_budget(24 << 20)
        for v in views:
            H.add_view(v.camera, v.seg, v.table)
        E, w = H.finalize()
    sub = np.sort(np.random.default_rng(3).choice(s.gaussians.n, 10_000, replace=False))
    num, den, _ = O.lift(s.gaussians, views, sub_ids=sub, threads=max(1, min(4, os.cpu_count() or 1)))
    Eo = O.normalise(num, den)
    Es, ws = E[sub].astype(np.float64), w[sub].astype(np.float64)
    ok = den >= 1e-3
    assert ok.sum() > 300
    assert np.linalg.norm(Es - Eo) / np.linalg.norm(Eo) <= 1e-4
    assert np.linalg.norm(ws - den) / np.linalg.norm(den) <= 1e-4
    cos = (Es[ok] * Eo[ok]).sum(1) / (np.linalg.norm(Es[ok], axis=1) * np.linalg.norm(Eo[ok], axis=1))
    assert cos.min() >= 0.99999
    assert np.all(E[w == 0] == 0)
