"""The learned latent form (SLAG_PREC_LATENT32).

Checks, from the autoencoder's kernels to the lifted embeddings:
  * the encoder and decoder against a float64 PyTorch evaluation of the same
    network (erf-GELU; weights rounded to bfloat16, as the kernels take them);
  * the training kernels' gradient: the first Adam step moves every clearly
    non-zero parameter gradient's parameter by -lr sign(g), with g from
    float64 autograd on the same batch;
  * training lowers the loss and reconstructs held-out embeddings;
  * lifting in the latent space against the plain float32 path, reported as
    1 - cosine per touched Gaussian; a stated measurement, not a pinned value,
    at two noise levels of the segment embeddings: the literal N(0, 0.1) per
    coordinate of the configurations (noise norm ~0.1 sqrt(D), far above the
    unit prototype: a 32-d code cannot carry it) and sigma = 0.1 / sqrt(D)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

H, L = 256, 32


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


def _unpack(p, D, torch, bf16=True, grad=False):
    sizes = [("W1", D * H, (D, H)), ("b1", H, (H,)), ("W2", H * L, (H, L)), ("b2", L, (L,)),
             ("W3", L * H, (L, H)), ("b3", H, (H,)), ("W4", H * D, (H, D)), ("b4", D, (D,))]
    out, at = {}, 0
    for name, n, shape in sizes:
        t = torch.tensor(p[at:at + n].astype(np.float64).reshape(shape), requires_grad=grad)
        out[name] = t
        at += n
    assert at == p.size
    return out


def _ref_forward(P, X, torch, mode):
    F = torch.nn.functional

    def w(t):   # the kernels take the weights rounded to bfloat16 (straight-through for gradients)
        return t + (t.to(torch.bfloat16).to(torch.float64) - t).detach() if t.dim() == 2 else t

    z = X
    if mode in (0, 2):
        z = F.gelu(z @ w(P["W1"]) + P["b1"]) @ w(P["W2"]) + P["b2"]
        if mode == 0:
            return z
    return F.gelu(z @ w(P["W3"]) + P["b3"]) @ w(P["W4"]) + P["b4"]


def test_autoencoder_forward_matches_float64(slag):
    import torch
    D = 256
    rng = np.random.default_rng(3)
    p = (rng.standard_normal(slag.latent_param_count(D)) * 0.05).astype(np.float32)
    X = rng.standard_normal((300, D)).astype(np.float32)
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    P = _unpack(p, D, torch)
    Xt = torch.tensor(X.astype(np.float64))
    for mode in (0, 2):
        ref = _ref_forward(P, Xt, torch, mode).numpy()
        got = slag.latent_apply(p, X, mode)
        np.testing.assert_allclose(got, ref, rtol=0, atol=2e-5 * np.abs(ref).max())
    Z = _ref_forward(P, Xt, torch, 0).numpy().astype(np.float32)
    ref = _ref_forward(P, torch.tensor(Z.astype(np.float64)), torch, 1).numpy()
    np.testing.assert_allclose(slag.latent_apply(p, Z, 1), ref, rtol=0, atol=2e-5 * np.abs(ref).max())


@pytest.mark.parametrize("D,rows", [(512, 50000), (384, 20000)])
def test_decoder_many_tiles_matches_float64(slag, D, rows):
    # the decoder's dense layers are persistent: with more 128-row tiles than SMs each CTA takes
    # several, alternating its two TMEM accumulators (D = 384: 128-column tiles, else 256)
    import torch
    rng = np.random.default_rng(7)
    p = (rng.standard_normal(slag.latent_param_count(D)) * 0.05).astype(np.float32)
    Z = rng.standard_normal((rows, L)).astype(np.float32)
    P = _unpack(p, D, torch)
    ref = _ref_forward(P, torch.tensor(Z.astype(np.float64)), torch, 1).numpy()
    got = slag.latent_apply(p, Z, 1)
    assert got.shape == (rows, D)
    np.testing.assert_allclose(got, ref, rtol=0, atol=2e-5 * np.abs(ref).max())


def test_first_adam_step_follows_the_gradient(slag):
    import torch
    D, n = 128, 512
    X = synth.segment_samples(5, n, D, 8, noise_sigma=0.1 / np.sqrt(D))
    p0, _ = slag.latent_train(X, epochs=1, batch=n, lr=1e-30, seed=11)     # the initial parameters
    p1, _ = slag.latent_train(X, epochs=1, batch=n, lr=1e-3, seed=11)      # one full-batch Adam step
    P = _unpack(p0, D, torch, grad=True)
    Xt = torch.tensor(X.astype(np.float64))
    Y = _ref_forward(P, Xt, torch, 2)
    loss = (((Y - Xt) ** 2).mean(1) + (1 - torch.nn.functional.cosine_similarity(Y, Xt, dim=1))).mean()
    loss.backward()
    g = np.concatenate([P[k].grad.numpy().ravel() for k in ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4")])
    step = (p1.astype(np.float64) - p0.astype(np.float64)) / 1e-3
    big = np.abs(g) > 1e-3 * np.abs(g).max()
    agree = np.mean(np.sign(step[big]) == -np.sign(g[big]))
    assert big.sum() > 1000
    assert agree >= 0.99, agree
    # and the step has Adam's first-step size, lr per parameter
    assert np.median(np.abs(step[big])) == pytest.approx(1.0, rel=0.05)


def test_training_reconstructs_held_out_embeddings(slag):
    D = 256
    X = synth.segment_samples(6, 16384, D, 8, noise_sigma=0.1 / np.sqrt(D), sample_seed=0)
    Xv = synth.segment_samples(6, 1024, D, 8, noise_sigma=0.1 / np.sqrt(D), sample_seed=1)
    p, losses = slag.latent_train(X, epochs=8, batch=512, lr=2e-3, seed=2)
    assert losses[-1] < 0.5 * losses[0]
    R = slag.latent_apply(p, Xv, 2)
    cos = (R * Xv).sum(1) / (np.linalg.norm(R, axis=1) * np.linalg.norm(Xv, axis=1))
    print("latent round trip, held-out: loss %.4f -> %.4f, mean cos %.5f, min cos %.5f"
          % (losses[0], losses[-1], cos.mean(), cos.min()))
    assert cos.mean() >= 0.99


@pytest.mark.parametrize("sigma_kind", ["literal", "scaled"])
def test_latent_lifting_against_plain(slag, sigma_kind):
    D, protos = 256, 8
    sigma = 0.1 if sigma_kind == "literal" else 0.1 / np.sqrt(D)
    s = synth.small_scene(44, 6000, 3, 200, 120, 9, dim=D, surfaces=5, n_protos=protos, noise_sigma=sigma)
    views = list(s.views())
    X = synth.segment_samples(44, 32768, D, protos, noise_sigma=sigma)
    p, losses = slag.latent_train(X, epochs=8, batch=512, lr=2e-3, seed=3)
    with slag.Lifter(s.gaussians, dim=D) as Lf:
        for v in views:
            Lf.add_view(v.camera, v.seg, v.table)
        Ef, wf = Lf.finalize()
    with slag.Lifter(s.gaussians, dim=D, precision=slag.PREC_LATENT32, latent_params=p) as Ll:
        for v in views:
            Ll.add_view(v.camera, v.seg, v.table)
        El, wl = Ll.finalize()
        Q = Ef[wf > 1e-3][:200]
        Q = Q / np.linalg.norm(Q, axis=1, keepdims=True)
        il, _, _ = Ll.query_batch(Q.astype(np.float32), 10)
    with slag.Lifter(s.gaussians, dim=D) as Lf2:
        for v in views:
            Lf2.add_view(v.camera, v.seg, v.table)
        Lf2.finalize()
        if_, _, _ = Lf2.query_batch(Q.astype(np.float32), 10)
    np.testing.assert_allclose(wl, wf, rtol=1e-6)                 # sum w is the plain path's
    ok = wf >= 1e-3
    a, b = El[ok].astype(np.float64), Ef[ok].astype(np.float64)
    cos = (a * b).sum(1) / (np.linalg.norm(a, axis=1) * np.linalg.norm(b, axis=1))
    agree = np.mean([len(set(x.tolist()) & set(y.tolist())) / 10.0 for x, y in zip(il, if_)])
    # tie-tolerant: a latent answer counts when its float32 cosine is within 1e-2 (the latent
    # form's error scale) of the float32 10th best
    En = Ef.astype(np.float64) / np.maximum(np.linalg.norm(Ef.astype(np.float64), axis=1, keepdims=True), 1e-300)
    Qd = Q.astype(np.float64)
    tie = np.mean([np.mean(En[xl] @ q >= (En[xf] @ q).min() - 1e-2) for q, xl, xf in zip(Qd, il, if_)])
    print("latent lifting (%s noise, sigma %.4f): 1-cos mean %.3e, max %.3e over %d Gaussians; "
          "top-10 agreement with the float32 path: strict %.3f, tie-tolerant %.3f; training loss %.4f -> %.4f"
          % (sigma_kind, sigma, (1 - cos).mean(), (1 - cos).max(), ok.sum(), agree, tie, losses[0], losses[-1]))
    assert not (El[~(wf > 0)]).any()                             # untouched Gaussians stay 0
    # stated measurements with regression bounds: the isotropic noise outside the 32-d code
    # cannot be reconstructed (1 - cos ~ sigma^2 D (1 - 32 / D) / 2 per segment embedding)
    assert (1 - cos).mean() < (0.5 if sigma_kind == "literal" else 1e-2)


# ----------------------------------------------------------------------------
# the linear 32-d code (SLAG_PREC_LINEAR32)
# ----------------------------------------------------------------------------

def test_linear_code_fit_is_the_principal_subspace(slag):
    # samples drawn from 20 prototype directions plus small noise: the fitted U must span the
    # same 32-d principal subspace as numpy's eigendecomposition of the sample covariance
    D = 256
    X = synth.segment_samples(31, 20000, D, 20, noise_sigma=0.02 / np.sqrt(D))
    params, kept = slag.linear_code_fit(X)
    U, mu = params[:D * L].reshape(D, L).astype(np.float64), params[D * L:].astype(np.float64)
    Xd = X.astype(np.float64)
    np.testing.assert_allclose(mu, Xd.mean(0), atol=1e-6)
    C = np.cov(Xd.T, bias=True)
    w, V = np.linalg.eigh(C)
    V = V[:, ::-1][:, :L]
    np.testing.assert_allclose(U.T @ U, np.eye(L), atol=1e-4)
    # projectors onto the leading 19 directions (the prototype part; the rest is noise whose
    # directions are not unique) agree, and the 32-d projector captures the same variance
    P_ref = V[:, :19] @ V[:, :19].T
    assert np.linalg.norm(U @ U.T @ P_ref - P_ref) < 1e-3
    assert abs(kept - w[::-1][:L].sum() / w.sum()) < 1e-4


def test_linear_code_lifting_is_the_projection_of_the_aggregate(slag):
    # aggregation of linear codes is exact: the decoded embedding of every touched Gaussian is
    # mu + U U^T (E_k - mu) of the float32 path's E_k (to float32 rounding)
    D = 256
    s = synth.small_scene(41, 6000, 4, 160, 120, 12, dim=D, surfaces=4, n_protos=20,
                          noise_sigma=0.1 / np.sqrt(D))
    views = [s.view(i) for i in range(s.n_views)]
    X = synth.segment_samples(41, 50000, D, 20, noise_sigma=0.1 / np.sqrt(D))
    params, _ = slag.linear_code_fit(X)
    U, mu = params[:D * L].reshape(D, L).astype(np.float64), params[D * L:].astype(np.float64)
    with slag.Lifter(s.gaussians, dim=D) as Lf:
        for v in views:
            Lf.add_view(v.camera, v.seg, v.table)
        Ef, wf = Lf.finalize()
    with slag.Lifter(s.gaussians, dim=D, precision=slag.PREC_LINEAR32, linear_code=params) as Ll:
        for v in views:
            Ll.add_view(v.camera, v.seg, v.table)
        El, wl = Ll.finalize()
        ids = Ll.query_threshold(views[0].table[0] / np.linalg.norm(views[0].table[0]), 0.28)
    # the weight sums are the float32 path's (float32 atomics add in a run-dependent order)
    np.testing.assert_allclose(wl, wf, rtol=1e-5, atol=1e-7)
    ok = wf >= 1e-3
    assert ok.sum() > 500
    E = Ef[ok].astype(np.float64)
    proj = mu + (E - mu) @ U @ U.T
    # the decoder multiplies the codes (exact hi/lo TF32 planes) by U rounded to TF32 (relative
    # error <= 2^-11 per element): rows agree to that rounding
    rel = np.linalg.norm(El[ok] - proj, axis=1) / np.linalg.norm(proj, axis=1)
    assert rel.max() <= 5e-4, rel.max()
    assert np.all(El[wl == 0] == 0)
    cos = (El[ok] * E).sum(1) / (np.linalg.norm(El[ok], axis=1) * np.linalg.norm(E, axis=1))
    print("linear code vs float32 path: mean 1 - cos %.2e, max %.2e" % ((1 - cos).mean(), (1 - cos).max()))
    assert len(ids) > 0
