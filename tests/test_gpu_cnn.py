"""GPU: the proposal network's own kernels against the FP64 reference; training; top-k; gathered scoring."""
import math

import numpy as np
import pytest

import oracle
from oracle import cnn as ocnn
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1609_06634_gb300 as bioem
    from paper_1609_06634_gb300 import build
    build.build()
    return bioem, bioem.Context(0)


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def _fp16_exact(rng, n, scale):
    return (rng.standard_normal(n) * scale).astype(np.float16).astype(np.float64)


def test_gradients_match_reference(env):
    bioem, ctx = env
    rng = np.random.default_rng(11)
    px, down, C, nq, nd, B = 32, 2, 8, 12, 4, 6
    net = bioem.CNN(ctx, image_px=px, downsample=down, channels=C, n_qbins=nq, n_dbins=nd, max_batch=8, seed=5)
    _, _, F, n = ocnn.layout(px // down, C, nq, nd)
    assert net.n_params == n
    theta = _fp16_exact(rng, n, 0.3)
    imgs = rng.standard_normal((B, px, px)).astype(np.float32)
    yq = rng.integers(0, nq, B).astype(np.int32)
    yd = rng.integers(0, nd, B).astype(np.int32)
    net.set_params(_dev(theta.astype(np.float32)))
    g, loss = net.gradients(_dev(imgs), _dev(yq), _dev(yd))
    lq, ld = net.forward(_dev(imgs))
    want_loss, want_g = ocnn.loss_and_grad(theta, imgs.astype(np.float64), yq, yd, down, C, nq, nd)
    wq, wd, _ = ocnn.forward(theta, imgs.astype(np.float64), down, C, nq, nd)
    np.testing.assert_allclose(lq.cpu().numpy(), wq, rtol=0, atol=1e-3 * np.abs(wq).max())
    np.testing.assert_allclose(ld.cpu().numpy(), wd, rtol=0, atol=1e-3 * np.abs(wd).max())
    np.testing.assert_allclose(loss.cpu().numpy(), want_loss, rtol=2e-4)
    got = g.cpu().numpy().astype(np.float64)
    offs, heads, _, _ = ocnn.layout(px // down, C, nq, nd)
    tensors = [o for pair in offs for o in pair] + list(heads)
    for off, shape in tensors:
        sl = slice(off, off + int(np.prod(shape)))
        err = np.linalg.norm(got[sl] - want_g[sl]) / max(np.linalg.norm(want_g[sl]), 1e-12)
        assert err < 2e-3, (off, shape, err)


def test_training_reduces_loss(env):
    """Labels determined by the image content (a shifted blob per class): loss must fall."""
    import torch
    bioem, ctx = env
    rng = np.random.default_rng(12)
    px, nq, nd, B = 32, 6, 2, 64
    net = bioem.CNN(ctx, image_px=px, downsample=2, channels=16, n_qbins=nq, n_dbins=nd, max_batch=B, seed=9)
    yy, xx = np.mgrid[0:px, 0:px]

    def batch():
        yq = rng.integers(0, nq, B)
        yd = rng.integers(0, nd, B)
        cx = 6 + 4 * yq
        imgs = np.exp(-((xx[None] - cx[:, None, None]) ** 2 + (yy[None] - 16) ** 2) / (2 * (2 + 3 * yd[:, None, None]) ** 2))
        imgs = imgs + 0.3 * rng.standard_normal((B, px, px))
        return _dev(imgs.astype(np.float32)), _dev(yq.astype(np.int32)), _dev(yd.astype(np.int32))

    first = None
    for step in range(300):
        x, yq, yd = batch()
        loss = net.train_step(x, yq, yd, 2e-3)
        if step < 10:
            first = loss.mean().item() if first is None else first + loss.mean().item()
    first /= 10
    last = np.mean([net.train_step(*batch(), 2e-3).mean().item() for _ in range(10)])
    assert last < 0.3 * first, (first, last)
    del torch


def test_propose_topk_matches_reference(env):
    bioem, ctx = env
    rng = np.random.default_rng(13)
    px, C, nq, nd, k = 32, 8, 40, 4, 7
    net = bioem.CNN(ctx, image_px=px, downsample=2, channels=C, n_qbins=nq, n_dbins=nd, max_batch=4, seed=3)
    _, _, _, n = ocnn.layout(16, C, nq, nd)
    theta = _fp16_exact(rng, n, 0.5)
    net.set_params(_dev(theta.astype(np.float32)))
    imgs = rng.standard_normal((10, px, px)).astype(np.float32)      # 10 images: 3 batches of <= 4
    bins, scores = net.propose(_dev(imgs), k)
    bins, scores = bins.cpu().numpy(), scores.cpu().numpy()
    lq, ld, _ = ocnn.forward(theta, imgs.astype(np.float64), 2, C, nq, nd)
    joint = (ocnn.log_softmax(lq)[:, :, None] + ocnn.log_softmax(ld)[:, None, :]).reshape(10, -1)
    for i in range(10):
        order = np.argsort(-joint[i], kind="stable")
        gaps = -np.diff(joint[i][order[:k + 1]])
        if np.all(gaps > 1e-3):
            assert list(bins[i]) == list(order[:k])
        np.testing.assert_allclose(scores[i], joint[i][bins[i]], atol=2e-3)
        assert np.all(np.diff(scores[i]) <= 0)


def test_gathered_scoring_matches_oracle(env):
    import torch
    bioem, ctx = env
    cfg = workloads.get_config("tiny", n_orient=40)
    wl = workloads.workload(cfg, n_img=5)
    imgs = oracle.synthesize_images(wl)
    ref = oracle.score(imgs, wl["atoms"], wl["quats"], wl["ctfs"], cfg.sigma_A, cfg.pixel_A, cfg.max_shift)
    n_ps = len(wl["quats"]) * len(wl["ctfs"])
    rng = np.random.default_rng(14)
    lists = [np.sort(rng.choice(n_ps, size=int(rng.integers(1, 120)), replace=False)) for _ in range(5)]
    im = bioem.prepare_images(ctx, _dev(imgs), cfg.pixel_A)
    ps = bioem.project_model(ctx, _dev(wl["atoms"]), cfg.sigma_A, _dev(wl["quats"]), wl["ctfs"], cfg.npix, cfg.pixel_A)
    S = cfg.n_shift

    def csr(ls):
        off = np.concatenate([[0], np.cumsum([len(x) for x in ls])]).astype(np.int32)
        return _dev(off), _dev(np.concatenate(ls).astype(np.int32)), max(len(x) for x in ls)

    acc = torch.empty((5, 2), dtype=torch.float64, device="cuda:0")
    o, p, mx = csr(lists)
    bioem.score_gathered(ctx, im, ps, cfg.max_shift, o, p, mx, acc, True)
    # the same work split over two calls folds to the same posterior
    acc2 = torch.empty((5, 2), dtype=torch.float64, device="cuda:0")
    halves = [[x[: len(x) // 2] for x in lists], [x[len(x) // 2:] for x in lists]]
    for h, part in enumerate(halves):
        o2, p2, mx2 = csr([x if len(x) else np.zeros(0, np.int64) for x in part])
        bioem.score_gathered(ctx, im, ps, cfg.max_shift, o2, p2, max(mx2, 1), acc2, h == 0)
    lp = bioem.acc_logP(ctx, acc, 0.0).cpu().numpy()
    lp2 = bioem.acc_logP(ctx, acc2, 0.0).cpu().numpy()
    assert ctx.status() == 0
    for w in range(5):
        want = oracle.logsumexp(ref["pair_lse"][w, lists[w]])
        assert abs(lp[w] - want) < 1e-3, (w, lp[w], want)
        assert abs(lp2[w] - lp[w]) < 1e-9
    norm = bioem.acc_logP(ctx, acc, math.log(120 * S)).cpu().numpy()
    np.testing.assert_allclose(norm, lp - math.log(120 * S), atol=1e-9)
