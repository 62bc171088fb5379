"""GPU: the learned proposal end to end at a small scale, against the full grid and random proposals.

Trains the network (own kernels) on forward-model projections, proposes the top-k joint (coarse
Hopf cell, defocus) bins of fresh images, scores each image only on its proposed fine parameter
sets, and compares with the full fine grid (the judge) and with random proposals of the same size:
the gain of the learned part is the posterior mass it keeps beyond what random cells keep.
"""
import math

import numpy as np
import pytest

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


def test_proposal_end_to_end(env):
    """Scaled down so that a short training run learns: one model, 72 coarse cells (Hopf level 0) of
    8 fine orientations each, 64 px images, SNR 1.  The full-scale workload is measured by bench.py."""
    import torch
    bioem, ctx = env
    from paper_1609_06634_gb300 import proposal
    cfg = workloads.ProposalConfig(n_models=1, atoms_range=(3000, 3000), npix=64, pixel_A=2.2, max_shift=8,
                                   coarse_level=0, fine_level=1, top_k=8, n_train=12288, n_infer=40, channels=16,
                                   snr=1.0)
    dev = torch.device("cuda", 0)
    gen = torch.Generator(device=dev).manual_seed(1)
    atoms = [torch.from_numpy(a).to(dev) for a in workloads.proposal_models(cfg)]
    tr = workloads.proposal_draws(cfg, cfg.n_train, 8)
    imgs = proposal.compose(ctx, atoms, tr, cfg, gen)
    net = bioem.CNN(ctx, image_px=cfg.npix, downsample=cfg.downsample, channels=cfg.channels,
                    n_qbins=cfg.n_coarse, n_dbins=cfg.n_defocus, max_batch=128, seed=2)
    losses = proposal.train(net, imgs, torch.from_numpy(tr["label_q"]).to(dev), torch.from_numpy(tr["label_d"]).to(dev),
                            epochs=8, batch=128, lr=2e-3, gen=gen)
    assert losses[-1] < losses[0]
    inf = workloads.proposal_draws(cfg, cfg.n_infer, 9, models=False)
    x = proposal.compose(ctx, [atoms[0]], inf, cfg, gen)
    bins, _ = net.propose(x, cfg.top_k)
    bins = bins.cpu().numpy().astype(np.int64)
    im = bioem.prepare_images(ctx, x, cfg.pixel_A)
    rng = np.random.default_rng(3)
    n_joint = cfg.n_coarse * cfg.n_defocus
    rand = np.stack([rng.choice(n_joint, cfg.top_k, replace=False) for _ in range(cfg.n_infer)])
    prop = proposal.score_cells(ctx, im, atoms[0], bins, cfg)
    rnd = proposal.score_cells(ctx, im, atoms[0], rand, cfg)
    full = proposal.score_cells(ctx, im, atoms[0], proposal.all_bins(cfg.n_infer, cfg), cfg)
    assert ctx.status() == 0
    # subsets of the grid, normalised by the full grid, can only lose mass
    assert np.all(prop["logP"] <= full["logP"] + 1e-6)
    assert np.all(rnd["logP"] <= full["logP"] + 1e-6)
    assert prop["evals"] == cfg.n_infer * cfg.top_k * cfg.children * len(cfg.bfactors)
    # the wave-gathered full grid equals one bioem_score over the whole fine grid
    fq = torch.from_numpy(workloads.hopf_grid(cfg.fine_level).astype(np.float32)).to(dev)
    ps = bioem.project_model(ctx, atoms[0], cfg.sigma_A, fq, cfg.ctf_rows(), cfg.npix, cfg.pixel_A)
    ref = bioem.score(ctx, im, ps, cfg.max_shift).cpu().numpy()
    np.testing.assert_allclose(full["logP"], ref, rtol=0, atol=1e-6)
    # the learned proposal keeps more posterior mass than random cells of the same number
    kept_prop = prop["logP"] - full["logP"]
    kept_rand = rnd["logP"] - full["logP"]
    print(f"losses {losses}; kept (log mass) proposal median {np.median(kept_prop):.3f} mean {np.mean(kept_prop):.3f}; "
          f"random mean {np.mean(kept_rand):.3f}; evals proposal {prop['evals']} full {full['evals']}")
    assert np.mean(kept_prop) > np.mean(kept_rand) + 1.0, (np.mean(kept_prop), np.mean(kept_rand))
    truth = inf["label_q"].astype(np.int64) * cfg.n_defocus + inf["label_d"]
    recall = np.mean([t in b for t, b in zip(truth, bins)])
    assert recall > cfg.top_k / n_joint
    # exact re-ranking of a 4x wider proposal at the coarse grid points, keeping top_k bins
    big = net.propose(x, 4 * cfg.top_k)[0].cpu().numpy().astype(np.int64)
    rr = proposal.rerank_coarse(ctx, im, atoms[0], big, cfg, cfg.top_k)
    assert rr["bins"].shape == bins.shape and rr["evals"] == cfg.n_infer * 4 * cfg.top_k * len(cfg.bfactors)
    assert all(set(r) <= set(b) for r, b in zip(rr["bins"], big))
    prop_rr = proposal.score_cells(ctx, im, atoms[0], rr["bins"], cfg)
    kept_rr = prop_rr["logP"] - full["logP"]
    recall_rr = np.mean([t in b for t, b in zip(truth, rr["bins"])])
    print(f"re-ranked: recall {recall_rr:.3f} (network top-k {recall:.3f}); kept mean {np.mean(kept_rr):.3f}")
    # the coarse grid point is only a proxy for a cell's fine mass: better than random cells
    assert np.mean(kept_rr) > np.mean(kept_rand) + 1.0, (np.mean(kept_rr), np.mean(kept_rand))
    # the same re-ranking over each cell's 8 children one level finer: its score of a bin is the
    # log-sum-exp, over those orientations and both B, of the library's per-pair values
    rr3 = proposal.rerank_coarse(ctx, im, atoms[0], big, cfg, cfg.top_k, level=cfg.coarse_level + 1)
    assert rr3["evals"] == cfg.n_infer * 4 * cfg.top_k * 8 * len(cfg.bfactors)
    assert all(set(r) <= set(b) for r, b in zip(rr3["bins"], big))
    w = 3
    cells = big[w] // cfg.n_defocus
    q3 = workloads.hopf_grid(cfg.coarse_level + 1).astype(np.float32)
    kids = workloads.hopf_children(cfg.coarse_level, cfg.coarse_level + 1, cells)        # [K, 8]
    ps3 = bioem.project_model(ctx, atoms[0], cfg.sigma_A, torch.from_numpy(q3[kids.ravel()]).to(dev),
                              cfg.ctf_rows(), cfg.npix, cfg.pixel_A)
    im1 = bioem.prepare_images(ctx, x[w:w + 1].contiguous(), cfg.pixel_A)
    _, plse = bioem.score_pairs(ctx, im1, ps3, cfg.max_shift)
    plse = plse.cpu().numpy()[0].reshape(len(cells), 8, cfg.n_defocus, len(cfg.bfactors))
    dd = big[w] % cfg.n_defocus
    v = plse[np.arange(len(cells)), :, dd, :].reshape(len(cells), -1)
    score = v.max(axis=1) + np.log(np.exp(v - v.max(axis=1, keepdims=True)).sum(axis=1))
    # every bin kept scores at least the k-th best score (up to the two kernels' rounding)
    kth = np.sort(score)[::-1][cfg.top_k - 1]
    by_bin = dict(zip(big[w].tolist(), score.tolist()))
    assert all(by_bin[b] >= kth - 1e-3 for b in rr3["bins"][w].tolist())
    # here that level is the fine grid itself, so a bin's score is its fine posterior mass and the k
    # best bins keep the most mass any k of the wide proposal can: at least the network's top k
    assert cfg.coarse_level + 1 == cfg.fine_level
    kept_rr3 = proposal.score_cells(ctx, im, atoms[0], rr3["bins"], cfg)["logP"] - full["logP"]
    assert np.all(kept_rr3 >= kept_prop - 1e-6) and np.all(kept_rr3 >= kept_rr - 1e-6)


def test_gathered_pairs_match_score_pairs(env):
    """Per-pair values of per-image lists equal bioem_score_pairs on the same (image, set) pairs."""
    import torch
    bioem, ctx = env
    import oracle
    cfg = workloads.get_config("tiny")
    wl = workloads.workload(cfg, n_img=5)
    imgs = oracle.synthesize_images(wl)
    dev = torch.device("cuda", 0)
    im = bioem.prepare_images(ctx, torch.from_numpy(imgs).to(dev), cfg.pixel_A)
    ps = bioem.project_model(ctx, torch.from_numpy(wl["atoms"]).to(dev), cfg.sigma_A,
                             torch.from_numpy(wl["quats"][:40]).to(dev), wl["ctfs"], cfg.npix, cfg.pixel_A)
    _, plse = bioem.score_pairs(ctx, im, ps, cfg.max_shift)
    plse = plse.cpu().numpy()
    rng = np.random.default_rng(8)
    lists = [np.sort(rng.choice(240, size=n, replace=False)) for n in (1, 37, 0, 240, 100)]
    off = np.concatenate([[0], np.cumsum([len(x) for x in lists])]).astype(np.int32)
    flat = np.concatenate(lists).astype(np.int32)
    got = bioem.score_gathered_pairs(ctx, im, ps, cfg.max_shift, torch.from_numpy(off).to(dev),
                                     torch.from_numpy(flat).to(dev), 240).cpu().numpy()
    assert ctx.status() == 0
    ref = np.concatenate([plse[w, x] for w, x in enumerate(lists)])
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-9)
