"""GPU parity at the throughput workload's full size: 2048 images of 128 x 128 px against 294,912
parameter sets (36,864 Hopf orientations x 4 defocus x 2 B), shifts within +-16 px, scored with the
same entry point and kernel configuration bench.py times.  The oracle cannot score 6e8 pairs, so it
checks sampled outputs it can compute one by one (per-orientation posteriors, the claimed maximum)
and the full result is checked through properties that hold at any size.  The images are made by
the oracle's forward model (no oracle input comes from the CUDA path).
"""
import math

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu
TOL = 1e-3


@pytest.fixture(scope="module")
def full():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1609_06634_gb300 as bioem
    from paper_1609_06634_gb300 import build
    build.build()
    cfg = workloads.get_config("throughput")
    wl = workloads.workload(cfg)
    imgs = oracle.synthesize_images(wl)                     # 2048 x 128 x 128, float32
    ctx = bioem.Context(0)
    dev = torch.device("cuda", 0)
    im = bioem.prepare_images(ctx, torch.from_numpy(imgs).to(dev), cfg.pixel_A)
    ps = bioem.project_model(ctx, torch.from_numpy(wl["atoms"]).to(dev), cfg.sigma_A,
                             torch.from_numpy(wl["quats"]).to(dev), wl["ctfs"], cfg.npix, cfg.pixel_A)
    logp = bioem.score(ctx, im, ps, cfg.max_shift).cpu().numpy()   # the benchmarked call
    out = bioem.score_all(ctx, im, ps, cfg.max_shift, per_orient=True, best=True)
    res = {k: v.cpu().numpy() for k, v in out.items()}
    assert ctx.status() == 0
    ps.close()
    return cfg, wl, imgs, logp, res


def test_full_size_reductions_consistent(full):
    """ln P equals the log-mean over orientations of the per-orientation posteriors (any size)."""
    cfg, wl, imgs, logp, res = full
    assert logp.shape == (2048,) and np.all(np.isfinite(logp))
    np.testing.assert_allclose(res["logP"], logp, rtol=0, atol=1e-9)
    nq = res["logP_orient"].shape[1]
    lse = oracle.logsumexp(res["logP_orient"], axis=1) - math.log(nq)
    np.testing.assert_allclose(lse, logp, rtol=0, atol=1e-6)
    # the maximum lies in the orientation it names: its per-orientation posterior is the largest
    bq = res["best_q"]
    assert np.mean(np.argmax(res["logP_orient"], axis=1) == bq) > 0.95


def test_full_size_sampled_orientations_match_oracle(full):
    """Per-orientation ln P at sampled (image, orientation) pairs, recomputed by the oracle."""
    cfg, wl, imgs, logp, res = full
    rng = np.random.default_rng(2048)
    imgs_sel = rng.choice(2048, size=6, replace=False)
    for w in imgs_sel:
        qs = [int(res["best_q"][w])] + list(rng.choice(36864, size=2, replace=False))
        r = oracle.score(imgs[w:w + 1], wl["atoms"], wl["quats"][qs], wl["ctfs"], cfg.sigma_A, cfg.pixel_A,
                         cfg.max_shift)
        for j, q in enumerate(qs):
            assert abs(res["logP_orient"][w, q] - r["logP_orient"][0, j]) <= TOL, (w, q)
        # the claimed maximum: its ln L, and its parameters, under the oracle
        b = r["best"][0]
        assert abs(res["best_logL"][w] - b[4]) <= TOL
        if b[0] == 0:   # the oracle's best over the claimed orientation's PSFs and shifts
            assert (int(res["best_ctf"][w]), int(res["best_dy"][w]), int(res["best_dx"][w])) == tuple(b[1:4])
