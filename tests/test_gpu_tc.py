"""GPU parity of the FP32 form with its column transforms on the tensor cores (precision mode
"fp16x2_fft": split-FP16 tcgen05 products for the ky stage of the pruned inverse transform, the
rest in FP32), against the FP64 oracle, element by element, at the FP32 path's 1e-3.

Cases: 128 px throughput-model images against parameter sets around each image's true orientation
(the posterior peak, where rho is largest and the FP32 error budget is tightest) and random ones;
per-orientation posteriors and maximising parameters; per-pair values over a ragged range (the
last group of four pairs partly empty); smaller shift windows than the kernel's +-16; more work
items than SMs (several groups and items per block); unsupported sizes refused.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu
TOL = 1e-3


@pytest.fixture(scope="module")
def bioem():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1609_06634_gb300 as pkg
    from paper_1609_06634_gb300 import build
    build.build()
    return pkg


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


@pytest.fixture(scope="module")
def case(bioem):
    """6 throughput-workload images; orientations: each image's 12 nearest grid orientations and
    24 shared random ones (x 8 PSFs)."""
    cfg = workloads.get_config("throughput")
    wl = workloads.workload(cfg, n_img=6)
    imgs = oracle.synthesize_images(wl)
    rng = np.random.default_rng(128)
    qs = list(rng.choice(len(wl["quats"]), size=24, replace=False))
    for i in range(6):
        for q in workloads.nearest_orientations(wl["quats"], workloads.image_truth(cfg, i)["quat"], 12):
            if q not in qs:
                qs.append(int(q))
    quats = wl["quats"][np.array(qs)]
    projs = oracle.projections(wl["atoms"], quats, wl["ctfs"], cfg.sigma_A, cfg.npix, cfg.pixel_A)
    ref = oracle.score(imgs, wl["atoms"], quats, wl["ctfs"], cfg.sigma_A, cfg.pixel_A, cfg.max_shift, projs=projs)
    ctx = bioem.Context(0)
    im = bioem.prepare_images(ctx, _dev(imgs), cfg.pixel_A)
    ps = bioem.project_model(ctx, _dev(wl["atoms"]), cfg.sigma_A, _dev(quats), wl["ctfs"], cfg.npix, cfg.pixel_A)
    return cfg, wl, imgs, quats, projs, ref, ctx, im, ps


def _with_mode(ctx, mode, fn):
    ctx.set_precision(mode)
    try:
        return fn()
    finally:
        ctx.set_precision("fp32")


def test_tc_matches_oracle_at_the_peak(bioem, case):
    cfg, wl, imgs, quats, projs, ref, ctx, im, ps = case
    out = _with_mode(ctx, "fp16x2_fft", lambda: bioem.score_all(ctx, im, ps, cfg.max_shift, per_orient=True,
                                                                 best=True))
    assert ctx.status() == 0
    got = {k: v.cpu().numpy() for k, v in out.items()}
    np.testing.assert_allclose(got["logP"], ref["logP"], rtol=0, atol=TOL)
    np.testing.assert_allclose(got["logP_orient"], ref["logP_orient"], rtol=0, atol=TOL)
    np.testing.assert_allclose(got["best_logL"], [b[4] for b in ref["best"]], rtol=0, atol=TOL)
    for w, b in enumerate(ref["best"]):
        srt = np.sort(ref["pair_max"][w])
        if srt[-1] - srt[-2] > 10 * TOL:
            g = (got["best_q"][w], got["best_ctf"][w], got["best_dy"][w], got["best_dx"][w])
            assert tuple(int(v) for v in g) == b[:4], (w, g, b)
    # and against the FP32 form on the CUDA cores
    fp32 = bioem.score(ctx, im, ps, cfg.max_shift).cpu().numpy()
    np.testing.assert_allclose(got["logP"], fp32, rtol=0, atol=TOL)


def test_tc_pairs_ragged_range(bioem, case):
    """Per-pair max_d ln L and ln sum_d L for 7 parameter sets from an odd offset (groups of four
    pairs: the second one ragged), and for every set."""
    cfg, wl, imgs, quats, projs, ref, ctx, im, ps = case
    pmax, plse = _with_mode(ctx, "fp16x2_fft", lambda: bioem.score_pairs(ctx, im, ps, cfg.max_shift, 13, 7))
    assert ctx.status() == 0
    np.testing.assert_allclose(pmax.cpu().numpy(), ref["pair_max"][:, 13:20], rtol=0, atol=TOL)
    np.testing.assert_allclose(plse.cpu().numpy(), ref["pair_lse"][:, 13:20], rtol=0, atol=TOL)
    pmax, plse = _with_mode(ctx, "fp16x2_fft", lambda: bioem.score_pairs(ctx, im, ps, cfg.max_shift))
    np.testing.assert_allclose(pmax.cpu().numpy(), ref["pair_max"], rtol=0, atol=TOL)
    np.testing.assert_allclose(plse.cpu().numpy(), ref["pair_lse"], rtol=0, atol=TOL)


@pytest.mark.parametrize("s", [0, 3, 9])
def test_tc_smaller_windows(bioem, case, s):
    """The +-16 kernel scores smaller windows by masking displacements outside them."""
    cfg, wl, imgs, quats, projs, ref, ctx, im, ps = case
    r = oracle.score(imgs[:3], wl["atoms"], quats[:16], wl["ctfs"], cfg.sigma_A, cfg.pixel_A, s, projs=projs[:128])
    ps16 = bioem.project_model(ctx, _dev(wl["atoms"]), cfg.sigma_A, _dev(quats[:16]), wl["ctfs"], cfg.npix,
                               cfg.pixel_A)
    im3 = bioem.prepare_images(ctx, _dev(imgs[:3]), cfg.pixel_A)
    out = _with_mode(ctx, "fp16x2_fft", lambda: bioem.score_all(ctx, im3, ps16, s, per_orient=True, best=True))
    assert ctx.status() == 0
    np.testing.assert_allclose(out["logP"].cpu().numpy(), r["logP"], rtol=0, atol=TOL)
    np.testing.assert_allclose(out["logP_orient"].cpu().numpy(), r["logP_orient"], rtol=0, atol=TOL)
    np.testing.assert_allclose(out["best_logL"].cpu().numpy(), [b[4] for b in r["best"]], rtol=0, atol=TOL)


def test_tc_many_items_matches_fp32_form(bioem):
    """Many work items per block (600 images x 2304 sets: ~9 items and ~1300 groups per block,
    items spanning several chunks): ln P and per-orientation ln P within 1e-3 of the FP32 form,
    and two runs bit-identical."""
    import torch
    cfg = workloads.get_config("throughput")
    wl = workloads.workload(cfg, n_img=0)
    ctx = bioem.Context(0)
    gen = torch.Generator(device="cuda:0").manual_seed(5)
    base = torch.from_numpy(oracle.synthesize_images(workloads.workload(cfg, n_img=4))).cuda()
    imgs = base.repeat(150, 1, 1) + 0.3 * torch.randn((600, 128, 128), generator=gen, device="cuda:0")
    im = bioem.prepare_images(ctx, imgs.contiguous(), cfg.pixel_A)
    ps = bioem.project_model(ctx, _dev(wl["atoms"]), cfg.sigma_A, _dev(wl["quats"][::128][:288]), wl["ctfs"],
                             cfg.npix, cfg.pixel_A)
    want = bioem.score_all(ctx, im, ps, cfg.max_shift, per_orient=True)
    a = _with_mode(ctx, "fp16x2_fft", lambda: bioem.score_all(ctx, im, ps, cfg.max_shift, per_orient=True))
    b = _with_mode(ctx, "fp16x2_fft", lambda: bioem.score_all(ctx, im, ps, cfg.max_shift, per_orient=True))
    assert ctx.status() == 0
    np.testing.assert_allclose(a["logP"].cpu().numpy(), want["logP"].cpu().numpy(), rtol=0, atol=TOL)
    np.testing.assert_allclose(a["logP_orient"].cpu().numpy(), want["logP_orient"].cpu().numpy(), rtol=0, atol=TOL)
    assert torch.equal(a["logP"], b["logP"]) and torch.equal(a["logP_orient"], b["logP_orient"])


def test_tc_unsupported_sizes_refused(bioem):
    import torch
    cfg = workloads.get_config("tiny")
    wl = workloads.workload(cfg, n_img=2)
    ctx = bioem.Context(0)
    im = bioem.prepare_images(ctx, _dev(oracle.synthesize_images(wl)), cfg.pixel_A)
    ps = bioem.project_model(ctx, _dev(wl["atoms"]), cfg.sigma_A, _dev(wl["quats"][:4]), wl["ctfs"], cfg.npix,
                             cfg.pixel_A)
    ctx.set_precision("fp16x2_fft")
    try:
        with pytest.raises(bioem.BioEMError) as e:
            bioem.score(ctx, im, ps, cfg.max_shift)
        assert e.value.code == bioem.ERR_UNSUPPORTED_SIZE
    finally:
        ctx.set_precision("fp32")
    assert torch.isfinite(bioem.score(ctx, im, ps, cfg.max_shift)).all()
