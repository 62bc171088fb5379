"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, element by element.

Tolerance: |d log P| <= 1e-3 per image (the FP32 path's bound), the same for per-orientation and
per-pair values; maximising grid points must match exactly wherever the oracle's best exceeds its
runner-up by more than that tolerance.
"""
import math

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


@pytest.fixture(scope="module")
def ctx(bioem):
    return bioem.Context(0)


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def _gpu_score(bioem, ctx, imgs, atoms, quats, ctfs, cfg, max_shift, **kw):
    im = bioem.prepare_images(ctx, _dev(imgs), cfg.pixel_A)
    ps = bioem.project_model(ctx, _dev(atoms), cfg.sigma_A, _dev(quats), ctfs, cfg.npix, cfg.pixel_A)
    out = bioem.score_all(ctx, im, ps, max_shift, **kw)
    assert ctx.status() == 0
    return {k: v.cpu().numpy() for k, v in out.items()}, im, ps


@pytest.fixture(scope="module")
def tiny_case():
    cfg = workloads.get_config("tiny")
    wl = workloads.workload(cfg)
    imgs = oracle.synthesize_images(wl)
    ref = oracle.score(imgs, wl["atoms"], wl["quats"], wl["ctfs"], cfg.sigma_A, cfg.pixel_A, cfg.max_shift)
    return cfg, wl, imgs, ref


def _best_margin(ref_pairs_max_row):
    s = np.sort(ref_pairs_max_row)
    return s[-1] - s[-2]


def test_tiny_full_grid_logP(bioem, ctx, tiny_case):
    cfg, wl, imgs, ref = tiny_case
    out, _, _ = _gpu_score(bioem, ctx, imgs, wl["atoms"], wl["quats"], wl["ctfs"], cfg, cfg.max_shift,
                           per_orient=True, best=True)
    np.testing.assert_allclose(out["logP"], ref["logP"], rtol=0, atol=TOL)
    np.testing.assert_allclose(out["logP_orient"], ref["logP_orient"], rtol=0, atol=TOL)
    np.testing.assert_allclose(out["best_logL"], [b[4] for b in ref["best"]], rtol=0, atol=TOL)
    for w, b in enumerate(ref["best"]):
        if _best_margin(ref["pair_max"][w]) > 10 * TOL:
            got = (out["best_q"][w], out["best_ctf"][w], out["best_dy"][w], out["best_dx"][w])
            assert tuple(int(v) for v in got) == b[:4], (w, got, b)


def test_tiny_pairs(bioem, ctx, tiny_case):
    cfg, wl, imgs, ref = tiny_case
    _, im, ps = _gpu_score(bioem, ctx, imgs[:4], wl["atoms"], wl["quats"], wl["ctfs"], cfg, cfg.max_shift)
    pmax, plse = bioem.score_pairs(ctx, im, ps, cfg.max_shift, 100, 700)
    np.testing.assert_allclose(pmax.cpu().numpy(), ref["pair_max"][:4, 100:800], rtol=0, atol=TOL)
    np.testing.assert_allclose(plse.cpu().numpy(), ref["pair_lse"][:4, 100:800], rtol=0, atol=TOL)


@pytest.mark.parametrize("noisy", [False, True])
def test_recovers_truth(bioem, ctx, noisy):
    cfg = workloads.get_config("tiny", n_orient=40, snr=50.0)
    wl = workloads.workload(cfg, n_img=5)
    truth = [(3, 1, -2, 4), (17, 4, 3, -1), (0, 5, 0, 0), (39, 2, -4, -4), (21, 0, 4, 3)]
    imgs = []
    for i, (iq, ic, dy, dx) in enumerate(truth):
        img1 = oracle.apply_psf(oracle.project(wl["atoms"], wl["quats"][iq], cfg.sigma_A, cfg.npix, cfg.pixel_A),
                                wl["ctfs"][ic], cfg.pixel_A)
        imgs.append(oracle.synthesize_image(img1, dx, dy, 1.3, 0.4, wl["noise"][i] if noisy else None, cfg.snr))
    imgs = np.asarray(imgs, dtype=np.float32)
    import torch
    im = bioem.prepare_images(ctx, _dev(imgs), cfg.pixel_A)
    ps = bioem.project_model(ctx, _dev(wl["atoms"]), cfg.sigma_A, _dev(wl["quats"]), wl["ctfs"], cfg.npix, cfg.pixel_A)
    b = bioem.best_params(ctx, im, ps, cfg.max_shift)
    ctx.status()   # noiseless images may reach |rho| = 1 in float32: the status word may say NUMERIC
    got = list(zip(*(b[k].cpu().numpy().tolist() for k in ("q", "ctf", "dy", "dx"))))
    assert [tuple(g) for g in got] == truth
    del torch


def test_throughput_shape_subset(bioem, ctx):
    """128 x 128 images, +-16 px shifts, 256 orientations x 8 PSFs: all values against the oracle."""
    cfg = workloads.get_config("throughput")
    wl = workloads.workload(cfg, n_img=6)
    quats = wl["quats"][::144][:256]
    imgs = oracle.synthesize_images(wl)
    ref = oracle.score(imgs, wl["atoms"], quats, wl["ctfs"], cfg.sigma_A, cfg.pixel_A, cfg.max_shift)
    out, im, ps = _gpu_score(bioem, ctx, imgs, wl["atoms"], quats, wl["ctfs"], cfg, cfg.max_shift,
                             per_orient=True, best=True)
    np.testing.assert_allclose(out["logP"], ref["logP"], rtol=0, atol=TOL)
    np.testing.assert_allclose(out["logP_orient"], ref["logP_orient"], rtol=0, atol=TOL)
    np.testing.assert_allclose(out["best_logL"], [b[4] for b in ref["best"]], rtol=0, atol=TOL)
    pmax, plse = bioem.score_pairs(ctx, im, ps, cfg.max_shift)
    np.testing.assert_allclose(pmax.cpu().numpy(), ref["pair_max"], rtol=0, atol=TOL)
    np.testing.assert_allclose(plse.cpu().numpy(), ref["pair_lse"], rtol=0, atol=TOL)


@pytest.mark.parametrize("s", [16, 9])
def test_throughput_pairs_ragged_ranges(bioem, ctx, s):
    """128 px, the +-16 px kernel (pairs of a batch split between four thread groups): per-pair values
    for ranges that leave groups with only some, or none, of their pairs inside the range (7 sets
    from an odd offset, 3 sets, 13 sets across two batches), against the oracle."""
    cfg = workloads.get_config("throughput")
    wl = workloads.workload(cfg, n_img=3)
    imgs = oracle.synthesize_images(wl)
    quats = wl["quats"][::1024][:4]                       # 32 parameter sets
    ref = oracle.score(imgs, wl["atoms"], quats, wl["ctfs"], cfg.sigma_A, cfg.pixel_A, s)
    im = bioem.prepare_images(ctx, _dev(imgs), cfg.pixel_A)
    ps = bioem.project_model(ctx, _dev(wl["atoms"]), cfg.sigma_A, _dev(quats), wl["ctfs"], cfg.npix, cfg.pixel_A)
    for begin, count in ((5, 7), (9, 3), (17, 13), (0, 32)):
        pmax, plse = bioem.score_pairs(ctx, im, ps, s, begin, count)
        assert ctx.status() == 0
        np.testing.assert_allclose(pmax.cpu().numpy(), ref["pair_max"][:, begin:begin + count], rtol=0, atol=TOL)
        np.testing.assert_allclose(plse.cpu().numpy(), ref["pair_lse"][:, begin:begin + count], rtol=0, atol=TOL)


@pytest.mark.parametrize("name,nq,max_shift", [("tiny", 13, 4), ("tiny", 11, 2), ("tiny", 7, 0),
                                              ("precision64", 9, 4), ("precision64", 5, 8), ("precision128", 6, 4),
                                              ("precision128", 3, 11)])
def test_ragged_and_partial_windows(bioem, ctx, name, nq, max_shift):
    """Parameter-set counts that leave a ragged last batch, shift windows below the kernel's maximum."""
    cfg = workloads.get_config(name)
    wl = workloads.workload(cfg, n_img=3)
    imgs = oracle.synthesize_images(wl)
    quats = wl["quats"][:nq]
    ref = oracle.score(imgs, wl["atoms"], quats, wl["ctfs"], cfg.sigma_A, cfg.pixel_A, max_shift)
    out, _, _ = _gpu_score(bioem, ctx, imgs, wl["atoms"], quats, wl["ctfs"], cfg, max_shift, per_orient=True, best=True)
    np.testing.assert_allclose(out["logP"], ref["logP"], rtol=0, atol=TOL)
    np.testing.assert_allclose(out["logP_orient"], ref["logP_orient"], rtol=0, atol=TOL)
    np.testing.assert_allclose(out["best_logL"], [b[4] for b in ref["best"]], rtol=0, atol=TOL)


def test_waves_match_single_pass(bioem, ctx, tiny_case):
    """A small record budget splits the grid into many waves; results agree with one wave."""
    cfg, wl, imgs, ref = tiny_case
    one, _, _ = _gpu_score(bioem, ctx, imgs, wl["atoms"], wl["quats"], wl["ctfs"], cfg, cfg.max_shift,
                           per_orient=True, best=True)
    ctx.set_scratch_limit(16 * 12 * 600)   # 600 parameter sets per wave for 16 images
    try:
        many, _, _ = _gpu_score(bioem, ctx, imgs, wl["atoms"], wl["quats"], wl["ctfs"], cfg, cfg.max_shift,
                                per_orient=True, best=True)
    finally:
        ctx.set_scratch_limit(2 << 30)
    np.testing.assert_allclose(many["logP"], one["logP"], rtol=0, atol=1e-9)
    np.testing.assert_array_equal(many["logP_orient"], one["logP_orient"])
    for k in ("best_q", "best_ctf", "best_dx", "best_dy", "best_logL"):
        np.testing.assert_array_equal(many[k], one[k])


def test_invariances_on_gpu(bioem, ctx, tiny_case):
    """log P is unchanged by an image offset and shifts by -(n-3) ln s under image scaling."""
    cfg, wl, imgs, ref = tiny_case
    quats = wl["quats"][:64]
    base, _, _ = _gpu_score(bioem, ctx, imgs, wl["atoms"], quats, wl["ctfs"], cfg, cfg.max_shift)
    off, _, _ = _gpu_score(bioem, ctx, imgs + np.float32(2.5), wl["atoms"], quats, wl["ctfs"], cfg, cfg.max_shift)
    sc, _, _ = _gpu_score(bioem, ctx, imgs * np.float32(4.0), wl["atoms"], quats, wl["ctfs"], cfg, cfg.max_shift)
    n = cfg.npix ** 2
    np.testing.assert_allclose(off["logP"], base["logP"], rtol=0, atol=TOL)
    np.testing.assert_allclose(sc["logP"], base["logP"] - (n - 3) * math.log(4.0), rtol=0, atol=TOL)


def test_deterministic(bioem, ctx, tiny_case):
    cfg, wl, imgs, ref = tiny_case
    a, _, _ = _gpu_score(bioem, ctx, imgs, wl["atoms"], wl["quats"][:200], wl["ctfs"], cfg, cfg.max_shift, best=True)
    b, _, _ = _gpu_score(bioem, ctx, imgs, wl["atoms"], wl["quats"][:200], wl["ctfs"], cfg, cfg.max_shift, best=True)
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])


def test_synthetic_maps_match_oracle(bioem, ctx):
    cfg = workloads.get_config("precision64")
    wl = workloads.workload(cfg, n_img=1)
    quats = wl["quats"][:4]
    ctfs = wl["ctfs"][[0, 1, 4, 5]]
    got = bioem.synthetic_maps(ctx, _dev(wl["atoms"]), cfg.sigma_A, _dev(quats), ctfs, cfg.npix, cfg.pixel_A)
    got = got.cpu().numpy()
    for i in range(4):
        want = oracle.apply_psf(oracle.project(wl["atoms"], quats[i], cfg.sigma_A, cfg.npix, cfg.pixel_A),
                                ctfs[i], cfg.pixel_A)
        assert np.max(np.abs(got[i] - want)) <= 1e-4 * np.max(np.abs(want))


def test_errors_and_status(bioem, ctx):
    import torch
    with pytest.raises(bioem.BioEMError) as e:
        bioem.prepare_images(ctx, torch.zeros((2, 48, 48), device="cuda:0"), 1.0)
    assert e.value.code == bioem.ERR_UNSUPPORTED_SIZE
    cfg = workloads.get_config("tiny")
    wl = workloads.workload(cfg, n_img=1)
    im = bioem.prepare_images(ctx, torch.ones((2, 32, 32), device="cuda:0"), cfg.pixel_A)   # zero variance
    assert ctx.status() == bioem.ERR_NUMERIC
    ps = bioem.project_model(ctx, _dev(wl["atoms"]), cfg.sigma_A, _dev(wl["quats"][:4]), wl["ctfs"], 32, cfg.pixel_A)
    with pytest.raises(bioem.BioEMError) as e:
        bioem.score(ctx, im, ps, 5)
    assert e.value.code == bioem.ERR_UNSUPPORTED_SIZE
    im64 = bioem.prepare_images(ctx, torch.randn((1, 64, 64), device="cuda:0"), cfg.pixel_A)
    with pytest.raises(bioem.BioEMError) as e:
        bioem.score(ctx, im64, ps, 2)
    assert e.value.code == bioem.ERR_INVALID_ARG
    empty = bioem.prepare_images(ctx, torch.zeros((0, 32, 32), device="cuda:0"), cfg.pixel_A)
    assert bioem.score(ctx, empty, ps, 2).numel() == 0
    assert ctx.status() == 0
