"""GPU parity of the split-precision tensor-core scoring forms (BF16 and FP16 two-term GEMMs, Sec. 3.9's
single- versus double-precision question taken to 16-bit operands; over the half spectrum and, as in
Sec. 3.3's real-space variant, over pixels) against the FP64 oracle.

Tolerance: |d log P| <= 1e-2 per image for the split-precision forms (the FP32 form's bound stays
1e-3, checked on the same inputs).  Maximising grid points must match wherever the oracle's best
exceeds its runner-up by more than 0.1.  The precision subsets (64 images x 6912 parameter sets,
128 px and 64 px, shifts +-4) are compared with oracle values stored by tests/golden/make_golden.py.
"""
import os

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu
TOL = 1e-2
TOL_FP32 = 1e-3
MODES = ["bf16x2", "fp16x2", "bf16x2_real", "fp16x2_real"]
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


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


def _handles(bioem, ctx, imgs, atoms, quats, ctfs, cfg):
    im = bioem.prepare_images(ctx, _dev(imgs), cfg.pixel_A)
    ps = bioem.project_model(ctx, _dev(atoms), cfg.sigma_A, _dev(quats), ctfs, cfg.npix, cfg.pixel_A)
    return im, ps


def _score(bioem, ctx, mode, im, ps, max_shift, **kw):
    ctx.set_precision(mode)
    try:
        out = bioem.score_all(ctx, im, ps, max_shift, **kw)
        assert ctx.status() == 0
        return {k: v.cpu().numpy() for k, v in out.items()}
    finally:
        ctx.set_precision("fp32")


def _check_best(out, ref, tol):
    np.testing.assert_allclose(out["best_logL"], [b[4] for b in ref["best"]], rtol=0, atol=tol)
    for w, b in enumerate(ref["best"]):
        s = np.sort(ref["pair_max"][w])
        if s[-1] - s[-2] > 0.1:
            got = (out["best_q"][w], out["best_ctf"][w], out["best_dy"][w], out["best_dx"][w])
            assert tuple(int(v) for v in got) == tuple(b[:4]), (w, got, b)


@pytest.mark.parametrize("mode", MODES)
def test_small_case(bioem, ctx, mode):
    """32 px, 3 images x 7 orientations x 6 PSFs, +-4 px: every output against the oracle."""
    cfg = workloads.get_config("tiny")
    wl = workloads.workload(cfg, n_img=3)
    imgs = oracle.synthesize_images(wl)
    quats = wl["quats"][:7]
    ref = oracle.score(imgs, wl["atoms"], quats, wl["ctfs"], cfg.sigma_A, cfg.pixel_A, cfg.max_shift)
    im, ps = _handles(bioem, ctx, imgs, wl["atoms"], quats, wl["ctfs"], cfg)
    out = _score(bioem, ctx, mode, im, ps, cfg.max_shift, per_orient=True, best=True)
    np.testing.assert_allclose(out["logP"], ref["logP"], rtol=0, atol=TOL)
    np.testing.assert_allclose(out["logP_orient"], ref["logP_orient"], rtol=0, atol=TOL)
    _check_best(out, ref, TOL)


# (config, orientations, images, max_shift): parameter-set counts that leave a ragged last row tile
# (6 PSFs per orientation; 128 sets per tile), image counts that leave a ragged column tile
# (floor(256 / (2 s + 1)^2) images per tile), the smallest and largest windows (s = 0: one column per
# image; s = 7: 225 of 256 columns), and the 64 and 128 px sizes.
CASES = [("tiny", 45, 5, 4), ("tiny", 11, 7, 2), ("tiny", 5, 4, 0), ("tiny", 30, 2, 7),
         ("precision64", 23, 4, 4), ("precision64", 9, 3, 6), ("precision128", 25, 4, 4), ("precision128", 6, 2, 7)]


@pytest.mark.parametrize("name,nq,n_img,max_shift", CASES)
@pytest.mark.parametrize("mode", MODES)
def test_ragged_tiles_and_windows(bioem, ctx, mode, name, nq, n_img, max_shift):
    cfg = workloads.get_config(name)
    wl = workloads.workload(cfg, n_img=n_img)
    imgs = oracle.synthesize_images(wl)
    quats = wl["quats"][:nq]
    ref = oracle.score(imgs, wl["atoms"], quats, wl["ctfs"], cfg.sigma_A, cfg.pixel_A, max_shift)
    im, ps = _handles(bioem, ctx, imgs, wl["atoms"], quats, wl["ctfs"], cfg)
    out = _score(bioem, ctx, mode, im, ps, max_shift, per_orient=True, best=True)
    np.testing.assert_allclose(out["logP"], ref["logP"], rtol=0, atol=TOL)
    np.testing.assert_allclose(out["logP_orient"], ref["logP_orient"], rtol=0, atol=TOL)
    _check_best(out, ref, TOL)


@pytest.mark.parametrize("npix,max_shift", [(96, 5), (192, 7)])
@pytest.mark.parametrize("mode", ["bf16x2", "fp16x2_real"])
def test_other_image_sizes(bioem, ctx, mode, npix, max_shift):
    """96 and 192 px (K = 9408 / 37,248 Fourier terms, 9216 / 36,864 pixels), ragged tiles."""
    cfg = workloads.get_config("tiny", npix=npix, pixel_A=2.0)
    wl = workloads.workload(cfg, n_img=3)
    imgs = oracle.synthesize_images(wl)
    quats = wl["quats"][:23]
    ref = oracle.score(imgs, wl["atoms"], quats, wl["ctfs"], cfg.sigma_A, cfg.pixel_A, max_shift)
    im, ps = _handles(bioem, ctx, imgs, wl["atoms"], quats, wl["ctfs"], cfg)
    out = _score(bioem, ctx, mode, im, ps, max_shift, per_orient=True, best=True)
    np.testing.assert_allclose(out["logP"], ref["logP"], rtol=0, atol=TOL)
    np.testing.assert_allclose(out["logP_orient"], ref["logP_orient"], rtol=0, atol=TOL)
    _check_best(out, ref, TOL)


@pytest.mark.parametrize("mode", MODES)
def test_pairs_unaligned_range(bioem, ctx, mode):
    """score_pairs over sets [100, 800): row tiles cut by the range at both ends."""
    cfg = workloads.get_config("tiny")
    wl = workloads.workload(cfg, n_img=4)
    imgs = oracle.synthesize_images(wl)
    quats = wl["quats"][:150]
    ref = oracle.score(imgs, wl["atoms"], quats, wl["ctfs"], cfg.sigma_A, cfg.pixel_A, cfg.max_shift)
    im, ps = _handles(bioem, ctx, imgs, wl["atoms"], quats, wl["ctfs"], cfg)
    ctx.set_precision(mode)
    try:
        pmax, plse = bioem.score_pairs(ctx, im, ps, cfg.max_shift, 100, 700)
        assert ctx.status() == 0
    finally:
        ctx.set_precision("fp32")
    np.testing.assert_allclose(pmax.cpu().numpy(), ref["pair_max"][:, 100:800], rtol=0, atol=TOL)
    np.testing.assert_allclose(plse.cpu().numpy(), ref["pair_lse"][:, 100:800], rtol=0, atol=TOL)


@pytest.mark.parametrize("mode", MODES)
def test_waves_match_single_pass(bioem, ctx, mode):
    """A small record budget splits the grid into waves (row tiles recomputed at cut points)."""
    cfg = workloads.get_config("tiny")
    wl = workloads.workload(cfg, n_img=5)
    imgs = oracle.synthesize_images(wl)
    quats = wl["quats"][:200]
    im, ps = _handles(bioem, ctx, imgs, wl["atoms"], quats, wl["ctfs"], cfg)
    one = _score(bioem, ctx, mode, im, ps, cfg.max_shift, per_orient=True, best=True)
    ctx.set_scratch_limit(5 * 12 * 200)   # 200 sets per wave: not a multiple of the 128-set tile
    try:
        many = _score(bioem, ctx, mode, im, ps, cfg.max_shift, per_orient=True, best=True)
    finally:
        ctx.set_scratch_limit(2 << 30)
    for k in one:
        np.testing.assert_allclose(many[k], one[k], rtol=0, atol=1e-9, err_msg=k)


def test_mode_switch_rebuilds_operands(bioem, ctx):
    """FP32 -> BF16 -> FP16 -> BF16 at another window -> FP32: operands rebuilt as needed and the
    FP32 result unchanged by the detour."""
    cfg = workloads.get_config("tiny")
    wl = workloads.workload(cfg, n_img=4)
    imgs = oracle.synthesize_images(wl)
    quats = wl["quats"][:20]
    im, ps = _handles(bioem, ctx, imgs, wl["atoms"], quats, wl["ctfs"], cfg)
    first = _score(bioem, ctx, "fp32", im, ps, 4)["logP"]
    r4 = oracle.score(imgs, wl["atoms"], quats, wl["ctfs"], cfg.sigma_A, cfg.pixel_A, 4)["logP"]
    r2 = oracle.score(imgs, wl["atoms"], quats, wl["ctfs"], cfg.sigma_A, cfg.pixel_A, 2)["logP"]
    for mode, s, ref in [("bf16x2", 4, r4), ("fp16x2", 4, r4), ("bf16x2", 2, r2), ("fp16x2_real", 2, r2),
                         ("bf16x2_real", 4, r4), ("fp16x2", 2, r2)]:
        np.testing.assert_allclose(_score(bioem, ctx, mode, im, ps, s)["logP"], ref, rtol=0, atol=TOL)
    np.testing.assert_array_equal(_score(bioem, ctx, "fp32", im, ps, 4)["logP"], first)


def test_errors(bioem, ctx):
    import torch
    cfg = workloads.get_config("tiny")
    wl = workloads.workload(cfg, n_img=2)
    imgs = oracle.synthesize_images(wl)
    im, ps = _handles(bioem, ctx, imgs, wl["atoms"], wl["quats"][:4], wl["ctfs"], cfg)
    with pytest.raises(bioem.BioEMError) as e:
        ctx.set_precision(7)
    assert e.value.code == bioem.ERR_INVALID_ARG
    ctx.set_precision("fp16x2")
    try:
        assert ctx.precision == "fp16x2"
        im64 = bioem.prepare_images(ctx, torch.randn((1, 64, 64), device="cuda:0"), cfg.pixel_A)
        ps64 = bioem.project_model(ctx, _dev(wl["atoms"]), cfg.sigma_A, _dev(wl["quats"][:2]), wl["ctfs"], 64,
                                   cfg.pixel_A)
        with pytest.raises(bioem.BioEMError) as e:
            bioem.score(ctx, im64, ps64, 8)   # 17^2 columns per image exceed one 256-column tile
        assert e.value.code == bioem.ERR_UNSUPPORTED_SIZE
        # the allocation-free entry point keeps the FP32 form whatever the mode
        out = torch.empty(2, dtype=torch.float64, device="cuda:0")
        bioem.score_noalloc(ctx, im, ps, 4, out)
        got = out.cpu().numpy()
    finally:
        ctx.set_precision("fp32")
    np.testing.assert_array_equal(got, bioem.score(ctx, im, ps, 4).cpu().numpy())
    assert ctx.status() == 0


def _golden(name):
    path = os.path.join(GOLDEN, f"{name}_subset.txt")
    t = np.loadtxt(path, ndmin=2)
    return {"logP": t[:, 0], "best_logL": t[:, 1], "best": t[:, 2:6].astype(int), "margin": t[:, 6]}


@pytest.mark.parametrize("name", ["precision64", "precision128"])
def test_precision_subset(bioem, ctx, name):
    """The 64-image subsets on the full 6912-set grid: every form against the stored oracle values."""
    cfg = workloads.get_config(name)
    ref = _golden(name)
    wl = workloads.workload(cfg)
    imgs = oracle.synthesize_images(wl)
    im, ps = _handles(bioem, ctx, imgs, wl["atoms"], wl["quats"], wl["ctfs"], cfg)
    report = []
    for mode, tol in [("fp32", TOL_FP32)] + [(m, TOL) for m in MODES]:
        out = _score(bioem, ctx, mode, im, ps, cfg.max_shift, best=True)
        diff = out["logP"] - ref["logP"]
        err = np.abs(diff)
        report.append(f"{name} {mode}: max |dlogP| {err.max():.3e} median {np.median(err):.3e} "
                      f"mean signed {diff.mean():+.3e}")
        assert err.max() <= tol, report[-1]
        np.testing.assert_allclose(out["best_logL"], ref["best_logL"], rtol=0, atol=tol)
        clear = ref["margin"] > 0.1
        got = np.stack([out["best_q"], out["best_ctf"], out["best_dy"], out["best_dx"]], axis=1)
        np.testing.assert_array_equal(got[clear], ref["best"][clear])
    print("\n" + "\n".join(report))
