"""The allocation-free scoring entry point (bioem_score_noalloc) against bioem_score.

bioem_score_noalloc exists for callers that may not allocate device memory while they score
(device memory reserved up front by another allocator, or loops that must not stall on
cudaMalloc / cudaFree): its scratch is a fixed 16 MiB array the library reserves when it is
loaded.  These tests call it through the C ABI twice in a row (the second call finds the
previous call's data in the shared array) on a case that needs several passes through that
array, compare both results with bioem_score within the parity tolerance, and check that a
case too large for the array is refused.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu
TOL = 1e-3


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1609_06634_gb300 as bioem
    from paper_1609_06634_gb300 import build
    build.build()
    return bioem, bioem.Context(0)


def _noalloc(bioem, ctx, im, ps, max_shift, out):
    return bioem.lib().bioem_score_noalloc(ctx._h, im._h, ps._h, int(max_shift), ctypes.c_void_p(out.data_ptr()))


def test_noalloc_first_on_a_fresh_context_allocates_nothing(env):
    """On a new context, before any other scoring call: after one warm-up call (which loads the
    kernels' code), a further call leaves the device's free memory unchanged, and both results
    equal bioem_score's, which runs afterwards on the same context."""
    import torch
    bioem, _ = env
    ctx = bioem.Context(0)
    cfg = workloads.get_config("tiny")
    wl = workloads.workload(cfg, n_img=8)
    dev = torch.device("cuda", 0)
    im = bioem.prepare_images(ctx, torch.from_numpy(oracle.synthesize_images(wl)).to(dev), cfg.pixel_A)
    ps = bioem.project_model(ctx, torch.from_numpy(wl["atoms"]).to(dev), cfg.sigma_A,
                             torch.from_numpy(wl["quats"]).to(dev), wl["ctfs"], cfg.npix, cfg.pixel_A)
    out1 = torch.full((8,), float("nan"), dtype=torch.float64, device=dev)
    out2 = torch.full((8,), float("nan"), dtype=torch.float64, device=dev)
    assert _noalloc(bioem, ctx, im, ps, cfg.max_shift, out1) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(dev)
    assert _noalloc(bioem, ctx, im, ps, cfg.max_shift, out2) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(dev)
    assert free1 == free0
    assert ctx.status() == 0
    want = bioem.score(ctx, im, ps, cfg.max_shift).cpu().numpy()
    np.testing.assert_allclose(out1.cpu().numpy(), want, rtol=0, atol=TOL)
    np.testing.assert_allclose(out2.cpu().numpy(), want, rtol=0, atol=TOL)


def test_noalloc_matches_score_twice(env):
    import torch
    bioem, ctx = env
    cfg = workloads.get_config("tiny")
    wl = workloads.workload(cfg)
    base = oracle.synthesize_images(wl)                      # 16 images, 32 x 32
    rng = np.random.default_rng(7)
    imgs = np.tile(base, (128, 1, 1)) + 0.05 * rng.standard_normal((2048, 32, 32))
    dev = torch.device("cuda", 0)
    im = bioem.prepare_images(ctx, torch.from_numpy(imgs.astype(np.float32)).to(dev), cfg.pixel_A)
    ps = bioem.project_model(ctx, torch.from_numpy(wl["atoms"]).to(dev), cfg.sigma_A,
                             torch.from_numpy(wl["quats"]).to(dev), wl["ctfs"], cfg.npix, cfg.pixel_A)
    want = bioem.score(ctx, im, ps, cfg.max_shift).cpu().numpy()
    for _ in range(2):
        out = torch.full((2048,), float("nan"), dtype=torch.float64, device=dev)
        assert _noalloc(bioem, ctx, im, ps, cfg.max_shift, out) == 0
        assert ctx.status() == 0
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        np.testing.assert_allclose(got, want, rtol=0, atol=TOL)


def test_noalloc_refuses_oversized_case(env):
    import torch
    bioem, ctx = env
    cfg = workloads.get_config("tiny")
    wl = workloads.workload(cfg, n_img=1)
    dev = torch.device("cuda", 0)
    ctfs = np.array([(5000.0 + 10.0 * i, 0.1, 0.0, 300.0) for i in range(1500)])
    ps = bioem.project_model(ctx, torch.from_numpy(wl["atoms"]).to(dev), cfg.sigma_A,
                             torch.from_numpy(wl["quats"][:1]).to(dev), ctfs, cfg.npix, cfg.pixel_A)
    gen = torch.Generator(device=dev).manual_seed(3)
    im = bioem.prepare_images(ctx, torch.randn((1200, 32, 32), generator=gen, device=dev), cfg.pixel_A)
    out = torch.empty(1200, dtype=torch.float64, device=dev)
    assert _noalloc(bioem, ctx, im, ps, 2, out) == bioem.ERR_UNSUPPORTED_SIZE
    assert b"static" in bioem.lib().bioem_last_error(ctx._h)
    assert torch.isfinite(bioem.score(ctx, im, ps, 2)).all()
    assert ctx.status() == 0
