"""GPU: the chunked, resumable orientation scan gives bioem_score's log P (and the oracle's), also
when interrupted and resumed from its checkpoint, in the FP32 and a tensor-core form."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


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
def case(bioem):
    import torch
    cfg = workloads.get_config("tiny")
    wl = workloads.workload(cfg, n_img=6)
    imgs = oracle.synthesize_images(wl)
    ctx = bioem.Context(0)
    im = bioem.prepare_images(ctx, torch.from_numpy(imgs).cuda(), cfg.pixel_A)
    atoms = torch.from_numpy(wl["atoms"]).cuda()
    return cfg, wl, imgs, ctx, im, atoms


@pytest.mark.parametrize("mode", ["fp32", "bf16x2"])
def test_chunked_scan_equals_one_pass(bioem, case, mode, tmp_path):
    import torch
    from paper_1609_06634_gb300 import driver
    cfg, wl, imgs, ctx, im, atoms = case
    quats = wl["quats"][:700]
    ctx.set_precision(mode)
    try:
        ps = bioem.project_model(ctx, atoms, cfg.sigma_A, torch.from_numpy(quats).cuda(), wl["ctfs"], cfg.npix,
                                 cfg.pixel_A)
        one = bioem.score(ctx, im, ps, cfg.max_shift).cpu().numpy()
        ps.close()
        scan = driver.OrientationScan(ctx, im, atoms, cfg.sigma_A, quats, wl["ctfs"], cfg.npix, cfg.pixel_A,
                                      cfg.max_shift, chunk=160)
        assert scan.run()
        chunked = scan.log_p().cpu().numpy()
        # interrupted after two chunks, resumed by a new scan object from the checkpoint
        path = str(tmp_path / f"scan_{mode}.npz")
        first = driver.OrientationScan(ctx, im, atoms, cfg.sigma_A, quats, wl["ctfs"], cfg.npix, cfg.pixel_A,
                                       cfg.max_shift, chunk=160, checkpoint=path)
        assert not first.run(max_chunks=2)
        with pytest.raises(RuntimeError):
            first.log_p()
        second = driver.OrientationScan(ctx, im, atoms, cfg.sigma_A, quats, wl["ctfs"], cfg.npix, cfg.pixel_A,
                                        cfg.max_shift, chunk=160, checkpoint=path)
        assert second.next_chunk == 2
        assert second.run()
        resumed = second.log_p().cpu().numpy()
        assert ctx.status() == 0
    finally:
        ctx.set_precision("fp32")
    np.testing.assert_allclose(chunked, one, rtol=0, atol=1e-9)
    np.testing.assert_allclose(resumed, chunked, rtol=0, atol=1e-12)
    ref = oracle.score(imgs, wl["atoms"], quats, wl["ctfs"], cfg.sigma_A, cfg.pixel_A, cfg.max_shift)["logP"]
    np.testing.assert_allclose(chunked, ref, rtol=0, atol=1e-3 if mode == "fp32" else 1e-2)
