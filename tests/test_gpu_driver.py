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


def test_acc_merge_and_group_logsumexp(bioem):
    """The library's (M, S) merge equals the log-sum-exp of the union, folding parts in order (an
    empty part is the identity); its per-group log-sum-exp equals scipy's."""
    import scipy.special
    import torch
    ctx = bioem.Context(0)
    rng = np.random.default_rng(11)
    x = -4000.0 + 50.0 * rng.standard_normal((37, 1000))
    cuts = [(0, 1), (1, 333), (333, 334), (334, 1000)]
    parts = []
    for a, b in cuts:
        m = x[:, a:b].max(axis=1)
        parts.append(np.stack([m, np.exp(x[:, a:b] - m[:, None]).sum(axis=1)], axis=1))
    parts.append(np.tile([-np.inf, 0.0], (37, 1)))   # an empty part
    d = torch.from_numpy(np.stack(parts)).cuda()
    merged = bioem.acc_merge(ctx, d).cpu().numpy()
    np.testing.assert_allclose(merged[:, 0] + np.log(merged[:, 1]), scipy.special.logsumexp(x, axis=1), rtol=1e-14)
    from paper_1609_06634_gb300 import driver
    pair = driver.merge_partials(ctx, d[0], d[4]).cpu().numpy()
    np.testing.assert_array_equal(pair, parts[0])
    # in place: out aliases the first part
    inplace = bioem.acc_merge(ctx, d, out=d[0])
    np.testing.assert_array_equal(inplace.cpu().numpy(), merged)
    v = -300.0 + 20.0 * rng.standard_normal(3 * 2 * 1001)
    v[5] = -np.inf
    g = bioem.group_logsumexp(ctx, torch.from_numpy(v).cuda(), 2).cpu().numpy()
    np.testing.assert_allclose(g, scipy.special.logsumexp(v.reshape(-1, 2), axis=1), rtol=1e-14)
    allinf = bioem.group_logsumexp(ctx, torch.full((4,), -np.inf, dtype=torch.float64, device="cuda"), 4)
    assert allinf.item() == -np.inf
    assert ctx.status() == 0


def test_fma_peak_measures_cuda_core_throughput(bioem):
    """The FMA microbenchmark returns plausible CUDA-core rates: FP32 near 152 SMs x 128 lanes x 2
    flop x the SM clock (tens of TFLOP/s), FP64 far below FP32."""
    ctx = bioem.Context(0)
    f32 = bioem.fma_peak(ctx, "fp32", reps=2)
    f32x2 = bioem.fma_peak(ctx, "fp32x2", reps=2)
    f64 = bioem.fma_peak(ctx, "fp64", reps=2)
    assert 1e13 < max(f32, f32x2) < 3e14, (f32, f32x2)
    assert 1e10 < f64 < f32, (f64, f32)
