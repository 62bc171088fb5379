"""GPU failure detection without a GPU fault: a bounded barrier wait that is made to run out.

bioem_set_wait_test arms one tensor-core scoring launch to leave one K chunk unfed (no copies in the
split-precision GEMM, no MMAs and no commit in the tensor-core FFT form), with every barrier wait
limited to 5 ms.  The launch must end by itself within a fraction of a second with BIOEM_ERR_TIMEOUT
in the device status word (having waited for what it did issue and freed its tensor memory), and
the next, unarmed call on the same context must succeed with the same results as before.
"""
import time

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


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def _case(bioem, name, n_img, nq, max_shift):
    cfg = workloads.get_config(name)
    wl = workloads.workload(cfg, n_img=n_img)
    ctx = bioem.Context(0)
    im = bioem.prepare_images(ctx, _dev(oracle.synthesize_images(wl)), cfg.pixel_A)
    ps = bioem.project_model(ctx, _dev(wl["atoms"]), cfg.sigma_A, _dev(wl["quats"][:nq]), wl["ctfs"], cfg.npix,
                             cfg.pixel_A)
    return ctx, im, ps, max_shift


@pytest.mark.parametrize("mode,name,nq,max_shift,skip", [
    ("bf16x2", "precision64", 128, 4, 5),       # k_score_gemm: a chunk without copies
    ("fp16x2_fft", "throughput", 64, 16, 3),    # k_score_tc: a chunk without MMAs or commit
])
def test_bounded_wait_expires_cleanly(bioem, mode, name, nq, max_shift, skip):
    import torch
    ctx, im, ps, s = _case(bioem, name, 16, nq, max_shift)
    ctx.set_precision(mode)
    try:
        want = bioem.score(ctx, im, ps, s).cpu().numpy()
        assert ctx.status() == 0
        ctx.set_wait_test(skip, 5_000_000)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bioem.score(ctx, im, ps, s)
        status = ctx.status()
        dt = time.perf_counter() - t0
        assert status == bioem.ERR_TIMEOUT, status
        assert dt < 1.0, dt          # every block gave up after its 5 ms waits
        # the context stays usable: the next launch is unarmed and scores as before
        again = bioem.score(ctx, im, ps, s).cpu().numpy()
        assert ctx.status() == 0
        np.testing.assert_array_equal(again, want)
    finally:
        ctx.set_precision("fp32")


def test_wait_test_arguments(bioem):
    ctx = bioem.Context(0)
    with pytest.raises(bioem.BioEMError):
        ctx.set_wait_test(2, 10)            # limit below 1 us
    with pytest.raises(bioem.BioEMError):
        ctx.set_wait_test(-2, 5_000_000)
    ctx.set_wait_test(-1, 0)                # disarm
