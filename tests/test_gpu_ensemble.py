"""GPU parity of bioem_ensemble (Eq. 10) against the oracle: ensemble posterior, per-model
posteriors and EM weights, on float64 and float32 matrices, plus the batched log P matrix."""
import numpy as np
import pytest

import oracle

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
def ctx(bioem):
    return bioem.Context(0)


@pytest.mark.parametrize("m,n,dtype", [(1, 7, "f64"), (3, 1000, "f64"), (8, 4097, "f64"), (64, 2500, "f32"),
                                       (5, 300, "f32")])
def test_ensemble_matches_oracle(bioem, ctx, m, n, dtype):
    import torch
    rng = np.random.default_rng(m * 1000 + n)
    lp = -8000.0 + 3.0 * rng.standard_normal((m, n))
    if dtype == "f32":
        lp = lp.astype(np.float32).astype(np.float64)   # the values the device sees
    w0 = rng.uniform(0.1, 1.0, m)
    t = torch.from_numpy(lp.astype(np.float32) if dtype == "f32" else lp).cuda()
    for n_iter in (0, 1, 25):
        out = bioem.ensemble(ctx, t, torch.from_numpy(w0).cuda(), n_iter=n_iter)
        assert ctx.status() == 0
        w_ref, hist = oracle.em_weights(lp, w0, n_iter)
        np.testing.assert_allclose(out["weights"].cpu().numpy(), w_ref, rtol=1e-9, atol=1e-12)
        assert abs(float(out["log_post"]) - hist[-1]) <= 1e-9 * abs(hist[-1])
        np.testing.assert_allclose(out["model_log_post"].cpu().numpy(), oracle.model_log_posteriors(lp),
                                   rtol=1e-12)


def test_zero_weights_and_errors(bioem, ctx):
    import torch
    lp = torch.zeros((2, 10), dtype=torch.float64, device="cuda")
    out = bioem.ensemble(ctx, lp, torch.tensor([0.0, 2.0], dtype=torch.float64, device="cuda"), n_iter=3)
    assert ctx.status() == 0
    np.testing.assert_allclose(out["weights"].cpu().numpy(), [0.0, 1.0])
    bioem.ensemble(ctx, lp, torch.tensor([0.0, 0.0], dtype=torch.float64, device="cuda"))
    assert ctx.status() == bioem.ERR_NUMERIC
    with pytest.raises(bioem.BioEMError) as e:
        bioem.ensemble(ctx, torch.zeros((600, 4), dtype=torch.float64, device="cuda"))
    assert e.value.code == bioem.ERR_INVALID_ARG


def test_deterministic(bioem, ctx):
    import torch
    rng = np.random.default_rng(9)
    t = torch.from_numpy(-100.0 + rng.standard_normal((16, 30000))).cuda()
    a = bioem.ensemble(ctx, t, n_iter=10)
    b = bioem.ensemble(ctx, t, n_iter=10)
    assert torch.equal(a["weights"], b["weights"]) and torch.equal(a["log_post"], b["log_post"])
