"""ln(1 - rho^2) as the scoring kernels evaluate it (bioem_ln1m), against float64 log1p and against
the CUDA library's log1pf (torch.log1p on a CUDA tensor), over the whole range 0 <= x < 1: a
geometric sweep down to 1e-30, a dense sweep across the switch at x = 1/32, the switch point itself
and its float32 neighbours, and x = 0.  The series branch must stay within 2 float32 ulp of the exact
value (its truncation error is below 6e-9 relative), the library branch within the library's bound.
"""
import numpy as np
import pytest

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


def _grid():
    sw = np.float32(1.0 / 32.0)
    pts = [np.geomspace(1e-30, 0.999, 200_000),
           np.linspace(0.0, 0.0625, 200_001),
           np.linspace(0.0625, 1.0 - 2.0 ** -24, 100_001),
           [0.0, sw, np.nextafter(sw, np.float32(0)), np.nextafter(sw, np.float32(1)), 1.0 - 2.0 ** -24]]
    return np.concatenate([np.asarray(p, dtype=np.float64) for p in pts]).astype(np.float32)


def test_ln1m_within_two_ulp(bioem):
    import torch
    ctx = bioem.Context(0)
    x = _grid()
    got = bioem.ln1m(ctx, torch.from_numpy(x).cuda()).cpu().numpy()
    assert ctx.status() == 0
    exact = np.log1p(-x.astype(np.float64))
    ulp = np.spacing(np.abs(exact).astype(np.float32)).astype(np.float64)
    err = np.abs(got.astype(np.float64) - exact) / np.where(ulp > 0, ulp, 1.0)
    small = x <= np.float32(1.0 / 32.0)
    assert got[x == 0].tolist() == [0.0] * int((x == 0).sum())
    assert err[small].max() <= 2.0, float(err[small].max())
    assert err[~small].max() <= 2.0, float(err[~small].max())
    # and against CUDA's own log1pf on the same inputs
    lib_t = torch.log1p(-torch.from_numpy(x).cuda()).cpu().numpy()
    d = np.abs(got.astype(np.float64) - lib_t.astype(np.float64)) / np.where(ulp > 0, ulp, 1.0)
    assert d.max() <= 3.0, float(d.max())
