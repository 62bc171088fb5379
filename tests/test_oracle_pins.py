"""Pins of the FP64 oracle against things other than itself (no GPU).

Each test fixes the oracle to a library routine, a brute-force computation, an
exact invariance of the method or a textbook value, chosen so that a dropped
term, a wrong sign, index or power, or a transposed operand fails one of them.
"""
import math
import os

import numpy as np
import pytest
import scipy.integrate
import scipy.special
import scipy.stats
from scipy.spatial.transform import Rotation

import oracle
import workloads

HERE = os.path.dirname(os.path.abspath(__file__))


# ---------------------------------------------------------------- closed form vs brute-force quadrature
def _quadrature_loglik(o: np.ndarray, c: np.ndarray) -> float:
    """ln of the integral of Eq. 8 over N, mu (real line) and lambda > 0, by brute-force quadrature.

    The integrand is evaluated literally from the residual sum; nodes are placed
    on the principal axes of the (numerically computed) least-squares problem,
    a change of variables that does not use the closed form.
    """
    o = o.ravel().astype(np.float64)
    c = c.ravel().astype(np.float64)
    n = o.size
    design = np.stack([c, -np.ones(n)], axis=1)          # I_cal = N c - mu
    theta0, *_ = np.linalg.lstsq(design, o, rcond=None)
    r0 = float(np.sum((o - design @ theta0) ** 2))
    hess = design.T @ design
    evals, evecs = np.linalg.eigh(hess)
    t, wt = np.polynomial.legendre.leggauss(96)
    t = 12.0 * t
    wt = 12.0 * wt
    t1, t2 = np.meshgrid(t, t, indexing="ij")
    w2 = np.log(np.outer(wt, wt)).ravel()
    unit = np.stack([t1.ravel(), t2.ravel()], axis=1)      # coordinates on principal axes
    lam_peak = math.sqrt(r0 / (n - 2))
    u = np.linspace(math.log(lam_peak) - 4.0, math.log(lam_peak) + 4.0, 4001)
    du = u[1] - u[0]
    logs = np.empty_like(u)
    for i, ui in enumerate(u):
        lam = math.exp(ui)
        scale = lam / np.sqrt(evals)
        theta = theta0[None, :] + (unit * scale[None, :]) @ evecs.T
        resid = o[None, :] - theta @ design.T
        rss = np.sum(resid * resid, axis=1)
        log_l = -rss / (2 * lam * lam) - (n / 2.0) * math.log(2 * math.pi * lam * lam)
        log_jac = float(np.sum(np.log(scale)))             # d(N, mu) = prod(scale) d(t1, t2)
        logs[i] = scipy.special.logsumexp(log_l + w2) + log_jac + ui   # d lambda = lambda du
    trap = np.full(u.size, math.log(du))
    trap[0] = trap[-1] = math.log(du / 2)
    return float(scipy.special.logsumexp(logs + trap))


@pytest.mark.parametrize("npix,seed", [(4, 1), (4, 2), (6, 3)])
def test_closed_form_matches_quadrature(npix, seed):
    rng = np.random.default_rng(seed)
    c = rng.standard_normal((npix, npix)) + 0.3
    o = 1.7 * c - 0.4 + 0.8 * rng.standard_normal((npix, npix))
    n = npix * npix
    c_o, c_oo = oracle.moments(o)
    c_c, c_cc = oracle.moments(c)
    c_co = float(np.sum(o * c))
    closed = float(oracle.closed_form_loglik(c_o, c_oo, c_c, c_cc, c_co, n))
    quad = _quadrature_loglik(o, c)
    assert abs(closed - quad) <= 1e-8 * max(1.0, abs(quad)), (closed, quad)


@pytest.mark.parametrize("n,seed", [(16, 4), (400, 5), (16384, 6)])
def test_closed_form_zero_mean_projection_special_case(n, seed):
    """With sum c = 0 the residual splits as sum (o' - N c)^2 + n (o_mean + mu)^2 (o' = o - o_mean),
    so the three integrals are textbook ones, at any image size (quadrature needs tiny n):
    mu gives sqrt(2 pi lambda^2 / n), N gives sqrt(2 pi lambda^2 / C_cc) with the minimum residual
    R = sum o'^2 - (sum o' c)^2 / C_cc, and int_0^inf lambda^(2-n) exp(-R / 2 lambda^2) d lambda =
    Gamma((n-3)/2) (R/2)^((3-n)/2) / 2."""
    rng = np.random.default_rng(seed)
    c = rng.standard_normal(n)
    c -= c.mean()
    o = 0.7 * c + 2.5 + rng.standard_normal(n)
    op = o - o.mean()
    c_cc = float(np.sum(c * c))
    r = float(np.sum(op * op) - np.sum(op * c) ** 2 / c_cc)
    want = ((1 - n / 2) * math.log(2 * math.pi) - 0.5 * math.log(n * c_cc) - math.log(2.0)
            + math.lgamma((n - 3) / 2) + (3 - n) / 2 * math.log(r / 2))
    c_o, c_oo = float(o.sum()), float(np.sum(o * o))
    got = float(oracle.closed_form_loglik(c_o, c_oo, float(c.sum()), c_cc, float(np.sum(o * c)), n))
    assert abs(got - want) <= 1e-9 * max(1.0, abs(want)), (got, want)


# ---------------------------------------------------------------- transforms and correlation
def test_dft_pair_matches_numpy():
    rng = np.random.default_rng(7)
    img = rng.standard_normal((12, 12))
    spec = oracle.dft2(img)
    # Eq. 2 uses exp(+2 pi i ...) without normalisation: numpy's inverse FFT times Npix.
    np.testing.assert_allclose(spec, np.fft.ifft2(img) * img.size, rtol=0, atol=1e-12 * np.abs(spec).max())
    spec2 = rng.standard_normal((12, 12)) + 1j * rng.standard_normal((12, 12))
    np.testing.assert_allclose(oracle.idft2(spec2), np.fft.fft2(spec2) / spec2.size, atol=1e-13)
    np.testing.assert_allclose(oracle.idft2(oracle.dft2(img)).real, img, atol=1e-12)


def test_correlation_direct_sum_matches_fft():
    rng = np.random.default_rng(11)
    o = rng.standard_normal((16, 16))
    cs = rng.standard_normal((3, 16, 16))
    s = 5
    got = oracle.correlation_all_shifts(o, cs, s)
    fo = np.fft.fft2(o)
    for p in range(3):
        cc = np.fft.ifft2(np.conj(fo) * np.fft.fft2(cs[p])).real   # sum_r o(r) c(r + d)
        want = np.array([cc[dy % 16, dx % 16] for dy, dx in oracle.shift_list(s)])
        np.testing.assert_allclose(got[p], want, rtol=1e-10, atol=1e-10 * np.abs(want).max())


def test_shift_list_order():
    sl = oracle.shift_list(2)
    assert sl.shape == (25, 2)
    assert list(sl[0]) == [-2, -2] and list(sl[1]) == [-2, -1] and list(sl[-1]) == [2, 2]


def test_parseval_projection_energy():
    wl = workloads.workload(workloads.get_config("tiny"), n_img=1)
    cfg = wl["config"]
    img0 = oracle.project(wl["atoms"], wl["quats"][0], cfg.sigma_A, cfg.npix, cfg.pixel_A)
    img1 = oracle.apply_psf(img0, wl["ctfs"][2], cfg.pixel_A)
    e_real = float(np.sum(img1 ** 2))
    e_fourier = float(np.sum(np.abs(oracle.dft2(img1)) ** 2)) / img1.size
    assert abs(e_real - e_fourier) <= 1e-12 * e_real


def test_logsumexp_matches_scipy():
    rng = np.random.default_rng(5)
    v = rng.standard_normal((7, 40)) * 300.0 - 1e5
    np.testing.assert_allclose(oracle.logsumexp(v, axis=1), scipy.special.logsumexp(v, axis=1), rtol=1e-15)
    assert abs(oracle.logsumexp(v) - scipy.special.logsumexp(v)) < 1e-9


# ---------------------------------------------------------------- geometry and projection
def test_rotation_matches_scipy():
    rng = np.random.default_rng(3)
    for _ in range(5):
        q = rng.standard_normal(4)
        q /= np.linalg.norm(q)
        ref = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()   # scipy: (x, y, z, w), active
        np.testing.assert_allclose(oracle.rotation_matrix(q), ref, atol=1e-14)
        np.testing.assert_allclose(oracle.rotation_matrix(-q), ref, atol=1e-14)
    # 90 degrees about z takes +x to +y
    q = np.array([math.cos(math.pi / 4), 0, 0, math.sin(math.pi / 4)])
    np.testing.assert_allclose(oracle.rotation_matrix(q) @ [1, 0, 0], [0, 1, 0], atol=1e-15)


def test_projection_mass_and_centre():
    atom = np.array([[0.0, 0.0, 0.0, 2.5]], dtype=np.float32)
    img0 = oracle.project(atom, [1, 0, 0, 0], 1.5, 32, 2.0)
    assert abs(img0.sum() - 2.5) < 1e-12
    assert np.unravel_index(np.argmax(img0), img0.shape) == (16, 16)


def test_projection_pixel_integrals_match_normal_cdf_and_quadrature():
    atom = np.array([[1.3, -2.1, 0.7, 1.0]], dtype=np.float32)
    q = np.array([0.9, 0.1, -0.3, 0.2])
    sigma, npix, dx = 1.5, 16, 2.0
    img0 = oracle.project(atom, q, sigma, npix, dx)
    pos = oracle.rotation_matrix(q) @ atom[0, :3].astype(np.float64)
    xc = (np.arange(npix) - npix // 2) * dx
    gx = scipy.stats.norm.cdf((xc + dx / 2 - pos[0]) / sigma) - scipy.stats.norm.cdf((xc - dx / 2 - pos[0]) / sigma)
    gy = scipy.stats.norm.cdf((xc + dx / 2 - pos[1]) / sigma) - scipy.stats.norm.cdf((xc - dx / 2 - pos[1]) / sigma)
    np.testing.assert_allclose(img0, np.outer(gy, gx), atol=1e-14)
    # one pixel by 2-D quadrature of the projected density (z already integrated: unit 2-D Gaussian)
    k, j = 7, 8
    dens = lambda y, x: math.exp(-((x - pos[0]) ** 2 + (y - pos[1]) ** 2) / (2 * sigma ** 2)) / (2 * math.pi * sigma ** 2)
    val, _ = scipy.integrate.dblquad(dens, xc[j] - dx / 2, xc[j] + dx / 2, xc[k] - dx / 2, xc[k] + dx / 2,
                                     epsabs=1e-13, epsrel=1e-12)
    assert abs(img0[k, j] - val) < 1e-11


# ---------------------------------------------------------------- CTF / physics
def test_electron_wavelength_textbook():
    rows = np.loadtxt(os.path.join(HERE, "golden", "electron_wavelength.txt"))
    for kv, nm in rows:
        got = oracle.electron_wavelength_A(kv) / 10.0
        assert abs(got - nm) <= 0.006 * nm + 5e-6, (kv, got, nm)


def test_ctf_matches_textbook_k_space_form():
    """The paper's s-space form with converted (a, b) equals the textbook form in k = 1/d units:
    CTF(k) = -(A cos chi + sqrt(1-A^2) sin chi), chi = pi lambda df k^2, amplitude envelope exp(-B k^2 / 4)."""
    df, amp, bfac, kv = 15000.0, 0.1, 80.0, 300.0
    lam = oracle.electron_wavelength_A(kv)
    k = np.linspace(0.0, 0.45, 200)
    chi = math.pi * lam * df * k ** 2
    want = -(amp * np.cos(chi) + math.sqrt(1 - amp ** 2) * np.sin(chi)) * np.exp(-bfac * k ** 2 / 4.0)
    a, amp2, b = oracle.ctf_coefficients(df, amp, bfac, kv)
    got = oracle.ctf_env((2 * math.pi * k) ** 2, a, amp2, b)
    np.testing.assert_allclose(got, want, atol=1e-12)
    # B-factor: amplitude at resolution d = 5 A with B = 100 A^2 is exp(-1)
    _, _, b = oracle.ctf_coefficients(df, 0.0, 100.0, kv)
    assert abs(math.exp(-b * (2 * math.pi / 5.0) ** 2 / 2) - math.exp(-1.0)) < 1e-15


def test_ctf_dc_term():
    """CTF(0) = -A and Env(0) = 1, so the PSF keeps -A times the projected mass: C_c = -A sum I0."""
    wl = workloads.workload(workloads.get_config("tiny"), n_img=1)
    cfg = wl["config"]
    img0 = oracle.project(wl["atoms"], wl["quats"][5], cfg.sigma_A, cfg.npix, cfg.pixel_A)
    for row in wl["ctfs"]:
        img1 = oracle.apply_psf(img0, row, cfg.pixel_A)
        assert abs(img1.sum() - (-row[1]) * img0.sum()) < 1e-10 * abs(img0.sum())
    s2 = oracle.frequency_s2(8, 1.0)
    assert s2[0, 0] == 0.0 and s2[4, 0] == s2[0, 4] == (2 * math.pi * 4 / 8) ** 2


# ---------------------------------------------------------------- invariances of the posterior
@pytest.fixture(scope="module")
def small_case():
    cfg = workloads.get_config("tiny", n_orient=8)
    wl = workloads.workload(cfg, n_img=3)
    imgs = oracle.synthesize_images(wl)
    ctfs = wl["ctfs"][[0, 5]]
    base = oracle.score(imgs, wl["atoms"], wl["quats"], ctfs, cfg.sigma_A, cfg.pixel_A, 2)
    return cfg, wl, imgs, ctfs, base


def test_invariance_offset(small_case):
    cfg, wl, imgs, ctfs, base = small_case
    r = oracle.score(imgs.astype(np.float64) + 3.7, wl["atoms"], wl["quats"], ctfs, cfg.sigma_A, cfg.pixel_A, 2)
    np.testing.assert_allclose(r["logP"], base["logP"], rtol=1e-11)


def test_invariance_image_scale(small_case):
    cfg, wl, imgs, ctfs, base = small_case
    n = cfg.npix ** 2
    r = oracle.score(imgs.astype(np.float64) * 2.5, wl["atoms"], wl["quats"], ctfs, cfg.sigma_A, cfg.pixel_A, 2)
    np.testing.assert_allclose(r["logP"], base["logP"] - (n - 3) * math.log(2.5), rtol=1e-11)


def test_invariance_projection_scale_and_quaternion_sign(small_case):
    cfg, wl, imgs, ctfs, base = small_case
    atoms = wl["atoms"].copy()
    atoms[:, 3] *= 3.0
    r = oracle.score(imgs, atoms, -wl["quats"], ctfs, cfg.sigma_A, cfg.pixel_A, 2)
    np.testing.assert_allclose(r["logP"], base["logP"] - math.log(3.0), rtol=1e-11)
    assert [b[:4] for b in r["best"]] == [b[:4] for b in base["best"]]


# ---------------------------------------------------------------- recovery of the truth
@pytest.mark.parametrize("noisy", [False, True])
def test_recovers_true_grid_point_and_shift(noisy):
    cfg = workloads.get_config("tiny", n_orient=24, snr=50.0)
    wl = workloads.workload(cfg, n_img=4)
    quats, ctfs = wl["quats"], wl["ctfs"]
    truth = [(3, 1, -2, 4), (17, 4, 3, -1), (0, 5, 0, 0), (23, 2, -4, -4)]
    imgs = []
    for i, (iq, ic, dy, dx) in enumerate(truth):
        img0 = oracle.project(wl["atoms"], quats[iq], cfg.sigma_A, cfg.npix, cfg.pixel_A)
        img1 = oracle.apply_psf(img0, ctfs[ic], cfg.pixel_A)
        imgs.append(oracle.synthesize_image(img1, dx, dy, 1.3, 0.4, wl["noise"][i] if noisy else None, cfg.snr))
    r = oracle.score(np.array(imgs), wl["atoms"], quats, ctfs, cfg.sigma_A, cfg.pixel_A, cfg.max_shift)
    assert [b[:4] for b in r["best"]] == truth


def test_posterior_outputs_consistent(small_case):
    cfg, wl, imgs, ctfs, base = small_case
    n_ctf, s = len(ctfs), 25
    n_q = base["logP_orient"].shape[1]
    # log P is the log-mean over orientations of the per-orientation posteriors
    np.testing.assert_allclose(oracle.logsumexp(base["logP_orient"], axis=1) - math.log(n_q), base["logP"], rtol=1e-13)
    np.testing.assert_allclose(oracle.logsumexp(base["pair_lse"], axis=1) - math.log(n_ctf * n_q * s),
                               base["logP"], rtol=1e-13)
    for w, b in enumerate(base["best"]):
        assert abs(b[4] - base["pair_max"][w].max()) < 1e-9 * abs(b[4])


# ---------------------------------------------------------------- stored regression values
def test_tiny_logp_regression():
    path = os.path.join(HERE, "golden", "tiny_logP.txt")
    want = np.loadtxt(path)
    cfg = workloads.get_config("tiny")
    wl = workloads.workload(cfg, n_img=len(want))
    imgs = oracle.synthesize_images(wl)
    r = oracle.score(imgs, wl["atoms"], wl["quats"], wl["ctfs"], cfg.sigma_A, cfg.pixel_A, cfg.max_shift)
    np.testing.assert_allclose(r["logP"], want, rtol=1e-12)
