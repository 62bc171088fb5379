"""Forward model of a calculated image, float64 (test infrastructure only).

Steps of Fig. 1: rotate the model, project it, apply the PSF in Fourier space,
displace, scale and offset.  Image arrays are indexed [k, j] = [y, x]
(row-major, x fastest).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


def rotation_matrix(q) -> np.ndarray:
    """3x3 rotation of a quaternion q = (w, x, y, z) (Sec. 3.1).

    Reading (the paper names quaternions but no convention): Hamilton product,
    active rotation r' = R(q) r, q normalised first, so q and -q give the same R.
    """
    w, x, y, z = (float(v) for v in q)
    nrm = math.sqrt(w * w + x * x + y * y + z * z)
    w, x, y, z = w / nrm, x / nrm, y / nrm, z / nrm
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def pixel_centres(npix: int, pixel_A: float) -> np.ndarray:
    """Pixel-centre coordinates x_j = (j - npix/2) * pixel_A, j = 0..npix-1 (Eq. 1's x_j).

    Reading: 0-based indices with the box centre at pixel npix/2.
    """
    return (np.arange(npix) - npix // 2) * float(pixel_A)


def _pixel_integrals(centres: np.ndarray, pos: np.ndarray, sigma: float, pixel_A: float) -> np.ndarray:
    """G[a, j] = integral over pixel j of a unit 1-D Gaussian centred at pos[a]."""
    s = sigma * math.sqrt(2.0)
    hi = (centres[None, :] + pixel_A / 2 - pos[:, None]) / s
    lo = (centres[None, :] - pixel_A / 2 - pos[:, None]) / s
    return 0.5 * (erf(hi) - erf(lo))


def project(atoms, q, sigma_A: float, npix: int, pixel_A: float) -> np.ndarray:
    """Ideal projection I0[k, j] of Eq. 1 for a model of isotropic Gaussian atoms.

    rho(r) = sum_a w_a (2 pi sigma^2)^(-3/2) exp(-|r - R(q) r_a|^2 / (2 sigma^2)).
    The z integral leaves a 2-D Gaussian of mass w_a; the pixel integrals in x
    and y factorise into differences of erf.  All atoms are summed with no
    cutoff; mass outside the box is cropped (reading: the paper is silent).
    """
    atoms = np.asarray(atoms, dtype=np.float64)
    rot = rotation_matrix(q)
    xyz = atoms[:, :3] @ rot.T
    c = pixel_centres(npix, pixel_A)
    gx = _pixel_integrals(c, xyz[:, 0], sigma_A, pixel_A)
    gy = _pixel_integrals(c, xyz[:, 1], sigma_A, pixel_A)
    return (gy * atoms[:, 3:4]).T @ gx


def _dft_matrix(n: int, sign: float) -> np.ndarray:
    idx = np.arange(n)
    return np.exp(sign * 2j * math.pi * np.outer(idx, idx) / n)


def dft2(img: np.ndarray) -> np.ndarray:
    """Eq. 2: F(l, n) = sum_{j,k} I(j, k) exp(+2 pi i (l j / Nx + n k / Ny)), dense matrices.

    Reading: the printed exponent lacks the 1/Nx, 1/Ny factors (garbled); the
    indices are taken 0-based (a global phase only).  Result indexed [n, l].
    """
    ny, nx = img.shape
    return _dft_matrix(ny, +1.0) @ img @ _dft_matrix(nx, +1.0).T


def idft2(spec: np.ndarray) -> np.ndarray:
    """Eq. 3: I(j, k) = (1 / Npix) sum_{l,n} F(l, n) exp(-2 pi i (l j / Nx + n k / Ny))."""
    ny, nx = spec.shape
    return _dft_matrix(ny, -1.0) @ spec @ _dft_matrix(nx, -1.0).T / (nx * ny)


def electron_wavelength_A(voltage_kV: float) -> float:
    """Relativistic electron wavelength (A) at an accelerating voltage.

    lambda = h / sqrt(2 m0 e V (1 + e V / (2 m0 c^2))) = 12.2643 / sqrt(V (1 + 0.97845e-6 V)) A, V in volts.
    """
    v = voltage_kV * 1.0e3
    return 12.2643 / math.sqrt(v * (1.0 + 0.97845e-6 * v))


def ctf_coefficients(defocus_A: float, amp_contrast: float, bfactor_A2: float, voltage_kV: float):
    """(a, A, b) of the CTF/Env forms after Eq. 4, from physical parameters.

    Reading (the paper gives only a, A, b): with s = 2 pi k (k in 1/A), the
    defocus phase pi lambda df k^2 equals a s^2 / 2, so a = lambda df / (2 pi);
    the B-factor amplitude exp(-B k^2 / 4) equals exp(-b s^2 / 2), so
    b = B / (8 pi^2); A is the amplitude contrast.  No spherical aberration.
    """
    lam = electron_wavelength_A(voltage_kV)
    return lam * defocus_A / (2.0 * math.pi), float(amp_contrast), bfactor_A2 / (8.0 * math.pi ** 2)


def ctf_env(s2: np.ndarray, a: float, amp: float, b: float) -> np.ndarray:
    """CTF(s|a,A) Env(s|b) = (-A cos(a s^2/2) - sqrt(1-A^2) sin(a s^2/2)) exp(-b s^2/2) (after Eq. 4)."""
    ctf = -amp * np.cos(a * s2 / 2.0) - math.sqrt(1.0 - amp * amp) * np.sin(a * s2 / 2.0)
    return ctf * np.exp(-b * s2 / 2.0)


def frequency_s2(npix: int, pixel_A: float) -> np.ndarray:
    """|s|^2 on the [n, l] DFT grid, s = 2 pi (l / (Nx dx), n / (Ny dy)) (after Eq. 2).

    Reading: index l is taken as the signed frequency l - N for l > N/2 (the DFT
    is periodic); the Nyquist index N/2 enters as +N/2 (|s| depends on l^2 only).
    """
    idx = np.arange(npix)
    signed = np.where(idx <= npix // 2, idx, idx - npix).astype(np.float64)
    f = 2.0 * math.pi * signed / (npix * pixel_A)
    return f[:, None] ** 2 + f[None, :] ** 2


def apply_psf(img0: np.ndarray, ctf_row, pixel_A: float) -> np.ndarray:
    """I1 = F^-1[F(I0) CTF Env] (Eq. 5), real part of the dense inverse DFT.

    ctf_row = (defocus_A, amp_contrast, bfactor_A2, voltage_kV).
    """
    a, amp, b = ctf_coefficients(*ctf_row)
    spec = dft2(img0) * ctf_env(frequency_s2(img0.shape[0], pixel_A), a, amp, b)
    return idft2(spec).real


def synthesize_image(img1: np.ndarray, dx: int, dy: int, norm: float, offset: float,
                     noise: np.ndarray | None, snr: float) -> np.ndarray:
    """Observed image N I1(r + d) - mu + eps (Eq. 7 plus the Gaussian noise of Eq. 8).

    Shifts are cyclic: I1(r + d) at pixel (j, k) is I1[(k + dy) mod N, (j + dx) mod N].
    The noise level is lambda^2 = Var(N I1) / snr over the whole box (reading:
    the SNR definition is not in the paper); noise=None gives a noiseless image.
    """
    signal = norm * np.roll(img1, shift=(-dy, -dx), axis=(0, 1))
    out = signal - offset
    if noise is not None:
        out = out + math.sqrt(np.var(signal) / snr) * noise
    return out


def synthesize_images(wl: dict, indices=None, noiseless: bool = False) -> np.ndarray:
    """[n, N, N] float32 observed images for workload draws ``wl`` (from ``workloads.workload``)."""
    cfg = wl["config"]
    idx = range(len(wl["truth"])) if indices is None else indices
    out = []
    for i in idx:
        t = wl["truth"][i]
        img0 = project(wl["atoms"], t["quat"], cfg.sigma_A, cfg.npix, cfg.pixel_A)
        img1 = apply_psf(img0, (t["defocus_A"], t["amp_contrast"], t["bfactor"], t["voltage_kV"]), cfg.pixel_A)
        out.append(synthesize_image(img1, t["dx"], t["dy"], t["norm"], t["offset"],
                                    None if noiseless else wl["noise"][i], cfg.snr))
    return np.asarray(out, dtype=np.float32)
