"""Marginal likelihood and grid posterior, float64 (test infrastructure only).

Notation: n = Npix; o an observed image; c = I1 a PSF-filtered projection.
Moments C_o = sum o, C_oo = sum o^2, C_c = sum c, C_cc = sum c^2 and, for a
displacement d, C_co(d) = sum_r o(r) c((r + d) mod N) (the correlation the
Fourier variant of Sec. 3.3 evaluates; cyclic, Sec. 3.3).
"""
from __future__ import annotations

import math

import numpy as np

from .forward import apply_psf, project


def shift_list(max_shift: int) -> np.ndarray:
    """[(2s+1)^2, 2] int (dy, dx), dy-major ascending, so index order is lexicographic in (dy, dx)."""
    r = np.arange(-max_shift, max_shift + 1)
    dy, dx = np.meshgrid(r, r, indexing="ij")
    return np.stack([dy.ravel(), dx.ravel()], axis=1)


def moments(img: np.ndarray) -> tuple[float, float]:
    """(sum x, sum x^2) over all pixels, float64."""
    x = np.asarray(img, dtype=np.float64)
    return float(x.sum()), float((x * x).sum())


def correlation_all_shifts(img: np.ndarray, projs: np.ndarray, max_shift: int) -> np.ndarray:
    """C_co[p, d] = sum_r o(r) c_p((r + d) mod N) for every listed displacement d, as a direct sum.

    Relabelling the summation index r -> r - d (cyclic) gives
    C_co(d) = sum_r o((r - d) mod N) c_p(r): one row per d holding the image
    rolled by d, multiplied against every projection (a matmul serves as the
    sum over r; nothing else is reordered).
    """
    img = np.asarray(img, dtype=np.float64)
    rolled = np.stack([np.roll(img, shift=(int(dy), int(dx)), axis=(0, 1)).ravel()
                       for dy, dx in shift_list(max_shift)])
    flat = np.asarray(projs, dtype=np.float64).reshape(len(projs), -1)
    return flat @ rolled.T


def log_norm_constant(n: int) -> float:
    """c(n) = -ln 2 + (1 - n/2) ln 2 pi + ln Gamma((n-3)/2) + (n-3)/2 ln(2n)."""
    return (-math.log(2.0) + (1.0 - n / 2.0) * math.log(2.0 * math.pi)
            + math.lgamma((n - 3) / 2.0) + (n - 3) / 2.0 * math.log(2.0 * n))


def closed_form_loglik(c_o, c_oo, c_c, c_cc, c_co, n: int):
    """ln of Eq. 8 integrated over N in R, mu in R and lambda in (0, inf) with unit flat priors.

    The paper defers this closed form to its supplement; it is derived here from
    Eq. 8.  With R(N, mu) = sum (o - N c + mu)^2, the Gaussian integrals over N
    and mu give (2 pi)^(1 - n/2) lambda^(2-n) B^(-1/2) exp(-R_min / 2 lambda^2),
    R_min = D / (n B), and int_0^inf lambda^(2-n) exp(-R / 2 lambda^2) d lambda
    = Gamma((n-3)/2) (R/2)^((3-n)/2) / 2, so
        ln L = (3-n)/2 ln D + (n-4)/2 ln B + c(n),
    A = n C_oo - C_o^2, B = n C_cc - C_c^2, X = n C_co - C_o C_c, D = A B - X^2.
    Readings: flat unit priors on N, mu, lambda (the priors are in the absent
    supplement); N ranges over the whole real line.  D is floored at 1e-300 A B.
    """
    a = n * c_oo - c_o * c_o
    b = n * np.asarray(c_cc, dtype=np.float64) - np.asarray(c_c, dtype=np.float64) ** 2
    x = n * np.asarray(c_co, dtype=np.float64) - c_o * np.asarray(c_c, dtype=np.float64)
    d = np.maximum(a * b - x * x, 1.0e-300 * a * b)
    return (3 - n) / 2.0 * np.log(d) + (n - 4) / 2.0 * np.log(b) + log_norm_constant(n)


def logsumexp(v, axis=None):
    """ln sum exp v, shifted by the maximum."""
    v = np.asarray(v, dtype=np.float64)
    m = np.max(v, axis=axis, keepdims=True)
    out = m + np.log(np.sum(np.exp(v - m), axis=axis, keepdims=True))
    return np.squeeze(out, axis=axis) if axis is not None else float(out.ravel()[0])


def projections(atoms, quats, ctfs, sigma_A: float, npix: int, pixel_A: float) -> np.ndarray:
    """I1 for every parameter set p = q * n_ctf + ctf (rotate, project, PSF), [n_ps, N, N] float64."""
    out = np.empty((len(quats) * len(ctfs), npix, npix))
    for iq, q in enumerate(quats):
        img0 = project(atoms, q, sigma_A, npix, pixel_A)
        for ic, row in enumerate(ctfs):
            out[iq * len(ctfs) + ic] = apply_psf(img0, row, pixel_A)
    return out


def score(images, atoms, quats, ctfs, sigma_A: float, pixel_A: float, max_shift: int,
          projs: np.ndarray | None = None) -> dict:
    """Posterior of every image over the grid quats x ctfs x displacements (Eq. 9, Listing 1).

    Returns, per image w:
      logP[w]           = ln sum_{p,d} L(w | p, d) - ln(n_ps S)   (uniform weights over the grid;
                          reading: the prior weights are in the absent supplement)
      logP_orient[w, q] = ln sum_{ctf,d} L(w | q, ctf, d) - ln(n_ctf S)
      pair_max[w, p]    = max_d ln L,  pair_lse[w, p] = ln sum_d L
      best[w]           = (q, ctf, dy, dx, ln L) at the maximum; ties go to the lowest (q, ctf, dy, dx).
    """
    images = np.asarray(images, dtype=np.float64)
    n_img, npix, _ = images.shape
    n = npix * npix
    n_ctf = len(ctfs)
    if projs is None:
        projs = projections(atoms, quats, ctfs, sigma_A, npix, pixel_A)
    n_ps = projs.shape[0]
    n_q = n_ps // n_ctf
    c_c = projs.reshape(n_ps, -1).sum(axis=1)
    c_cc = (projs.reshape(n_ps, -1) ** 2).sum(axis=1)
    shifts = shift_list(max_shift)
    s_count = len(shifts)
    out = {
        "logP": np.empty(n_img),
        "logP_orient": np.empty((n_img, n_q)),
        "pair_max": np.empty((n_img, n_ps)),
        "pair_lse": np.empty((n_img, n_ps)),
        "best": [],
    }
    for w in range(n_img):
        c_o, c_oo = moments(images[w])
        c_co = correlation_all_shifts(images[w], projs, max_shift)
        lnl = closed_form_loglik(c_o, c_oo, c_c[:, None], c_cc[:, None], c_co, n)  # [n_ps, S]
        out["logP"][w] = logsumexp(lnl) - math.log(n_ps * s_count)
        out["logP_orient"][w] = logsumexp(lnl.reshape(n_q, n_ctf * s_count), axis=1) - math.log(n_ctf * s_count)
        out["pair_max"][w] = lnl.max(axis=1)
        out["pair_lse"][w] = logsumexp(lnl, axis=1)
        k = int(np.argmax(lnl))  # first maximum in (p, d) order = lowest (q, ctf, dy, dx)
        p, d = divmod(k, s_count)
        out["best"].append((p // n_ctf, p % n_ctf, int(shifts[d, 0]), int(shifts[d, 1]), float(lnl.flat[k])))
    return out
