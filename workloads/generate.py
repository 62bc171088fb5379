"""Seeded draws and parameter grids (no method arithmetic).

Every draw uses numpy's PCG64 through a SeedSequence whose spawn key names the
stream (atoms, grid, image i truth, image i noise), so image i of a config is
the same whether 16 or 2048 images are generated.
"""
from __future__ import annotations

import math

import numpy as np

from .configs import Config

_STREAM_ATOMS = 1
_STREAM_GRID = 2
_STREAM_TRUTH = 3
_STREAM_NOISE = 4


def _rng(seed: int, *key: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed, spawn_key=tuple(key))))


def atoms_in_ball(n_atoms: int, radius_A: float, seed: int, weight: float = 1.0) -> np.ndarray:
    """[n_atoms, 4] float32 (x, y, z, w): points uniform in a ball of the given radius (A)."""
    rng = _rng(seed, _STREAM_ATOMS)
    g = rng.standard_normal((n_atoms, 3))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    r = radius_A * rng.random(n_atoms) ** (1.0 / 3.0)
    out = np.empty((n_atoms, 4), dtype=np.float64)
    out[:, :3] = g * r[:, None]
    out[:, 3] = weight
    return out.astype(np.float32)


def random_quaternions(n: int, rng: np.random.Generator) -> np.ndarray:
    """[n, 4] float64 unit quaternions (w, x, y, z), uniform on SO(3) (normalised 4-D Gaussian)."""
    g = rng.standard_normal((n, 4))
    return g / np.linalg.norm(g, axis=1, keepdims=True)


# --- HEALPix nested pixel centres (Gorski et al. 2005), restated from the scheme's definition ---
_JRLL = np.array([2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4], dtype=np.int64)
_JPLL = np.array([1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7], dtype=np.int64)


def _compress_bits(v: np.ndarray) -> np.ndarray:
    """Keep the even-position bits of v, packed together."""
    out = np.zeros_like(v)
    for b in range(32):
        out |= ((v >> (2 * b)) & 1) << b
    return out


def healpix_nest_pix2ang(nside: int, ipix: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Centres (theta, phi) of HEALPix pixels in the NESTED numbering."""
    ipix = np.asarray(ipix, dtype=np.int64)
    npface = nside * nside
    face = ipix // npface
    ipf = ipix % npface
    ix = _compress_bits(ipf)
    iy = _compress_bits(ipf >> 1)
    jr = _JRLL[face] * nside - (ix + iy) - 1
    nr = np.where(jr < nside, jr, np.where(jr > 3 * nside, 4 * nside - jr, nside))
    z = np.where(jr < nside, 1.0 - nr.astype(np.float64) ** 2 / (3.0 * npface),
                 np.where(jr > 3 * nside, -(1.0 - nr.astype(np.float64) ** 2 / (3.0 * npface)),
                          (2 * nside - jr) * 2.0 / (3.0 * nside)))
    kshift = np.where((jr >= nside) & (jr <= 3 * nside), (jr - nside) & 1, 0)
    jp = (_JPLL[face] * nr + (ix - iy) + 1 + kshift) // 2
    jp = np.where(jp > 4 * nr, jp - 4 * nr, jp)
    jp = np.where(jp < 1, jp + 4 * nr, jp)
    phi = (jp - (kshift + 1) * 0.5) * (0.5 * math.pi / nr)
    theta = np.arccos(np.clip(z, -1.0, 1.0))
    return theta, phi


def _spread_bits(v: np.ndarray) -> np.ndarray:
    """Place the bits of v on the even bit positions."""
    out = np.zeros_like(v)
    for b in range(32):
        out |= ((v >> b) & 1) << (2 * b)
    return out


def healpix_nest_ang2pix(nside: int, theta: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """NESTED HEALPix pixel containing each direction (Gorski et al. 2005), inverse of pix2ang."""
    z = np.cos(np.asarray(theta, dtype=np.float64))
    za = np.abs(z)
    tt = np.mod(np.asarray(phi, dtype=np.float64), 2.0 * math.pi) * (2.0 / math.pi)   # in [0, 4)
    ipix = np.empty(z.shape, dtype=np.int64)
    eq = za <= 2.0 / 3.0
    # equatorial region
    t1 = nside * (0.5 + tt[eq])
    t2 = nside * z[eq] * 0.75
    jp = (t1 - t2).astype(np.int64)
    jm = (t1 + t2).astype(np.int64)
    ifp, ifm = jp // nside, jm // nside
    face = np.where(ifp == ifm, ifp | 4, np.where(ifp < ifm, ifp, ifm + 8))
    ix = jm & (nside - 1)
    iy = nside - (jp & (nside - 1)) - 1
    ipix[eq] = face * nside * nside + _spread_bits(ix) + (_spread_bits(iy) << 1)
    # polar caps
    pc = ~eq
    ntt = np.minimum(3, tt[pc].astype(np.int64))
    tp = tt[pc] - ntt
    tmp = nside * np.sqrt(3.0 * (1.0 - za[pc]))
    jp = np.minimum((tp * tmp).astype(np.int64), nside - 1)
    jm = np.minimum(((1.0 - tp) * tmp).astype(np.int64), nside - 1)
    north = z[pc] >= 0
    face = np.where(north, ntt, ntt + 8)
    ix = np.where(north, nside - jm - 1, jp)
    iy = np.where(north, nside - jp - 1, jm)
    ipix[pc] = face * nside * nside + _spread_bits(ix) + (_spread_bits(iy) << 1)
    return ipix


def hopf_cell(level: int, quats: np.ndarray) -> np.ndarray:
    """Index of the Hopf-grid cell (level) containing each unit quaternion (w, x, y, z); q and -q agree.

    Inverts q = (cos(t/2) cos(p/2), cos(t/2) sin(p/2), sin(t/2) cos(f + p/2), sin(t/2) sin(f + p/2)):
    t = 2 atan2(|(y, z)|, |(w, x)|), psi = 2 atan2(x, w) mod 2 pi, phi = atan2(z, y) - psi/2 mod 2 pi.
    """
    q = np.asarray(quats, dtype=np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    # sign convention: the half angle psi/2 = atan2(x, w) in [0, pi) (q -> -q shifts it by pi)
    half = np.arctan2(q[:, 1], q[:, 0])
    q = np.where(((half < 0.0) | (half >= math.pi))[:, None], -q, q)
    half = np.mod(np.arctan2(q[:, 1], q[:, 0]), math.pi)
    theta = 2.0 * np.arctan2(np.hypot(q[:, 2], q[:, 3]), np.hypot(q[:, 0], q[:, 1]))
    psi = 2.0 * half
    phi = np.mod(np.arctan2(q[:, 3], q[:, 2]) - half, 2.0 * math.pi)
    nside = 2 ** level
    n_psi = 6 * 2 ** level
    pix = healpix_nest_ang2pix(nside, theta, phi)
    k = np.minimum((psi / (2.0 * math.pi) * n_psi).astype(np.int64), n_psi - 1)
    return pix * n_psi + k


def hopf_children(coarse_level: int, fine_level: int, coarse_index: np.ndarray) -> np.ndarray:
    """[n, 8**(fine - coarse)] fine-grid indices of the cells nested in each coarse cell."""
    d = fine_level - coarse_level
    n_psi_c, n_psi_f = 6 * 2 ** coarse_level, 6 * 2 ** fine_level
    c = np.asarray(coarse_index, dtype=np.int64)
    pix, k = c // n_psi_c, c % n_psi_c
    sub_pix = (pix[:, None] << (2 * d)) + np.arange(4 ** d)[None, :]          # [n, 4^d]
    sub_k = (k[:, None] << d) + np.arange(2 ** d)[None, :]                      # [n, 2^d]
    return (sub_pix[:, :, None] * n_psi_f + sub_k[:, None, :]).reshape(len(c), -1)


def hopf_grid(level: int) -> np.ndarray:
    """[72 * 8**level, 4] float64 unit quaternions of the Hopf-fibration grid (Yershova et al. 2010).

    S^2 part: HEALPix nested pixel centres at nside = 2**level; circle part: 6 * 2**level
    equally spaced angles psi_k = (k + 1/2) * 2 pi / n_psi.  Index = pixel * n_psi + k, so a
    level-L point's level-l parent (l < L) is (pixel >> 2(L - l)) * n_psi(l) + (k >> (L - l)).
    """
    nside = 2 ** level
    n_psi = 6 * 2 ** level
    theta, phi = healpix_nest_pix2ang(nside, np.arange(12 * nside * nside))
    psi = (np.arange(n_psi) + 0.5) * (2.0 * math.pi / n_psi)
    th = theta[:, None]
    ph = phi[:, None]
    ps = psi[None, :]
    q = np.stack([np.cos(th / 2) * np.cos(ps / 2),
                  np.cos(th / 2) * np.sin(ps / 2),
                  np.sin(th / 2) * np.cos(ph + ps / 2),
                  np.sin(th / 2) * np.sin(ph + ps / 2)], axis=-1)
    return q.reshape(-1, 4)


def hopf_coarse_index(fine_level: int, coarse_level: int, fine_index: np.ndarray) -> np.ndarray:
    """Index in the coarse Hopf grid of the cell containing each fine-grid point."""
    d = fine_level - coarse_level
    n_psi_f = 6 * 2 ** fine_level
    n_psi_c = 6 * 2 ** coarse_level
    fine_index = np.asarray(fine_index, dtype=np.int64)
    pix, k = fine_index // n_psi_f, fine_index % n_psi_f
    return (pix >> (2 * d)) * n_psi_c + (k >> d)


def nearest_orientations(grid: np.ndarray, q: np.ndarray, k: int) -> np.ndarray:
    """Indices of the k grid quaternions closest to q (largest |<g, q>|: q and -q are one
    orientation), closest first.  Picks the "truth neighbourhood" of a synthetic image on a grid."""
    dots = np.abs(np.asarray(grid, dtype=np.float64) @ np.asarray(q, dtype=np.float64))
    idx = np.argpartition(-dots, k - 1)[:k]
    return idx[np.argsort(-dots[idx], kind="stable")]


def defocus_grid(n: int, lo_um: float, hi_um: float) -> np.ndarray:
    """n defocus values (A), evenly spaced over [lo, hi] um, endpoints included."""
    return np.linspace(lo_um, hi_um, n) * 1.0e4


def ctf_grid(cfg: Config) -> np.ndarray:
    """[n_ctf, 4] float64 rows (defocus_A, amp_contrast, bfactor_A2, voltage_kV); defocus-major."""
    rows = []
    for df in defocus_grid(cfg.n_defocus, *cfg.defocus_range_um):
        for b in cfg.bfactors:
            rows.append((df, cfg.amp_contrast, b, cfg.voltage_kV))
    return np.array(rows, dtype=np.float64)


def orientation_grid(cfg: Config) -> np.ndarray:
    """[n_quat, 4] float32 quaternions of the scoring grid."""
    if cfg.orient == "random":
        seed = cfg.grid_seed if cfg.grid_seed is not None else cfg.seed
        return random_quaternions(cfg.n_orient, _rng(seed, _STREAM_GRID)).astype(np.float32)
    return hopf_grid(cfg.hopf_level).astype(np.float32)


def image_truth(cfg: Config, i: int) -> dict:
    """True parameters of synthetic image i: quaternion, integer shift, N, mu, defocus, B."""
    rng = _rng(cfg.seed, _STREAM_TRUTH, i)
    q = random_quaternions(1, rng)[0].astype(np.float32)
    s = cfg.max_shift
    dx, dy = (int(v) for v in rng.integers(-s, s + 1, size=2))
    return {
        "quat": q,
        "dx": dx,
        "dy": dy,
        "norm": float(rng.uniform(*cfg.norm_range)),
        "offset": float(rng.uniform(*cfg.offset_range)),
        "defocus_A": float(rng.uniform(*cfg.defocus_range_um) * 1.0e4),
        "bfactor": float(rng.uniform(*cfg.bfactor_range)),
        "amp_contrast": cfg.amp_contrast,
        "voltage_kV": cfg.voltage_kV,
    }


def standard_normal_noise(cfg: Config, i: int) -> np.ndarray:
    """[npix, npix] float64 standard-normal field for image i (scaled by the noise level later)."""
    return _rng(cfg.seed, _STREAM_NOISE, i).standard_normal((cfg.npix, cfg.npix))


def workload(cfg: Config, n_img: int | None = None) -> dict:
    """All seeded inputs of a config: atoms, grid quaternions, CTF rows, per-image truth and noise."""
    n = cfg.n_img if n_img is None else n_img
    return {
        "config": cfg,
        "atoms": atoms_in_ball(cfg.n_atoms, cfg.radius_A, cfg.seed, cfg.atom_weight),
        "quats": orientation_grid(cfg),
        "ctfs": ctf_grid(cfg),
        "truth": [image_truth(cfg, i) for i in range(n)],
        "noise": [standard_normal_noise(cfg, i) for i in range(n)],
    }
