"""Seeded input generators: HEALPix / Hopf grids and draw stability (no GPU)."""
import math

import numpy as np

import workloads
from workloads.generate import healpix_nest_pix2ang


def test_healpix_base_pixels():
    """Nside = 1: four pixels centred at z = 2/3, four on the equator, four at z = -2/3."""
    th, ph = healpix_nest_pix2ang(1, np.arange(12))
    z = np.cos(th)
    np.testing.assert_allclose(z, [2 / 3] * 4 + [0] * 4 + [-2 / 3] * 4, atol=1e-15)
    np.testing.assert_allclose(ph[:4], np.array([1, 3, 5, 7]) * math.pi / 4, atol=1e-15)
    np.testing.assert_allclose(ph[4:8], np.array([0, 1, 2, 3]) * math.pi / 2, atol=1e-15)


def test_healpix_rings_equal_area():
    """Rings: polar ring i has 4i pixels at z = 1 - i^2/(3 nside^2); equatorial rings 4 nside pixels."""
    nside = 4
    th, ph = healpix_nest_pix2ang(nside, np.arange(12 * nside * nside))
    z = np.round(np.cos(th), 12)
    vals, counts = np.unique(z, return_counts=True)
    want = {}
    for i in range(1, nside):
        want[round(1 - i * i / (3 * nside * nside), 12)] = 4 * i
        want[round(-(1 - i * i / (3 * nside * nside)), 12)] = 4 * i
    for i in range(nside, 3 * nside + 1):
        want[round(4 / 3 - 2 * i / (3 * nside), 12)] = 4 * nside
    assert dict(zip(vals.tolist(), counts.tolist())) == want
    v = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], 1)
    assert len(np.unique(np.round(v, 9), axis=0)) == len(v)
    assert np.abs(v.mean(axis=0)).max() < 1e-12


def test_healpix_nesting():
    """The four nested children of a pixel surround it: their mean direction is near the parent centre."""
    th_p, ph_p = healpix_nest_pix2ang(4, np.arange(192))
    th_c, ph_c = healpix_nest_pix2ang(8, np.arange(768))
    vp = np.stack([np.sin(th_p) * np.cos(ph_p), np.sin(th_p) * np.sin(ph_p), np.cos(th_p)], 1)
    vc = np.stack([np.sin(th_c) * np.cos(ph_c), np.sin(th_c) * np.sin(ph_c), np.cos(th_c)], 1)
    m = vc.reshape(192, 4, 3).mean(axis=1)
    m /= np.linalg.norm(m, axis=1, keepdims=True)
    ang = np.arccos(np.clip(np.sum(m * vp, axis=1), -1, 1))
    pixel_size = math.sqrt(4 * math.pi / 192)
    assert ang.max() < 0.1 * pixel_size


def _rot_dist(qa, qb):
    return 2 * np.arccos(np.clip(np.abs(qa @ qb.T), 0, 1))


def test_hopf_grid_counts_and_uniformity():
    for level, n in [(0, 72), (1, 576), (2, 4608)]:
        q = workloads.hopf_grid(level)
        assert q.shape == (n, 4)
        np.testing.assert_allclose(np.linalg.norm(q, axis=1), 1.0, atol=1e-14)
        # second moment of a uniform distribution on SO(3) (q ~ -q): E[q q^T] = I / 4
        np.testing.assert_allclose(q.T @ q / n, np.eye(4) / 4, atol=0.02 if level == 0 else 0.005)
    q = workloads.hopf_grid(1)
    d = _rot_dist(q, q)
    np.fill_diagonal(d, np.inf)
    assert d.min() > 0.05   # distinct rotations


def test_hopf_coarse_parent_cells():
    """A fine point's coarse cell: its S^2 pixel is nested in the coarse pixel and its psi in the coarse psi bin.

    (Cells are products of a HEALPix pixel and a psi interval in Hopf coordinates; near the poles they are
    elongated on SO(3), so nearness is checked on S^2 and on the circle separately.)
    """
    fine_l, coarse_l = 2, 1
    fine = np.arange(72 * 8 ** fine_l)
    parent = workloads.hopf_coarse_index(fine_l, coarse_l, fine)
    assert np.all(np.bincount(parent) == 8)
    n_psi_f, n_psi_c = 6 * 2 ** fine_l, 6 * 2 ** coarse_l
    pix_f, k_f = fine // n_psi_f, fine % n_psi_f
    pix_c, k_c = parent // n_psi_c, parent % n_psi_c
    psi_f = (k_f + 0.5) * 2 * math.pi / n_psi_f
    assert np.all(np.abs(psi_f - (k_c + 0.5) * 2 * math.pi / n_psi_c) <= math.pi / n_psi_c + 1e-12)
    th_f, ph_f = healpix_nest_pix2ang(2 ** fine_l, pix_f)
    th_c, ph_c = healpix_nest_pix2ang(2 ** coarse_l, pix_c)
    vf = np.stack([np.sin(th_f) * np.cos(ph_f), np.sin(th_f) * np.sin(ph_f), np.cos(th_f)], 1)
    vc = np.stack([np.sin(th_c) * np.cos(ph_c), np.sin(th_c) * np.sin(ph_c), np.cos(th_c)], 1)
    ang = np.arccos(np.clip(np.sum(vf * vc, axis=1), -1, 1))
    assert ang.max() < math.sqrt(4 * math.pi / (12 * 4 ** coarse_l))


def test_draws_stable_under_subsetting():
    cfg = workloads.get_config("tiny")
    a = workloads.workload(cfg, n_img=3)
    b = workloads.workload(cfg, n_img=6)
    for i in range(3):
        assert a["truth"][i]["dx"] == b["truth"][i]["dx"]
        np.testing.assert_array_equal(a["noise"][i], b["noise"][i])
        np.testing.assert_array_equal(a["truth"][i]["quat"], b["truth"][i]["quat"])
    np.testing.assert_array_equal(a["atoms"], b["atoms"])
    assert a["ctfs"].shape == (6, 4) and a["quats"].shape == (1152, 4)
    p = workloads.get_config("precision64")
    assert np.array_equal(workloads.workload(p, 1)["quats"], a["quats"])   # reuses the tiny grid


def test_healpix_ang2pix_inverts_pix2ang():
    from workloads.generate import healpix_nest_ang2pix
    for nside in (1, 2, 4, 16):
        pix = np.arange(12 * nside * nside)
        th, ph = healpix_nest_pix2ang(nside, pix)
        np.testing.assert_array_equal(healpix_nest_ang2pix(nside, th, ph), pix)
    # random directions land in the pixel whose children (next level) contain them
    rng = np.random.default_rng(0)
    v = rng.standard_normal((2000, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    th, ph = np.arccos(v[:, 2]), np.arctan2(v[:, 1], v[:, 0])
    np.testing.assert_array_equal(healpix_nest_ang2pix(8, th, ph) >> 2, healpix_nest_ang2pix(4, th, ph))
    # equal areas: uniform directions fill the 192 pixels evenly
    counts = np.bincount(healpix_nest_ang2pix(4, th, ph), minlength=192)
    assert counts.min() > 0 and counts.max() < 3 * 2000 / 192


def test_hopf_cell_and_children():
    for level in (0, 1, 2):
        q = workloads.hopf_grid(level)
        np.testing.assert_array_equal(workloads.hopf_cell(level, q), np.arange(len(q)))
        np.testing.assert_array_equal(workloads.hopf_cell(level, -q), np.arange(len(q)))
    fine = workloads.hopf_grid(3)
    kids = workloads.hopf_children(1, 3, np.arange(576))
    assert kids.shape == (576, 64)
    np.testing.assert_array_equal(np.sort(kids.ravel()), np.arange(len(fine)))
    np.testing.assert_array_equal(workloads.hopf_coarse_index(3, 1, kids), np.repeat(np.arange(576), 64).reshape(576, 64))
    # a fine point's cell at the coarse level is its parent
    np.testing.assert_array_equal(workloads.hopf_cell(1, fine), workloads.hopf_coarse_index(3, 1, np.arange(len(fine))))


def test_nearest_orientations_brute_force():
    """The k nearest grid quaternions by |<g, q>| (q and -q one orientation), closest first."""
    rng = np.random.default_rng(12)
    grid = workloads.random_quaternions(500, rng)
    q = -grid[17] * 0.999 + 0.001 * rng.standard_normal(4)
    q /= np.linalg.norm(q)
    idx = workloads.nearest_orientations(grid, q, 10)
    assert idx[0] == 17
    d = np.abs(grid @ q)
    np.testing.assert_array_equal(idx, np.argsort(-d, kind="stable")[:10])
