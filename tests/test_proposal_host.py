"""Host logic of the proposal path (no GPU): the per-image parameter-set lists of proposed joint bins."""
import numpy as np

from paper_1609_06634_gb300 import proposal


def test_cell_lists_match_a_per_image_loop():
    rng = np.random.default_rng(4)
    n_coarse, nd, nb, kids = 50, 4, 2, 8
    bins = rng.integers(0, n_coarse * nd, size=(7, 5))
    wave = np.array([3, 9, 10, 22, 41])
    pos = np.full(n_coarse, -1)
    pos[wave] = np.arange(len(wave))
    mask, off, flat = proposal._cell_lists(bins, pos, nd, nb, kids)
    nctf = nd * nb
    want, counts = [], []
    for i in range(bins.shape[0]):
        row = []
        for k in range(bins.shape[1]):
            cell, d = divmod(int(bins[i, k]), nd)
            assert mask[i, k] == (pos[cell] >= 0)
            if pos[cell] < 0:
                continue
            for j in range(kids):
                for b in range(nb):
                    row.append((pos[cell] * kids + j) * nctf + d * nb + b)
        want += row
        counts.append(len(row))
    np.testing.assert_array_equal(flat, want)
    np.testing.assert_array_equal(off, np.concatenate([[0], np.cumsum(counts)]))


def test_wave_lists_match_cell_lists():
    """The once-sorted per-wave lists equal _cell_lists' per-wave pass over all bins."""
    rng = np.random.default_rng(9)
    n_coarse, nd, nb, kids, wave = 60, 4, 2, 8, 7
    bins = np.stack([rng.choice(n_coarse * nd, 11, replace=False) for _ in range(9)])
    used = np.unique(bins // nd)
    waves = list(proposal._wave_lists(bins, n_coarse, nd, nb, kids, wave))
    assert len(waves) == -(-len(used) // wave)
    for t, (wc, idx, off, flat) in enumerate(waves):
        np.testing.assert_array_equal(wc, used[t * wave:(t + 1) * wave])
        pos = np.full(n_coarse, -1)
        pos[wc] = np.arange(len(wc))
        mask, off_ref, flat_ref = proposal._cell_lists(bins, pos, nd, nb, kids)
        np.testing.assert_array_equal(idx, np.flatnonzero(mask.ravel()))
        np.testing.assert_array_equal(off, off_ref)
        np.testing.assert_array_equal(flat, flat_ref)
