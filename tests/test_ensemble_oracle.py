"""Pins of the ensemble posterior oracle (Sec. 2, Eq. 10) — no GPU."""
import numpy as np
import scipy.optimize

import oracle


def _mat(rng, m, n, spread=30.0):
    return -5000.0 + spread * rng.standard_normal((m, n))


def test_single_model_and_concentrated_weights_reduce_to_column_sums():
    rng = np.random.default_rng(1)
    lp = _mat(rng, 1, 50)
    assert abs(oracle.log_posterior(lp, [3.7]) - lp.sum()) < 1e-9
    lp = _mat(rng, 4, 50)
    per = oracle.model_log_posteriors(lp)
    for m in range(4):
        w = np.zeros(4)
        w[m] = 1.0
        assert abs(oracle.log_posterior(lp, w) - per[m]) < 1e-9 * abs(per[m])


def test_identical_models_make_weights_irrelevant():
    rng = np.random.default_rng(2)
    row = _mat(rng, 1, 40)[0]
    lp = np.stack([row, row, row])
    ref = row.sum()
    for w in ([1, 1, 1], [0.2, 0.7, 0.1], [5, 0, 1]):
        assert abs(oracle.log_posterior(lp, w) - ref) < 1e-9 * abs(ref)


def test_per_image_offsets_shift_the_posterior_and_keep_em_weights():
    rng = np.random.default_rng(3)
    lp = _mat(rng, 3, 60, spread=3.0)
    c = 100.0 * rng.standard_normal(60)
    w = np.array([0.2, 0.5, 0.3])
    assert abs(oracle.log_posterior(lp + c[None, :], w) - oracle.log_posterior(lp, w) - c.sum()) < 1e-7
    w1, _ = oracle.em_weights(lp, w, 20)
    w2, _ = oracle.em_weights(lp + c[None, :], w, 20)
    np.testing.assert_allclose(w1, w2, atol=1e-12)


def test_em_reaches_the_library_optimum_two_models():
    """Maximiser of f(w) = sum ln(w P1 + (1 - w) P2) from scipy's bounded scalar minimiser."""
    rng = np.random.default_rng(4)
    lp = _mat(rng, 2, 200, spread=2.0)

    def negf(x):
        return -oracle.log_posterior(lp, [x, 1.0 - x])

    r = scipy.optimize.minimize_scalar(negf, bounds=(0.0, 1.0), method="bounded", options={"xatol": 1e-10})
    w, hist = oracle.em_weights(lp, [0.5, 0.5], 2000)
    assert abs(w[0] - r.x) < 1e-4
    assert hist[-1] >= -r.fun - 1e-9


def test_em_monotone_and_beats_a_simplex_grid_three_models():
    rng = np.random.default_rng(5)
    lp = _mat(rng, 3, 150, spread=2.5)
    w, hist = oracle.em_weights(lp, [1, 1, 1], 500)
    assert all(b >= a - 1e-9 for a, b in zip(hist, hist[1:]))
    best = -np.inf
    g = np.linspace(0.0, 1.0, 101)
    for a in g:
        for b in g[g <= 1.0 - a + 1e-12]:
            best = max(best, oracle.log_posterior(lp, [a, b, max(0.0, 1.0 - a - b)]))
    assert hist[-1] >= best - 1e-9


def test_planted_mixture_weights():
    """Model 0 explains 70 % of the images and model 1 the rest, each by a margin of 50 nats: the
    optimal weights are the proportions (0.7, 0.3) to within e^-50."""
    n = 1000
    lp = np.full((2, n), -50.0)
    lp[0, :700] = 0.0
    lp[1, 700:] = 0.0
    w, _ = oracle.em_weights(lp, [0.5, 0.5], 200)
    np.testing.assert_allclose(w, [0.7, 0.3], atol=1e-9)
