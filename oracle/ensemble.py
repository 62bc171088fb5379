"""Posterior of a structural ensemble over a set of images (Sec. 2, Eq. 10) — test infrastructure.

For models m with weights w_m (w_m >= 0, sum w_m = 1) and independent images omega,
    P(M | Omega) is proportional to prod_omega sum_m w_m P_{m omega},
so, from the matrix of ln P_{m omega} that the single-model scoring produces,
    ln P(M | Omega) = sum_omega ln sum_m w_m exp(ln P_{m omega})      (up to the same constant).

Weights that maximise it: the objective is concave in w on the simplex (a sum of logarithms of
linear functions), and the fixed-point iteration of expectation-maximisation for a mixture with
fixed components,
    r_{m omega} = w_m P_{m omega} / sum_m' w_m' P_{m' omega},    w_m <- (1 / |Omega|) sum_omega r_{m omega},
never decreases it.  The paper states Eq. 10 and the ensemble-weighting problem without giving an
optimiser; this iteration is our reading (the textbook one for weights of fixed mixture components).
Float64 numpy, plain loops over iterations.  Pinned in tests/test_oracle_pins.py.
"""
from __future__ import annotations

import numpy as np

from .likelihood import logsumexp


def log_posterior(logP: np.ndarray, weights: np.ndarray) -> float:
    """ln P(M | Omega) = sum over images of ln sum_m w_m P_{m omega}; logP [n_models, n_img]."""
    logP = np.asarray(logP, dtype=np.float64)
    w = np.asarray(weights, dtype=np.float64)
    w = w / w.sum()
    with np.errstate(divide="ignore"):
        lw = np.log(w)
    return float(np.sum(logsumexp(lw[:, None] + logP, axis=0)))


def model_log_posteriors(logP: np.ndarray) -> np.ndarray:
    """ln P({m} | Omega) of each model alone (w = 1 on m): the column sums of ln P_{m omega}."""
    return np.sum(np.asarray(logP, dtype=np.float64), axis=1)


def em_weights(logP: np.ndarray, weights: np.ndarray, n_iter: int) -> tuple[np.ndarray, list]:
    """n_iter fixed-point steps from `weights`; returns the weights and ln P(M | Omega) before each
    step and after the last."""
    logP = np.asarray(logP, dtype=np.float64)
    w = np.asarray(weights, dtype=np.float64)
    w = w / w.sum()
    history = [log_posterior(logP, w)]
    n_img = logP.shape[1]
    for _ in range(n_iter):
        with np.errstate(divide="ignore"):
            lw = np.log(w)
        a = lw[:, None] + logP                       # ln (w_m P_{m omega})
        r = np.exp(a - logsumexp(a, axis=0)[None, :])  # responsibilities, columns sum to 1
        w = r.sum(axis=1) / n_img
        history.append(log_posterior(logP, w))
    return w, history
