"""Seeded draws for the learned-proposal workload.

Training: projections of several seeded models (atom counts 2000-10000, uniform balls with radius
80 A at 5000 atoms, scaled as atoms^(1/3)), each with the throughput workload's priors (uniform
orientation, integer shift within +-16 px, N ~ U[0.5, 2], mu ~ U[-1, 1], defocus ~ U[0.5, 2.5] um,
B ~ U[0, 50], SNR 0.1).  Labels: the coarse Hopf cell of the true orientation and the nearest of
the defocus grid values.  Inference: fresh draws of model 0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .generate import _rng, atoms_in_ball, defocus_grid, hopf_cell, random_quaternions


@dataclass(frozen=True)
class ProposalConfig:
    seed: int = 1609_0005
    n_models: int = 10
    atoms_range: tuple = (2000, 10000)
    npix: int = 128
    pixel_A: float = 1.1
    sigma_A: float = 1.5
    snr: float = 0.1
    max_shift: int = 16
    coarse_level: int = 2          # 4608 coarse cells
    fine_level: int = 4            # 294,912 fine orientations
    n_defocus: int = 4
    bfactors: tuple = (0.0, 50.0)
    top_k: int = 32
    n_train: int = 200_000
    n_infer: int = 10_000
    downsample: int = 2
    channels: int = 32
    voltage_kV: float = 300.0
    amp_contrast: float = 0.1

    @property
    def n_coarse(self) -> int:
        return 72 * 8 ** self.coarse_level

    @property
    def children(self) -> int:
        return 8 ** (self.fine_level - self.coarse_level)

    def defocus_values(self) -> np.ndarray:
        return defocus_grid(self.n_defocus, 0.5, 2.5)

    def ctf_rows(self) -> np.ndarray:
        """[n_defocus * n_B, 4] grid rows, defocus-major (index d * n_B + b)."""
        return np.array([(df, self.amp_contrast, b, self.voltage_kV) for df in self.defocus_values()
                         for b in self.bfactors], dtype=np.float64)


def proposal_models(cfg: ProposalConfig) -> list:
    out = []
    for m in range(cfg.n_models):
        rng = _rng(cfg.seed, 7, m)
        lo, hi = cfg.atoms_range
        n = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        out.append(atoms_in_ball(n, 80.0 * (n / 5000.0) ** (1.0 / 3.0), cfg.seed * 100 + m))
    return out


def draws(cfg: ProposalConfig, n: int, stream: int, chunk: int = 0, models: bool = True) -> dict:
    """n seeded image parameter draws (vectorised); stream 8 = training, 9 = inference."""
    rng = _rng(cfg.seed, stream, chunk)
    s = cfg.max_shift
    d = {
        "model": rng.integers(0, cfg.n_models, n) if models else np.zeros(n, dtype=np.int64),
        "quat": random_quaternions(n, rng).astype(np.float32),
        "dx": rng.integers(-s, s + 1, n),
        "dy": rng.integers(-s, s + 1, n),
        "norm": rng.uniform(0.5, 2.0, n),
        "offset": rng.uniform(-1.0, 1.0, n),
        "defocus_A": rng.uniform(0.5, 2.5, n) * 1.0e4,
        "bfactor": rng.uniform(0.0, 50.0, n),
    }
    d["label_q"] = hopf_cell(cfg.coarse_level, d["quat"]).astype(np.int32)
    dv = cfg.defocus_values()
    d["label_d"] = np.argmin(np.abs(d["defocus_A"][:, None] - dv[None, :]), axis=1).astype(np.int32)
    return d
