"""Seeded draws for the batched workload: several models against image stacks of mixed sizes.

Models: atom counts log-uniform in [500, 20000], radius scaled as atoms^(1/3) from 40 A at 500
atoms.  Stacks: 64 / 96 / 128 / 192 px over the same 140.8 A field of view, each with its own
image count, orientation grid (Hopf level 1-3 here; the configuration's full grids are levels
2-3) and defocus grid, shifts within N/8.  Every image comes from a seeded-random model.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .configs import Config
from .generate import atoms_in_ball, ctf_grid, hopf_grid, image_truth, standard_normal_noise, _rng

FOV_A = 140.8


@dataclass(frozen=True)
class StackSpec:
    npix: int
    n_img: int
    hopf_level: int
    n_defocus: int

    @property
    def pixel_A(self) -> float:
        return FOV_A / self.npix

    @property
    def max_shift(self) -> int:
        return self.npix // 8


@dataclass(frozen=True)
class BatchedConfig:
    seed: int = 1609_0004
    n_models: int = 4
    atoms_range: tuple = (500, 20000)
    stacks: tuple = field(default_factory=lambda: (StackSpec(64, 32, 1, 2), StackSpec(96, 32, 1, 2),
                                                   StackSpec(128, 32, 1, 2), StackSpec(192, 16, 1, 2)))
    sigma_A: float = 1.5
    snr: float = 0.1


def model_atoms(cfg: BatchedConfig, m: int) -> np.ndarray:
    rng = _rng(cfg.seed, 5, m)
    lo, hi = cfg.atoms_range
    n = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
    radius = 40.0 * (n / 500.0) ** (1.0 / 3.0)
    return atoms_in_ball(n, radius, cfg.seed * 1000 + m)


def stack_config(cfg: BatchedConfig, k: int) -> Config:
    st = cfg.stacks[k]
    return Config(name=f"batched-stack{k}", seed=cfg.seed * 10 + k, n_atoms=0, radius_A=0.0, sigma_A=cfg.sigma_A,
                  n_img=st.n_img, npix=st.npix, pixel_A=st.pixel_A, snr=cfg.snr, orient="hopf",
                  hopf_level=st.hopf_level, n_defocus=st.n_defocus, max_shift=st.max_shift)


def image_models(cfg: BatchedConfig, k: int) -> np.ndarray:
    """Model index of every image of stack k."""
    return _rng(cfg.seed, 6, k).integers(0, cfg.n_models, size=cfg.stacks[k].n_img)


def batched_workload(cfg: BatchedConfig) -> dict:
    stacks = []
    for k, st in enumerate(cfg.stacks):
        sc = stack_config(cfg, k)
        stacks.append({
            "config": sc,
            "quats": hopf_grid(st.hopf_level).astype(np.float32),
            "ctfs": ctf_grid(sc),
            "models": image_models(cfg, k),
            "truth": [image_truth(sc, i) for i in range(st.n_img)],
            "noise": [standard_normal_noise(sc, i) for i in range(st.n_img)],
        })
    return {"config": cfg, "atoms": [model_atoms(cfg, m) for m in range(cfg.n_models)], "stacks": stacks}
