"""Synthetic workload configurations (shapes, sizes, priors, seeds).

The paper measures on experimental Frh and GroEL particle images (Section 4)
that are not available here; these seeded synthetic stand-ins reproduce the
structure of its workloads: one or more atomic models, particle images with a
PSF, a centre displacement, normalisation, offset and noise (Section 2,
Fig. 1), scored over orientation x PSF x displacement grids (the numerical
integral of Eq. 9, Section 3).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace


@dataclass(frozen=True)
class Config:
    name: str
    seed: int
    # model
    n_atoms: int
    radius_A: float
    sigma_A: float = 1.5
    atom_weight: float = 1.0
    # images
    n_img: int = 16
    npix: int = 32
    pixel_A: float = 2.0
    snr: float = 0.1
    norm_range: tuple = (0.5, 2.0)
    offset_range: tuple = (-1.0, 1.0)
    defocus_range_um: tuple = (0.5, 2.5)
    bfactor_range: tuple = (0.0, 50.0)
    voltage_kV: float = 300.0
    amp_contrast: float = 0.1
    # scoring grid
    orient: str = "random"       # "random" (seeded uniform quaternions) or "hopf"
    n_orient: int = 1152         # for "random"
    hopf_level: int = 3          # for "hopf": 72 * 8**level orientations
    n_defocus: int = 3
    bfactors: tuple = (0.0, 50.0)
    max_shift: int = 4
    # seeds of the orientation grid (a config may reuse another config's grid)
    grid_seed: int | None = None
    extra: dict = field(default_factory=dict)

    @property
    def n_quat(self) -> int:
        return self.n_orient if self.orient == "random" else 72 * 8 ** self.hopf_level

    @property
    def n_ctf(self) -> int:
        return self.n_defocus * len(self.bfactors)

    @property
    def n_ps(self) -> int:
        return self.n_quat * self.n_ctf

    @property
    def n_shift(self) -> int:
        return (2 * self.max_shift + 1) ** 2


CONFIGS: dict[str, Config] = {
    # tiny: 1 model of 500 atoms in a 40 A ball, 16 images 32x32 @ 2 A, 1152 random
    # quaternions x 3 defocus x 2 B = 6912 parameter sets, shifts within +-4 px.
    "tiny": Config(name="tiny", seed=1609_0001, n_atoms=500, radius_A=40.0, n_img=16, npix=32,
                   pixel_A=2.0, orient="random", n_orient=1152, n_defocus=3, max_shift=4),
    # throughput: 5000 atoms in an 80 A ball, 2048 images 128x128 @ 1.1 A, Hopf level-3
    # grid (36,864 quaternions) x 4 defocus x 2 B = 294,912 parameter sets, shifts +-16 px.
    "throughput": Config(name="throughput", seed=1609_0002, n_atoms=5000, radius_A=80.0, n_img=2048,
                         npix=128, pixel_A=1.1, orient="hopf", hopf_level=3, n_defocus=4,
                         max_shift=16),
    # precision: the tiny grid (its 1152 quaternions x 3 defocus x 2 B) and +-4 px shifts, with
    # images from the throughput model at 128x128 @ 1.1 A and at 64x64 @ 2.2 A (same field of view).
    "precision128": Config(name="precision128", seed=1609_0003, n_atoms=5000, radius_A=80.0, n_img=64,
                           npix=128, pixel_A=1.1, orient="random", n_orient=1152, n_defocus=3,
                           max_shift=4, grid_seed=1609_0001),
    "precision64": Config(name="precision64", seed=1609_0003, n_atoms=5000, radius_A=80.0, n_img=64,
                          npix=64, pixel_A=2.2, orient="random", n_orient=1152, n_defocus=3,
                          max_shift=4, grid_seed=1609_0001),
}


def get_config(name: str, **overrides) -> Config:
    cfg = CONFIGS[name]
    return replace(cfg, **overrides) if overrides else cfg
