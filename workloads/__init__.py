"""Seeded synthetic inputs for the BioEM scoring workloads.

This module is shared by the FP64 oracle (``oracle/``) and by the CUDA path
(``paper_1609_06634_gb300``).  It holds only random draws and parameter grids:
atom coordinates, orientation grids, CTF parameter lists, the "true" parameters
of each synthetic image and its standard-normal noise field.  It contains none
of the method's arithmetic (no projection, no Fourier transform, no CTF
formula, no likelihood): each side turns these draws into images and scores
with its own code.

Workload shapes follow the paper's setting (Section 4: images of a model in
random orientation, with a PSF, a centre displacement, normalisation, offset and
Gaussian noise, scored over orientation x PSF x displacement grids); the sizes
are those of the configurations in ``configs.py`` and ``batched.py``.
"""
from .configs import CONFIGS, Config, get_config  # noqa: F401
from .batched import BatchedConfig, StackSpec, batched_workload, model_atoms  # noqa: F401
from .proposal import ProposalConfig, draws as proposal_draws, proposal_models  # noqa: F401
from .generate import (  # noqa: F401
    atoms_in_ball,
    ctf_grid,
    defocus_grid,
    healpix_nest_ang2pix,
    healpix_nest_pix2ang,
    hopf_cell,
    hopf_children,
    hopf_grid,
    hopf_coarse_index,
    image_truth,
    nearest_orientations,
    random_quaternions,
    standard_normal_noise,
    workload,
)
