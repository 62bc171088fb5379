"""FP64 CPU oracle of the BioEM scoring path — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
(the oracle baseline, the inputs of its CPU context leg, ``--impl reference``)
may import this package.  The product (``paper_1609_06634_gb300``)
never imports it, and this package never imports the product: the two share
no code.  Inputs both sides use come from ``workloads`` (seeded draws only).

What it computes (paper section / equation in brackets):

* ``forward``: rotation by a unit quaternion [Sec. 3.1], the pixel-integrated
  projection of Gaussian atoms [Eq. 1], the DFT pair [Eqs. 2, 3], CTF and
  envelope [Eq. 4 and the functional forms after it], the PSF in Fourier space
  [Eq. 5], and synthetic images I_cal = N I1(r + d) - mu [Eq. 7] plus Gaussian
  noise [Eq. 8's noise model].
* ``likelihood``: image and projection moments, the cyclic cross-correlation
  for every displacement as a direct real-space sum [Sec. 3.3, Eqs. 11-12], the
  likelihood of Eq. 8 with N, mu and lambda integrated out in closed form
  [Sec. 3, first paragraph], and the grid sum of Eq. 9 as a log-sum-exp.
* ``ensemble``: the posterior of a weighted ensemble of models over a set of
  images [Sec. 2, Eq. 10], per-model posteriors, and the weights that maximise
  it (an expectation-maximisation fixed point: our reading).
* ``cnn``: the proposal network (not in the paper) and its chain-rule gradient.

Everything is float64 numpy; library primitives (matmul, erf, lgamma) serve as
steps.  Where the paper is silent or garbled, the function that takes a
reading says so in its docstring (quaternion convention, DFT exponent, CTF
coefficients from physical units, priors, displacement sign, cropping).

Parity pins (tests/test_oracle_pins.py): dense DFT against numpy.fft; the
direct-sum correlation against an FFT correlation; the closed form against a
brute-force 3-D quadrature of Eq. 8; invariances of log P under image offset,
image scale, projection scale and q -> -q; recovery of the true grid point and
shift on noiseless images; projection mass conservation and pixel integrals
against scipy's normal CDF and 2-D quadrature; rotation against scipy's
Rotation; electron wavelengths against textbook values; CTF(0) = -A and
Env(0) = 1.  No function of this package is "parity unpinned".
"""
from .forward import (  # noqa: F401
    apply_psf,
    ctf_coefficients,
    ctf_env,
    dft2,
    electron_wavelength_A,
    frequency_s2,
    idft2,
    pixel_centres,
    project,
    rotation_matrix,
    synthesize_image,
    synthesize_images,
)
from .ensemble import em_weights, log_posterior, model_log_posteriors  # noqa: F401
from .likelihood import (  # noqa: F401
    closed_form_loglik,
    correlation_all_shifts,
    log_norm_constant,
    logsumexp,
    moments,
    projections,
    score,
    shift_list,
)
