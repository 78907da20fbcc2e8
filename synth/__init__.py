"""Seeded synthetic inputs for wideband radio-interferometric imaging.

This module draws the random inputs of the imaging problem and nothing else:
the truth cube built from the linear mixture model X = S H^T (Sec. 2.2,
Eq. "model"), per-channel uv coverage scaled by nu_l / nu_0 (Sec. 4.1), and
unit complex-normal noise draws. It holds none of the method's arithmetic:
the measurement operator, the noise level sigma, the l2 bounds epsilon and
everything downstream are computed separately by the oracle and by the CUDA
path, each from its own code.

Both sides read the same arrays from here, so a parity test compares the two
implementations on identical inputs.
"""

from .cubes import (  # noqa: F401
    CONFIGS,
    ProblemInputs,
    make_inputs,
    channel_freqs,
    gaussian_blobs,
    power_law_spectra,
    uv_coverage,
    uv_holes,
    in_holes,
    noise_draws,
)
