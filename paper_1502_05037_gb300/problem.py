"""Host-side set-up of an imaging problem for the GPU library: noise level
and per-block l2 bounds (problem (3) of the paper, Sec. 1: each eps_i bounds
the norm of the block's noise).

Reading of "an appropriate bound": complex noise n_m = sigma (a + i b)/sqrt 2
with a, b ~ N(0, 1), so (2/sigma^2) ||n_i||^2 ~ chi^2 with 2 M_i degrees of
freedom; eps_i is the chi^2 mean plus two standard deviations,
    eps_i = (sigma / sqrt 2) sqrt(2 M_i + 4 sqrt(M_i)),
and sigma = ||Phi x|| / sqrt(M) * 10^(-SNR/20) for an input SNR in dB.
"""
from __future__ import annotations

import numpy as np


def noise_sigma_from_norm(y_clean_norm: float, M: int, snr_db: float) -> float:
    return float(y_clean_norm / np.sqrt(M) * 10.0 ** (-snr_db / 20.0))


def chi2_epsilon(sigma: float, block_sizes) -> np.ndarray:
    m = np.asarray(block_sizes, dtype=np.float64)
    return sigma / np.sqrt(2.0) * np.sqrt(2.0 * m + 4.0 * np.sqrt(m))
