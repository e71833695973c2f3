"""Host-side set-up of an imaging problem: the noise level and the per-block
l2 bounds of problem (3) (Sec. 1, Eq. 3: eps_i bounds the norm of block i's
noise). Argument marshalling only: both values are computed by the library
(purify_noise_sigma, purify_chi2_epsilon in include/purify.h), which states
the chi^2 reading of "an appropriate bound" it uses.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from ._lib import check, load


def noise_sigma_from_norm(y_clean_norm: float, M: int, snr_db: float) -> float:
    """sigma for a noiseless ||Phi x|| and an input SNR in dB."""
    out = C.c_double()
    check(load().purify_noise_sigma(float(y_clean_norm), int(M), float(snr_db), C.byref(out)))
    return out.value


def chi2_epsilon(sigma: float, block_sizes) -> np.ndarray:
    """eps_i for blocks of the given sizes (the contiguous partition of Eq. 2)."""
    sizes = np.asarray(block_sizes, dtype=np.int64).ravel()
    offs = np.ascontiguousarray(np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64))
    eps = np.empty(sizes.size, dtype=np.float64)
    check(load().purify_chi2_epsilon(float(sigma), offs.ctypes.data_as(C.POINTER(C.c_int64)), int(sizes.size),
                                     eps.ctypes.data_as(C.POINTER(C.c_double))))
    return eps
