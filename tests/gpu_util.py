"""Shared helpers of the GPU parity tests (inputs from the seeded generators,
expected values from the FP64 oracle only)."""
import numpy as np
import torch

import paper_1502_05037_gb300 as pk
from paper_1502_05037_gb300 import synth

DEV = torch.device("cuda:0")

# operator tolerances: relative l2 error of outputs, FP32 and FP64 plans
TOL = {pk.PURIFY_F32: 1e-5, pk.PURIFY_F64: 1e-12}


def np_real(dtype):
    return np.float32 if dtype == pk.PURIFY_F32 else np.float64


def np_cplx(dtype):
    return np.complex64 if dtype == pk.PURIFY_F32 else np.complex128


def t_real(dtype):
    return torch.float32 if dtype == pk.PURIFY_F32 else torch.float64


def t_cplx(dtype):
    return torch.complex64 if dtype == pk.PURIFY_F32 else torch.complex128


def rel(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def make_plan(nx, ny, M, J, levels=3, R=1, dtype=pk.PURIFY_F32, seed=0, sigma=np.pi / 4, mask=0, tile=0,
              uniform_fraction=0.0, grid_mode=0):
    u, v = synth.uv_coverage(M, 2000 + seed, sigma=sigma, uniform_fraction=uniform_fraction,
                             dtype=np_real(dtype))
    offs = synth.block_offsets(synth.block_sizes(M, R, 4000 + seed)) if R > 1 else None
    plan = pk.Plan(nx, ny, torch.from_numpy(u).to(DEV), torch.from_numpy(v).to(DEV), kb_width=J, levels=levels,
                   block_offsets=offs, dtype=dtype, basis_mask=mask, tile=tile,
                   grid_mode=grid_mode)
    return plan, u, v, offs


def snr_db(x_true, x):
    """Reconstruction SNR in dB (computed here so that no CUDA output is fed
    to the oracle)."""
    x_true = np.asarray(x_true, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    return float(20.0 * np.log10(np.linalg.norm(x_true) / np.linalg.norm(x_true - x)))
