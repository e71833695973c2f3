"""C ABI checks that need no GPU: the library builds, loads, exports every
function include/purify.h declares, and the ctypes structures match the C
layout (checked by compiling a C probe against the header with gcc)."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_1502_05037_gb300 import _lib
from paper_1502_05037_gb300 import build as pbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "purify.h")


@pytest.fixture(scope="module")
def lib():
    pbuild.build()
    return _lib.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(purify_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    fns = declared_functions()
    for name in ("purify_plan_create", "purify_phi", "purify_phi_adj", "purify_psi", "purify_psi_adj",
                 "purify_sdmm_solve", "purify_reweight"):
        assert name in fns


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (purify_[a-z0-9_]+)", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    for f in declared_functions():
        assert hasattr(lib, f)
    assert sorted(_lib.exported_symbols()) == declared_functions()


def test_ctypes_layout_matches_c(lib):
    probe = r"""
#include <stddef.h>
#include <stdio.h>
#include "purify.h"
#define P(T, f) printf(#T "." #f " %zu\n", offsetof(T, f));
int main(void) {
  printf("desc %zu\n", sizeof(purify_plan_desc));
  printf("info %zu\n", sizeof(purify_plan_info));
  printf("params %zu\n", sizeof(purify_sdmm_params));
  printf("stats %zu\n", sizeof(purify_sdmm_stats));
  printf("ktime %zu\n", sizeof(purify_kernel_time));
  printf("pd %zu\n", sizeof(purify_pd_params));
  P(purify_pd_params, tau) P(purify_pd_params, nu)
  P(purify_plan_desc, tile) P(purify_plan_desc, stream) P(purify_plan_desc, dtype) P(purify_plan_desc, block_offsets)
  P(purify_sdmm_params, resume) P(purify_sdmm_params, check_every) P(purify_sdmm_params, toeplitz) P(purify_sdmm_stats, status)
  P(purify_sdmm_params, block_groups) P(purify_sdmm_params, group_seq)
  P(purify_plan_info, workspace_bytes) P(purify_plan_info, beta) P(purify_plan_info, grid_mode)
  P(purify_plan_info, lane_tile) P(purify_plan_info, fft_cols_per_thread)
  P(purify_plan_desc, grid_mode)
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "probe.c")
        exe = os.path.join(d, "probe")
        open(src, "w").write(probe)
        subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        lines = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(l.rsplit(" ", 1) for l in lines if l)
    assert int(got["desc"]) == ctypes.sizeof(_lib.purify_plan_desc)
    assert int(got["info"]) == ctypes.sizeof(_lib.purify_plan_info)
    assert int(got["params"]) == ctypes.sizeof(_lib.purify_sdmm_params)
    assert int(got["purify_sdmm_params.block_groups"]) == _lib.purify_sdmm_params.block_groups.offset
    assert int(got["purify_sdmm_params.group_seq"]) == _lib.purify_sdmm_params.group_seq.offset
    assert int(got["stats"]) == ctypes.sizeof(_lib.purify_sdmm_stats)
    assert int(got["ktime"]) == ctypes.sizeof(_lib.purify_kernel_time)
    assert int(got["pd"]) == ctypes.sizeof(_lib.purify_pd_params)
    assert int(got["purify_pd_params.tau"]) == _lib.purify_pd_params.tau.offset
    assert int(got["purify_pd_params.nu"]) == _lib.purify_pd_params.nu.offset
    assert int(got["purify_plan_desc.tile"]) == _lib.purify_plan_desc.tile.offset
    assert int(got["purify_plan_desc.stream"]) == _lib.purify_plan_desc.stream.offset
    assert int(got["purify_plan_desc.dtype"]) == _lib.purify_plan_desc.dtype.offset
    assert int(got["purify_plan_desc.grid_mode"]) == _lib.purify_plan_desc.grid_mode.offset
    assert int(got["purify_plan_info.grid_mode"]) == _lib.purify_plan_info.grid_mode.offset
    assert int(got["purify_plan_info.lane_tile"]) == _lib.purify_plan_info.lane_tile.offset
    assert int(got["purify_plan_info.fft_cols_per_thread"]) == _lib.purify_plan_info.fft_cols_per_thread.offset
    assert int(got["purify_plan_desc.block_offsets"]) == _lib.purify_plan_desc.block_offsets.offset
    assert int(got["purify_sdmm_params.resume"]) == _lib.purify_sdmm_params.resume.offset
    assert int(got["purify_sdmm_params.check_every"]) == _lib.purify_sdmm_params.check_every.offset
    assert int(got["purify_sdmm_params.toeplitz"]) == _lib.purify_sdmm_params.toeplitz.offset
    assert int(got["purify_sdmm_stats.status"]) == _lib.purify_sdmm_stats.status.offset
    assert int(got["purify_plan_info.workspace_bytes"]) == _lib.purify_plan_info.workspace_bytes.offset
    assert int(got["purify_plan_info.beta"]) == _lib.purify_plan_info.beta.offset


def test_invalid_description_is_rejected_before_any_launch(lib):
    # no GPU needed: validation happens on the host first
    d = _lib.purify_plan_desc(nx=30, ny=32, M=10, u=None, v=None, R=1, kb_width=6, levels=3)
    h = ctypes.c_void_p()
    assert lib.purify_plan_create(ctypes.byref(d), ctypes.byref(h)) == _lib.PURIFY_EINVAL
    assert b"powers of two" in lib.purify_last_error()
    assert lib.purify_plan_create(None, ctypes.byref(h)) == _lib.PURIFY_EINVAL
    assert lib.purify_phi(None, None, None) == _lib.PURIFY_EINVAL
    assert lib.purify_plan_destroy(None) == _lib.PURIFY_OK


@pytest.mark.parametrize("fields,msg", [
    ({"M": 0}, b"M must be"),                                     # no visibilities
    ({"R": 5, "M": 4}, b"R must be"),                             # more blocks than visibilities
    ({"kb_width": 9}, b"kb_width"),
    ({"kb_width": 1}, b"kb_width"),
    ({"levels": 6, "nx": 16, "ny": 16}, b"too small"),            # deeper than the image allows
    ({"tile": 12}, b"tile"),
    ({"grid_mode": 7}, b"grid_mode"),
    ({"grid_mode": -1}, b"grid_mode"),
    ({"grid_mode": 4, "dtype": 1}, b"grid_mode 3..6"),
    ({"grid_mode": 3, "dtype": 1}, b"grid_mode 3..6"),               # lanes are FP32 only
    ({"grid_mode": 3, "kb_width": 7}, b"grid_mode 3..6"),
    ({"grid_mode": 6, "dtype": 1}, b"grid_mode 3..6"),               # deterministic lanes too
    ({"grid_mode": 6, "kb_width": 8}, b"grid_mode 3..6"),
    ({"oversample": 1.5}, b"oversample"),
    ({"dtype": 7}, b"dtype"),
    ({"basis_mask": 0x200}, b"basis_mask"),
])
def test_degenerate_descriptions_are_rejected_on_the_host(lib, fields, msg):
    dummy = (ctypes.c_float * 8)()   # never read: validation fails first
    base = dict(nx=32, ny=32, M=100, u=ctypes.addressof(dummy), v=ctypes.addressof(dummy), R=1, kb_width=6,
                levels=3)
    base.update(fields)
    d = _lib.purify_plan_desc(**base)
    h = ctypes.c_void_p()
    assert lib.purify_plan_create(ctypes.byref(d), ctypes.byref(h)) == _lib.PURIFY_EINVAL
    assert msg in lib.purify_last_error()
    assert not h.value


@pytest.mark.parametrize("offs,msg", [
    ([0, 50, 50, 100], b"non-empty"),      # an empty block (problem (3) needs a bound per block)
    ([0, 60, 40, 100], b"non-empty"),      # decreasing offsets
    ([1, 50, 70, 100], b"start at 0"),
    ([0, 50, 70, 99], b"end at M"),
])
def test_block_partitions_must_cover_the_visibilities(lib, offs, msg):
    dummy = (ctypes.c_float * 8)()
    o = (ctypes.c_int64 * len(offs))(*offs)
    d = _lib.purify_plan_desc(nx=32, ny=32, M=100, u=ctypes.addressof(dummy), v=ctypes.addressof(dummy), R=3,
                              block_offsets=ctypes.cast(o, ctypes.POINTER(ctypes.c_int64)), kb_width=6, levels=3)
    h = ctypes.c_void_p()
    assert lib.purify_plan_create(ctypes.byref(d), ctypes.byref(h)) == _lib.PURIFY_EINVAL
    assert msg in lib.purify_last_error()


def test_launch_counter_starts_finite(lib):
    assert lib.purify_launch_count() >= 0


def test_problem_setup_matches_the_oracle_reading(lib):
    # sigma and the chi^2 bounds of Eq. 3 are host calls of the library (no
    # GPU work); they follow the oracle's reading of "an appropriate bound"
    import numpy as np

    from oracle import sdmm as osd
    from paper_1502_05037_gb300 import problem, synth

    g = np.random.default_rng(3)
    y = g.standard_normal(5000) + 1j * g.standard_normal(5000)
    assert abs(problem.noise_sigma_from_norm(np.linalg.norm(y), y.size, 27.5) - osd.noise_sigma(y, 27.5)) \
        <= 1e-14 * osd.noise_sigma(y, 27.5)
    sizes = synth.block_sizes(100000, 13, 4)
    got = problem.chi2_epsilon(0.37, sizes)
    want = osd.epsilon_chi2(0.37, sizes)
    assert np.max(np.abs(got - want) / want) <= 1e-14
    # a single visibility block of size 1: sqrt(2 + 4) sigma / sqrt 2
    assert abs(problem.chi2_epsilon(2.0, [1])[0] - np.sqrt(6.0) * 2.0 / np.sqrt(2.0)) <= 1e-14 * 4
    for bad in (lambda: problem.chi2_epsilon(0.0, sizes), lambda: problem.chi2_epsilon(-1.0, sizes),
                lambda: problem.chi2_epsilon(1.0, [3, 0, 2]), lambda: problem.noise_sigma_from_norm(1.0, 0, 30.0),
                lambda: problem.noise_sigma_from_norm(float("nan"), 10, 30.0)):
        with pytest.raises(_lib.PurifyError) as e:
            bad()
        assert e.value.status == _lib.PURIFY_EINVAL
