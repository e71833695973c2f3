"""The seeded input generators follow the stated recipe (CPU only): sky
positivity and peak, point sources inside the central 80%, (u, v) inside
[-pi, pi) with the stated spread, uniform fraction, block sizes that partition
M with each block non-empty, unit-variance complex noise, reproducibility per
seed, and the workload table's sizes."""
import numpy as np
import pytest

from paper_1502_05037_gb300 import synth


def test_sky_is_positive_with_unit_peak_and_reproducible():
    a = synth.sky(64, 32, 1000, n_points=12, n_blobs=2)
    b = synth.sky(64, 32, 1000, n_points=12, n_blobs=2)
    assert a.shape == (32, 64) and a.dtype == np.float64
    assert np.array_equal(a, b)
    assert a.min() >= 0.0 and a.max() == 1.0
    assert not np.array_equal(a, synth.sky(64, 32, 1001, n_points=12, n_blobs=2))


def test_point_sources_sit_inside_the_central_80_percent():
    # without blobs the image is the point sources alone
    n = 100
    x = synth.sky(n, n, 7, n_points=50, n_blobs=0)
    iy, ix = np.nonzero(x)
    assert iy.min() >= 10 and iy.max() < 90 and ix.min() >= 10 and ix.max() < 90


def test_diffuse_component_is_positive_everywhere():
    n = 64
    compact = synth.sky(n, n, 3, n_points=10, n_blobs=2)
    both = synth.sky(n, n, 3, n_points=10, n_blobs=2, diffuse=True)
    # both are normalised to peak 1; the exponentiated diffuse field is
    # positive everywhere, so it lifts every pixel above zero
    assert both.min() > 0.0 and compact.min() >= 0.0
    assert both.max() == 1.0


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_uv_inside_the_band_with_the_stated_spread(dtype):
    M = 200_000
    u, v = synth.uv_coverage(M, 2000, dtype=dtype)
    assert u.dtype == dtype and u.shape == (M,)
    for c in (u, v):
        assert c.min() >= -np.pi and c.max() < np.pi
        # a normal with sigma = pi/4 truncated at 4 sigma keeps its spread
        assert abs(float(np.std(c.astype(np.float64))) - np.pi / 4) < 0.01
        assert abs(float(np.mean(c.astype(np.float64)))) < 0.01


def test_uniform_fraction():
    M = 100_000
    u, v = synth.uv_coverage(M, 5, uniform_fraction=0.5)
    # beyond |u| = pi/2: half of the uniform half (25% of all samples) plus
    # the Gaussian half's 4.6% beyond two sigma (2.3%)
    beyond = np.mean(np.abs(u) > np.pi / 2)
    assert 0.25 < beyond < 0.30


def test_uv_never_rounds_to_plus_pi_in_float32():
    u, v = synth.uv_coverage(50_000, 9, uniform_fraction=1.0, dtype=np.float32)
    assert u.max() < np.float32(np.pi) and v.max() < np.float32(np.pi)


@pytest.mark.parametrize("M,R", [(1, 1), (10, 10), (655_360, 8), (10_485_760, 64), (1000, 37)])
def test_block_sizes_partition_M(M, R):
    s = synth.block_sizes(M, R, 4000)
    assert s.dtype == np.int64 and s.size == R
    assert int(s.sum()) == M and s.min() >= 1
    offs = synth.block_offsets(s)
    assert offs[0] == 0 and offs[-1] == M and np.all(np.diff(offs) == s)


def test_block_sizes_are_uneven_and_reject_impossible_partitions():
    s = synth.block_sizes(1_000_000, 64, 1)
    assert s.max() > 1.5 * s.min()
    with pytest.raises(ValueError):
        synth.block_sizes(3, 4, 0)


def test_unit_noise_has_unit_power_split_evenly():
    n = synth.unit_noise(400_000, 3000)
    assert n.dtype == np.complex128
    assert abs(np.mean(np.abs(n) ** 2) - 1.0) < 0.01
    assert abs(np.var(n.real) - 0.5) < 0.01 and abs(np.var(n.imag) - 0.5) < 0.01
    assert abs(np.mean(n.real * n.imag)) < 0.01


def test_group_sequence_is_uniform_over_the_groups():
    s = synth.group_sequence(80_000, 8, 11)
    assert s.dtype == np.int32 and s.min() == 0 and s.max() == 7
    counts = np.bincount(s, minlength=8)
    assert np.all(np.abs(counts - 10_000) < 500)
    assert np.array_equal(s, synth.group_sequence(80_000, 8, 11))


def test_workload_table():
    W = synth.WORKLOADS
    want = {"sara64_fp64": (64, 8192, 4, 3, 1, 30.0, "f64"),
            "sara256_r8": (256, 655_360, 6, 4, 8, 30.0, "f32"),
            "sara1024_r64": (1024, 10_485_760, 6, 5, 64, 20.0, "f32"),
            "sara256_warm": (256, 131_072, 4, 3, 1, 30.0, "f32")}
    for name, (n, M, J, L, R, snr, dt) in want.items():
        w = W[name]
        assert (w.nx, w.ny, w.M, w.J, w.levels, w.R, w.snr_db, w.dtype) == (n, n, M, J, L, R, snr, dt)
    assert W["sara1024_r64"].diffuse and W["sara1024_r64"].uniform_fraction == 0.1
    for ch in (0, 17, 31):
        c = synth.channel_workload(ch)
        N = 512 * 512
        assert N // 2 <= c.M <= 5 * N and 4 <= c.R <= 16 and c.nx == 512


def test_draw_uses_one_seed_per_role():
    w = synth.WORKLOADS["sara64_fp64"]
    x, u, v, offs, nz = w.draw()
    assert np.array_equal(x, synth.sky(64, 64, 1000))
    u2, v2 = synth.uv_coverage(w.M, 2000, dtype=np.float64)
    assert np.array_equal(u, u2) and np.array_equal(v, v2)
    assert np.array_equal(nz, synth.unit_noise(w.M, 3000))
    assert np.array_equal(offs, synth.block_offsets(synth.block_sizes(w.M, w.R, 4000)))
