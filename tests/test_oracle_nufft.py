"""Pins for the oracle's measurement operator (CPU only).

Each check ties oracle.nufft to something other than itself: the brute-force
DFT of the measurement model (Sec. 1, y = Phi x + n), the defining property of
an adjoint, delta-image closed forms, numerical quadrature of the gridding
kernel's Fourier transform and the DFT written as an explicit matrix.
"""
import numpy as np
import pytest
import scipy.integrate

from oracle import nufft as nf
from paper_1502_05037_gb300 import synth


def _problem(n, J, M=200, seed=5, sigma=1.5):
    u, v = synth.uv_coverage(M, seed, sigma=sigma)
    return nf.NufftPlan(n, n, u, v, J)


# Relative l2 error bounds of Kaiser-Bessel gridding at oversampling 2 and
# beta = 2.34 J, measured on these cases (J=4: 1.2e-3, J=6: 9e-6, J=8: 1e-7)
# and rounded up; they must also fall with J.
NUFFT_BOUND = {4: 2.5e-3, 6: 2.5e-5, 8: 5e-7}


@pytest.mark.parametrize("n", [8, 16, 32])
def test_phi_matches_brute_force_dft(n):
    x = np.random.default_rng(n).standard_normal((n, n))
    errs = {}
    for J in (4, 6, 8):
        p = _problem(n, J)
        ye = nf.phi_exact(x, p.u, p.v)
        errs[J] = np.linalg.norm(nf.phi(p, x) - ye) / np.linalg.norm(ye)
        assert errs[J] <= NUFFT_BOUND[J], (J, errs[J])
    assert errs[4] > errs[6] > errs[8]


def test_phi_adj_matches_brute_force_adjoint():
    n = 16
    p = _problem(n, 6)
    g = np.random.default_rng(1)
    y = g.standard_normal(p.M) + 1j * g.standard_normal(p.M)
    xe = nf.phi_exact_adj(y, p.u, p.v, n, n)
    err = np.linalg.norm(nf.phi_adj(p, y) - xe) / np.linalg.norm(xe)
    assert err <= NUFFT_BOUND[6]


@pytest.mark.parametrize("J", [4, 5, 6])
def test_adjoint_identity(J):
    n = 16
    p = _problem(n, J, M=300)
    g = np.random.default_rng(2)
    x = g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))
    y = g.standard_normal(p.M) + 1j * g.standard_normal(p.M)
    lhs = np.vdot(y, nf.phi(p, x))
    rhs = np.vdot(nf.phi_adj(p, y), x)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_dense_adjoint_is_conjugate_transpose():
    n = 8
    p = _problem(n, 4, M=40)
    A = nf.phi_matrix(p)
    B = np.empty((n * n, p.M), dtype=np.complex128)
    for m in range(p.M):
        e = np.zeros(p.M, dtype=np.complex128)
        e[m] = 1.0
        B[:, m] = nf.phi_adj(p, e).ravel()
    assert np.allclose(B, A.conj().T, rtol=0, atol=1e-12 * np.abs(A).max())


@pytest.mark.parametrize("J", [4, 6])
def test_centred_delta_gives_ones(J):
    # the exact model gives y_m = 1 for a unit impulse at n = 0
    n = 16
    p = _problem(n, J, M=500)
    d = np.zeros((n, n))
    d[n // 2, n // 2] = 1.0
    assert np.abs(nf.phi(p, d) - 1.0).max() <= NUFFT_BOUND[J]


@pytest.mark.parametrize("n0", [(3, -2), (-5, 7), (0, 4)])
def test_shifted_delta_phase(n0):
    # impulse at n = (n1, n2) gives exp(-i (u n1 + v n2)): pins sign and origin
    n = 16
    p = _problem(n, 6, M=300)
    d = np.zeros((n, n))
    d[n0[1] + n // 2, n0[0] + n // 2] = 1.0
    want = np.exp(-1j * (p.u * n0[0] + p.v * n0[1]))
    assert np.abs(nf.phi(p, d) - want).max() <= 2 * NUFFT_BOUND[6]


def test_rectangular_image_axes():
    # nx != ny keeps u on columns and v on rows
    nx, ny = 16, 8
    u, v = synth.uv_coverage(150, 9, sigma=1.2)
    p = nf.NufftPlan(nx, ny, u, v, 6)
    x = np.random.default_rng(3).standard_normal((ny, nx))
    ye = nf.phi_exact(x, u, v)
    assert np.linalg.norm(nf.phi(p, x) - ye) / np.linalg.norm(ye) <= NUFFT_BOUND[6]


def test_kb_ft_matches_quadrature():
    J, K = 6, 64
    beta = nf.default_beta(J)
    for nu in (0.0, 3.0, 10.0, 31.0, 40.0):
        re, _ = scipy.integrate.quad(
            lambda t: float(nf.kb_kernel(np.array([t]), J, beta)[0]) * np.cos(2 * np.pi * t * nu / K),
            -J / 2, J / 2, limit=200, epsabs=0, epsrel=1e-12)
        got = float(nf.kb_ft(np.array([nu]), J, K, beta)[0])
        assert abs(got - re) <= 1e-9 * abs(re) + 1e-12


def test_fft_matches_dft_matrix():
    K = 8
    g = np.random.default_rng(4)
    X = g.standard_normal((K, K)) + 1j * g.standard_normal((K, K))
    k = np.arange(K)
    Fm = np.exp(-2j * np.pi * np.outer(k, k) / K)
    assert np.allclose(nf.fft2(X), Fm @ X @ Fm.T, atol=1e-12)
    assert np.allclose(nf.ifft2_unnormalised(X), Fm.conj() @ X @ Fm.conj().T, atol=1e-12)


def test_taps_cover_kernel_support():
    J, K = 6, 64
    g = np.random.default_rng(5)
    c = g.uniform(-np.pi, np.pi, 1000)
    k, t = nf.taps(c, K, J)
    assert np.all(np.abs(t) <= J / 2 + 1e-12)
    kappa = c * K / (2 * np.pi)
    # the taps are exactly the integers in (kappa - J/2, kappa + J/2]
    assert np.all(k[:, 0] > kappa - J / 2) and np.all(k[:, 0] - 1 <= kappa - J / 2)


def test_wrap_at_band_edge():
    # visibilities at the edges of [-pi, pi) wrap around the periodic grid
    n = 16
    u = np.array([-np.pi, np.nextafter(np.pi, 0), 0.0, -np.pi])
    v = np.array([0.3, -np.pi, np.nextafter(np.pi, 0), -np.pi])
    p = nf.NufftPlan(n, n, u, v, 6)
    x = np.random.default_rng(6).standard_normal((n, n))
    ye = nf.phi_exact(x, u, v)
    assert np.linalg.norm(nf.phi(p, x) - ye) / np.linalg.norm(ye) <= NUFFT_BOUND[6]


def test_power_norm_matches_dense_spectrum():
    n = 8
    p = _problem(n, 4, M=60)
    A = nf.phi_matrix(p)
    lam = np.linalg.eigvalsh(np.real(A.conj().T @ A)).max()
    assert abs(nf.power_norm_sq(p, iters=300) - lam) <= 1e-8 * lam
