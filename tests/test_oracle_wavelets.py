"""Pins for the oracle's SARA dictionary (CPU only).

Checks oracle.wavelets against Daubechies' closed forms and defining
properties (orthonormality, vanishing moments, minimum phase), against the
Haar transform written out by hand, and against the tight-frame identity that
the 1/sqrt(q) normalisation of Psi = [Psi_1, ..., Psi_q] (Sec. 1) must give.
"""
import itertools
from math import comb

import numpy as np
import pytest

from oracle import wavelets as wv


def test_db1_is_haar():
    assert np.allclose(wv.daubechies(1), [2 ** -0.5, 2 ** -0.5], atol=1e-15)


def test_db2_closed_form():
    s3 = np.sqrt(3.0)
    want = np.array([1 + s3, 3 + s3, 3 - s3, 1 - s3]) / (4 * np.sqrt(2.0))
    assert np.allclose(wv.daubechies(2), want, atol=1e-14)


@pytest.mark.parametrize("p", range(1, 9))
def test_filter_identities(p):
    h = wv.daubechies(p)
    g = wv.highpass(h)
    assert h.size == 2 * p
    assert abs(h.sum() - np.sqrt(2)) < 1e-13
    for l in range(p):
        s = np.dot(h[: h.size - 2 * l], h[2 * l:])
        assert abs(s - (1.0 if l == 0 else 0.0)) < 1e-12
    n = np.arange(h.size, dtype=np.float64)
    for k in range(p):  # p vanishing moments of the wavelet
        assert abs(np.sum(g * n ** k)) < 1e-9 * max(1.0, np.sum(np.abs(g) * n ** k))


@pytest.mark.parametrize("p", range(2, 7))
def test_minimum_phase_has_most_early_energy(p):
    # among all spectral factors of the same |H|^2, the minimum-phase one has
    # the largest partial energy sum_{n<k} h_n^2 for every k (Robinson)
    coeffs = [comb(p - 1 + k, k) for k in range(p)][::-1]
    pairs = []
    for yj in np.roots(coeffs):
        c = 1.0 - 2.0 * yj
        d = np.sqrt(c * c - 1.0 + 0j)
        pairs.append((c + d, c - d))
    h0 = wv.daubechies(p)
    e0 = np.cumsum(h0 ** 2)
    for choice in itertools.product((0, 1), repeat=len(pairs)):
        zs = [-1.0] * p + [pr[ch] for pr, ch in zip(pairs, choice)]
        hc = np.poly(np.array(zs, dtype=np.complex128))
        if np.abs(hc.imag).max() > 1e-9 * np.abs(hc).max():
            continue  # conjugate roots split: not a real filter
        h = hc.real * (np.sqrt(2.0) / hc.real.sum())
        assert np.all(np.cumsum(h ** 2) <= e0 + 1e-12)


def test_haar_2x2_by_hand():
    a, b, c, d = 1.0, 2.0, 5.0, -3.0
    out = wv.dwt2(np.array([[a, b], [c, d]]), 1, 1)
    want = np.array([[a + b + c + d, a - b + c - d], [a + b - c - d, a - b - c + d]]) / 2
    assert np.allclose(out, want, atol=1e-15)


@pytest.mark.parametrize("p", range(1, 9))
@pytest.mark.parametrize("shape,levels", [((8, 8), 3), ((16, 32), 3), ((64, 64), 4)])
def test_perfect_reconstruction_and_parseval(p, shape, levels):
    x = np.random.default_rng(p).standard_normal(shape)
    c = wv.dwt2(x, p, levels)
    assert np.abs(wv.idwt2(c, p, levels) - x).max() < 1e-12
    assert abs(np.linalg.norm(c) - np.linalg.norm(x)) < 1e-12 * np.linalg.norm(x)


@pytest.mark.parametrize("p", [2, 4, 8])
def test_polynomial_annihilation(p):
    # first-level details of a degree < p polynomial vanish where the filter
    # does not wrap around the periodic boundary
    L = 64
    t = np.arange(L, dtype=np.float64)
    x = np.polyval(np.arange(1, p + 1, dtype=np.float64), t / L)
    A = wv.analysis_matrix(L, p)
    d = A[L // 2:] @ x
    k_ok = [k for k in range(L // 2) if 2 * k + 2 * p - 1 < L]
    assert np.abs(d[k_ok]).max() < 1e-9 * np.abs(x).max()


def test_shift_by_two_shifts_coefficients_by_one():
    # a[k] uses x[2k + n]: shifting x left by 2 shifts a and d left by 1
    L, p = 32, 3
    x = np.random.default_rng(7).standard_normal(L)
    A = wv.analysis_matrix(L, p)
    c, cs = A @ x, A @ np.roll(x, -2)
    assert np.allclose(cs[: L // 2], np.roll(c[: L // 2], -1), atol=1e-13)
    assert np.allclose(cs[L // 2:], np.roll(c[L // 2:], -1), atol=1e-13)


def test_first_coefficient_by_definition():
    L, p = 8, 4  # 8-tap filter on 8 samples: every tap wraps once
    x = np.random.default_rng(8).standard_normal(L)
    h, g = wv.daubechies(p), wv.highpass(wv.daubechies(p))
    A = wv.analysis_matrix(L, p)
    for k in range(L // 2):
        a = sum(h[n] * x[(2 * k + n) % L] for n in range(2 * p))
        d = sum(g[n] * x[(2 * k + n) % L] for n in range(2 * p))
        assert abs((A @ x)[k] - a) < 1e-14 and abs((A @ x)[L // 2 + k] - d) < 1e-14


@pytest.mark.parametrize("mask", [wv.DEFAULT_MASK, 0b11, 0b100000001])
def test_tight_frame(mask):
    levels = 3
    g = np.random.default_rng(9)
    x = g.standard_normal((16, 16))
    c = wv.psi_adj(x, levels, mask)
    q = len(wv.bases(mask))
    assert c.shape == (q, 16, 16)
    assert np.abs(wv.psi(c, levels, mask) - x).max() < 1e-12          # Psi Psi^dagger = I
    assert abs(np.linalg.norm(c) - np.linalg.norm(x)) < 1e-12 * np.linalg.norm(x)  # Parseval
    c2 = g.standard_normal(c.shape)
    P = wv.psi_adj(wv.psi(c2, levels, mask), levels, mask)
    assert np.abs(wv.psi_adj(wv.psi(P, levels, mask), levels, mask) - P).max() < 1e-12  # idempotent
    # <Psi^dagger x, c2> = <x, Psi c2>
    assert abs(np.sum(c * c2) - np.sum(x * wv.psi(c2, levels, mask))) < 1e-11


def test_dirac_plane_is_scaled_image():
    x = np.random.default_rng(10).standard_normal((8, 8))
    c = wv.psi_adj(x, 2)
    assert np.allclose(c[0], x / 3.0, atol=1e-15)
