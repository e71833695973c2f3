"""Oracle: Daubechies filters, periodic 2-D wavelet transforms and the SARA
dictionary Psi (FP64, NumPy).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper (Sec. 1) builds the sparsity dictionary as a concatenation of q
coherent bases, Psi = [Psi_1, ..., Psi_q], and promotes average sparsity of
the analysis coefficients Psi^dagger x. It does not name the bases; the
reading implemented here is the SARA choice of the Dirac basis plus the
Daubechies wavelets db1..db8 (q = 9), each an orthonormal periodic 2-D Mallat
transform with L levels, and Psi normalised by 1/sqrt(q) so that
Psi Psi^dagger = I (a tight frame).

Daubechies filters (Daubechies 1992, Ten Lectures, Sec. 6.1): the p-tap-pair
filter h (length 2p, sum sqrt(2)) is sqrt(2) ((1 + z^-1)/2)^p Q(z^-1) with
|Q(e^{iw})|^2 = P(sin^2(w/2)), P(y) = sum_{k<p} C(p-1+k, k) y^k. Each root y_j
of P gives a pair of z-roots of z^2 - (2 - 4 y_j) z + 1; the minimum-phase
choice keeps the root inside the unit circle. High-pass g[n] = (-1)^n h[2p-1-n].

One analysis level on a periodic signal of even length L:
    a[k] = sum_n h[n] x[(2k + n) mod L],   d[k] = sum_n g[n] x[(2k + n) mod L],
stored as [a | d]; indices wrap as many times as needed when 2p > L. In 2-D
the rows are transformed first, then the columns, and the next level acts on
the top-left (low-low) quarter (Mallat packing).
"""
from __future__ import annotations

from functools import lru_cache
from math import comb

import numpy as np

Q_MAX = 9                      # Dirac + db1..db8
DEFAULT_MASK = (1 << Q_MAX) - 1


@lru_cache(maxsize=None)
def daubechies(p: int) -> np.ndarray:
    """Minimum-phase Daubechies low-pass filter with p vanishing moments
    (length 2p, sum sqrt(2)), by spectral factorisation."""
    if p < 1:
        raise ValueError("p >= 1")
    zeros = [-1.0] * p
    if p > 1:
        # P(y) coefficients, highest degree first for numpy.roots
        coeffs = [comb(p - 1 + k, k) for k in range(p)][::-1]
        for yj in np.roots(coeffs):
            c = 1.0 - 2.0 * yj
            disc = np.sqrt(c * c - 1.0 + 0j)
            z1, z2 = c + disc, c - disc
            zeros.append(z1 if abs(z1) < 1.0 else z2)
    h = np.real(np.poly(np.array(zeros, dtype=np.complex128)))
    return h * (np.sqrt(2.0) / h.sum())


def highpass(h: np.ndarray) -> np.ndarray:
    n = np.arange(h.size)
    return ((-1.0) ** n) * h[::-1]


@lru_cache(maxsize=None)
def _analysis_matrix_cached(L: int, p: int) -> np.ndarray:
    h = daubechies(p)
    g = highpass(h)
    A = np.zeros((L, L))
    half = L // 2
    for k in range(half):
        for n in range(h.size):
            A[k, (2 * k + n) % L] += h[n]
            A[half + k, (2 * k + n) % L] += g[n]
    return A


def analysis_matrix(L: int, p: int) -> np.ndarray:
    """One periodic analysis level of db_p on length L as a dense [L][L]
    matrix: rows 0..L/2-1 give a, rows L/2..L-1 give d."""
    if L % 2:
        raise ValueError("even length required")
    return _analysis_matrix_cached(L, p)


def dwt2(x: np.ndarray, p: int, levels: int) -> np.ndarray:
    """Orthonormal periodic 2-D DWT (db_p, `levels` levels), Mallat packed."""
    c = np.array(x, dtype=np.float64, copy=True)
    ny, nx = c.shape
    for _ in range(levels):
        Ax = analysis_matrix(nx, p)
        Ay = analysis_matrix(ny, p)
        band = c[:ny, :nx]
        band = band @ Ax.T          # rows
        band = Ay @ band            # columns
        c[:ny, :nx] = band
        ny //= 2
        nx //= 2
    return c


def idwt2(c: np.ndarray, p: int, levels: int) -> np.ndarray:
    """Adjoint (= inverse) of dwt2."""
    x = np.array(c, dtype=np.float64, copy=True)
    ny0, nx0 = x.shape
    sizes = [(ny0 >> l, nx0 >> l) for l in range(levels)]
    for ny, nx in reversed(sizes):
        Ax = analysis_matrix(nx, p)
        Ay = analysis_matrix(ny, p)
        band = x[:ny, :nx]
        band = Ay.T @ band
        band = band @ Ax
        x[:ny, :nx] = band
    return x


def bases(mask: int = DEFAULT_MASK) -> list[int]:
    """Basis list in dictionary order: 0 = Dirac, p = db_p."""
    return [j for j in range(Q_MAX) if mask >> j & 1]


def psi_adj(x: np.ndarray, levels: int, mask: int = DEFAULT_MASK) -> np.ndarray:
    """Psi^dagger x = [Psi_1^T x; ...; Psi_q^T x] / sqrt(q) -> [q][ny][nx]."""
    bs = bases(mask)
    q = len(bs)
    out = np.empty((q,) + x.shape)
    for i, j in enumerate(bs):
        out[i] = x if j == 0 else dwt2(x, j, levels)
    return out / np.sqrt(q)


def psi(c: np.ndarray, levels: int, mask: int = DEFAULT_MASK) -> np.ndarray:
    """Psi c = sum_j Psi_j c_j / sqrt(q), c is [q][ny][nx]."""
    bs = bases(mask)
    q = len(bs)
    x = np.zeros(c.shape[1:])
    for i, j in enumerate(bs):
        x += c[i] if j == 0 else idwt2(c[i], j, levels)
    return x / np.sqrt(q)
