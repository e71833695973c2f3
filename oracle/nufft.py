"""Oracle: the measurement operator Phi and its adjoint (FP64, NumPy/SciPy).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper (Sec. 1) discretises the radio-interferometric measurement equation
as y = Phi x + n with x in R^N (later R_+^N, Eq. 1) and y in C^M, and leaves
the discretisation open. The reading implemented here:

* Image pixel (i, j), 0 <= i < ny, 0 <= j < nx, sits at centred integer
  coordinates n = (n1, n2) = (j - nx/2, i - ny/2); the column axis pairs with
  u and the row axis with v. (u, v) are in radians per pixel on [-pi, pi).
* Exact model (brute force, used to pin the NUFFT):
      y_m = sum_n x_n exp(-i (u_m n1 + v_m n2)).
* Fast model Phi = G F Z S, Kaiser-Bessel gridding (Fessler & Sutton 2003):
    - oversampled grid K = alpha * n per axis;
    - S: multiply pixel n by s_n = 1 / (ghat(n1) ghat(n2)), ghat the continuous
      Fourier transform of the gridding kernel g (closed form below);
    - Z: place the pixel at padded index (n mod K);
    - F: unnormalised forward 2-D DFT  X[k] = sum_p grid[p] exp(-2 pi i k.p / K);
    - G: kappa = u K / (2 pi); taps k_a = floor(kappa - J/2) + 1 + a,
      a = 0..J-1; y_m = sum_{a,b} g(kappa_u - k_a) g(kappa_v - k_b)
      X[k_b mod Ky][k_a mod Kx];
  with g(t) = I0(beta sqrt(1 - (2t/J)^2)) for |t| <= J/2 (0 outside) and
      ghat(nu) = J sinh(sqrt(beta^2 - (pi J nu / K)^2)) / sqrt(beta^2 - (pi J nu / K)^2)
  (sin/sqrt continuation when the radicand is negative), which is the exact
  integral of g(t) exp(2 pi i t nu / K) over |t| <= J/2.
* Adjoint Phi^dagger = S Z^T F^H G^H (the complex-conjugate transpose).

Nothing here is blocked, fused or reordered beyond the definitions above.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.fft
import scipy.special

TWO_PI = 2.0 * np.pi


def default_beta(J: int) -> float:
    """Kaiser-Bessel shape parameter beta = 2.34 J (Fessler & Sutton 2003,
    oversampling 2)."""
    return 2.34 * J


def pixel_coords(nx: int, ny: int) -> tuple[np.ndarray, np.ndarray]:
    """Centred coordinates n1 (columns) and n2 (rows)."""
    return np.arange(nx) - nx // 2, np.arange(ny) - ny // 2


# ---------------------------------------------------------------- exact model
def phi_exact(x: np.ndarray, u: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Brute-force y_m = sum_n x_n exp(-i (u_m n1 + v_m n2)); x is [ny][nx]."""
    ny, nx = x.shape
    n1, n2 = pixel_coords(nx, ny)
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    eu = np.exp(-1j * np.outer(u, n1))          # [M][nx]
    ev = np.exp(-1j * np.outer(v, n2))          # [M][ny]
    # y_m = sum_i sum_j ev[m,i] x[i,j] eu[m,j]
    return np.einsum("mi,ij,mj->m", ev, x.astype(np.complex128), eu)


def phi_exact_adj(y: np.ndarray, u: np.ndarray, v: np.ndarray, nx: int, ny: int) -> np.ndarray:
    """Conjugate transpose of phi_exact: x_n = sum_m y_m exp(+i (u_m n1 + v_m n2))."""
    n1, n2 = pixel_coords(nx, ny)
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    eu = np.exp(1j * np.outer(u, n1))
    ev = np.exp(1j * np.outer(v, n2))
    return np.einsum("m,mi,mj->ij", y.astype(np.complex128), ev, eu)


# ------------------------------------------------------- Kaiser-Bessel kernel
def kb_kernel(t: np.ndarray, J: int, beta: float) -> np.ndarray:
    """g(t) = I0(beta sqrt(1 - (2t/J)^2)) on |t| <= J/2, zero outside."""
    t = np.asarray(t, dtype=np.float64)
    r = 1.0 - (2.0 * t / J) ** 2
    out = scipy.special.i0(beta * np.sqrt(np.maximum(r, 0.0)))
    return np.where(np.abs(t) <= J / 2.0, out, 0.0)


def kb_ft(nu: np.ndarray, J: int, K: int, beta: float) -> np.ndarray:
    """ghat(nu) = J sinh(z)/z with z = sqrt(beta^2 - (pi J nu / K)^2);
    sin(|z|)/|z| when the radicand is negative, 1 at z = 0."""
    nu = np.asarray(nu, dtype=np.float64)
    a = beta * beta - (np.pi * J * nu / K) ** 2
    out = np.empty_like(a)
    pos = a > 0
    neg = a < 0
    zero = ~(pos | neg)
    zp = np.sqrt(a[pos])
    out[pos] = np.sinh(zp) / zp
    zn = np.sqrt(-a[neg])
    out[neg] = np.sin(zn) / zn
    out[zero] = 1.0
    return J * out


@dataclass
class NufftPlan:
    """Operator parameters shared by Phi and Phi^dagger."""
    nx: int
    ny: int
    u: np.ndarray
    v: np.ndarray
    J: int
    alpha: float = 2.0
    beta: float | None = None

    def __post_init__(self):
        if self.beta is None:
            self.beta = default_beta(self.J)
        self.Kx = int(round(self.alpha * self.nx))
        self.Ky = int(round(self.alpha * self.ny))
        self.u = np.asarray(self.u, dtype=np.float64)
        self.v = np.asarray(self.v, dtype=np.float64)

    @property
    def M(self) -> int:
        return int(self.u.size)


def correction(p: NufftPlan) -> np.ndarray:
    """S as an [ny][nx] array: s_n = 1 / (ghat_x(n1) ghat_y(n2))."""
    n1, n2 = pixel_coords(p.nx, p.ny)
    gx = kb_ft(n1, p.J, p.Kx, p.beta)
    gy = kb_ft(n2, p.J, p.Ky, p.beta)
    return 1.0 / np.outer(gy, gx)


def taps(coord: np.ndarray, K: int, J: int) -> tuple[np.ndarray, np.ndarray]:
    """For each coordinate: kappa = coord K / (2 pi), the J tap indices
    k_a = floor(kappa - J/2) + 1 + a (unwrapped, shape [M][J]) and the offsets
    t_a = kappa - k_a."""
    kappa = coord * (K / TWO_PI)
    k0 = np.floor(kappa - J / 2.0) + 1.0
    k = k0[:, None] + np.arange(J)[None, :]
    return k.astype(np.int64), kappa[:, None] - k


# -------------------------------------------------------------- the factors
def scale_pad(p: NufftPlan, x: np.ndarray) -> np.ndarray:
    """Z S: [ny][nx] image -> [Ky][Kx] complex grid, pixel n at (n mod K)."""
    n1, n2 = pixel_coords(p.nx, p.ny)
    grid = np.zeros((p.Ky, p.Kx), dtype=np.complex128)
    grid[np.ix_(n2 % p.Ky, n1 % p.Kx)] = correction(p) * x
    return grid


def fft2(grid: np.ndarray) -> np.ndarray:
    """F: unnormalised forward 2-D DFT."""
    return scipy.fft.fft2(grid)


def ifft2_unnormalised(grid: np.ndarray) -> np.ndarray:
    """F^H: sum_k X[k] exp(+2 pi i k.p / K), no 1/K^2 factor."""
    return scipy.fft.ifft2(grid) * grid.size


def degrid(p: NufftPlan, X: np.ndarray) -> np.ndarray:
    """G: interpolate the oversampled spectrum at (u, v)."""
    kx, tx = taps(p.u, p.Kx, p.J)
    ky, ty = taps(p.v, p.Ky, p.J)
    wx = kb_kernel(tx, p.J, p.beta)
    wy = kb_kernel(ty, p.J, p.beta)
    y = np.zeros(p.M, dtype=np.complex128)
    for b in range(p.J):
        for a in range(p.J):
            y += wy[:, b] * wx[:, a] * X[ky[:, b] % p.Ky, kx[:, a] % p.Kx]
    return y


def grid(p: NufftPlan, y: np.ndarray) -> np.ndarray:
    """G^H: spread each visibility onto its J x J footprint (real weights)."""
    kx, tx = taps(p.u, p.Kx, p.J)
    ky, ty = taps(p.v, p.Ky, p.J)
    wx = kb_kernel(tx, p.J, p.beta)
    wy = kb_kernel(ty, p.J, p.beta)
    X = np.zeros((p.Ky, p.Kx), dtype=np.complex128)
    y = np.asarray(y, dtype=np.complex128)
    for b in range(p.J):
        for a in range(p.J):
            np.add.at(X, (ky[:, b] % p.Ky, kx[:, a] % p.Kx), wy[:, b] * wx[:, a] * y)
    return X


def crop_scale(p: NufftPlan, grid_: np.ndarray) -> np.ndarray:
    """S Z^T: read pixel n from padded index (n mod K) and multiply by s_n."""
    n1, n2 = pixel_coords(p.nx, p.ny)
    return correction(p) * grid_[np.ix_(n2 % p.Ky, n1 % p.Kx)]


# ------------------------------------------------------------ the operators
def phi(p: NufftPlan, x: np.ndarray) -> np.ndarray:
    """y = G F Z S x (x real or complex [ny][nx]) -> complex [M]."""
    return degrid(p, fft2(scale_pad(p, x)))


def phi_adj(p: NufftPlan, y: np.ndarray) -> np.ndarray:
    """Phi^dagger y = S Z^T F^H G^H y -> complex [ny][nx]."""
    return crop_scale(p, ifft2_unnormalised(grid(p, y)))


def phi_matrix(p: NufftPlan) -> np.ndarray:
    """Dense [M][N] matrix of Phi, column by column (tiny sizes only)."""
    N = p.nx * p.ny
    A = np.empty((p.M, N), dtype=np.complex128)
    e = np.zeros(N)
    for k in range(N):
        e[:] = 0.0
        e[k] = 1.0
        A[:, k] = phi(p, e.reshape(p.ny, p.nx))
    return A


def power_norm_sq(p: NufftPlan, iters: int = 100, seed: int = 7) -> float:
    """||Phi||_2^2 for real inputs (largest eigenvalue of Re Phi^H Phi) by
    power iteration from a seeded random start."""
    g = np.random.Generator(np.random.PCG64(seed))
    x = g.standard_normal((p.ny, p.nx))
    x /= np.linalg.norm(x)
    lam = 0.0
    for _ in range(iters):
        w = np.real(phi_adj(p, phi(p, x)))
        lam = float(np.linalg.norm(w))
        x = w / lam
    return lam
