"""Matern prior covariance on the periodic parameter grid (oracle, FP64).

Test infrastructure only (see the package docstring).

The paper's prior covariance is block diagonal in time, each block the inverse
of an elliptic operator in space that represents a Matern covariance (Sec.
"State of the art", the Gaussian prior).  It gives no constants; the reading
used here (and by the GPU path, written independently) is:

* Gamma_pr = I_Nt (x) C, white in time;
* C is the stationary covariance on the periodic Nx x Ny grid over
  [0, Lx) x [0, Ly) whose eigenvalues in the discrete Fourier basis are
      s(k) = (kappa^2 + |k|^2)^(-(nu + d/2)),  d = 2,  kappa = sqrt(2 nu)/ell,
      k = 2 pi (p/Lx, q/Ly), p, q the signed integer frequencies,
  scaled so that the pointwise variance is exactly `var`:
      lambda_k = var * N * s(k) / sum_k s(k),   N = Nx Ny;
* C x = IDFT2(lambda * DFT2(x)), C^(1/2) uses sqrt(lambda), C^-1 uses 1/lambda.

The DFTs are written with explicit DFT matrices (no FFT library):
X^[p, q] = sum_{a,b} X[a, b] exp(-2 pi i (p a / Nx + q b / Ny)), and the
inverse carries the 1/N.  Flat parameter index k = a*Ny + b.
"""
from __future__ import annotations

import math

import numpy as np


def signed_frequencies(n: int) -> np.ndarray:
    """0, 1, ..., n//2, then the negative frequencies -(n - n//2 - 1) .. -1."""
    a = np.arange(n)
    return np.where(a <= n // 2, a, a - n)


def matern_spectrum(Nx: int, Ny: int, Lx: float = 1.0, Ly: float = 1.0,
                    nu: float = 1.0, ell: float = 0.1, var: float = 1.0) -> np.ndarray:
    """Eigenvalues lambda[p, q] of C (shape [Nx, Ny])."""
    kappa = math.sqrt(2.0 * nu) / ell
    kx = 2.0 * math.pi * signed_frequencies(Nx) / Lx
    ky = 2.0 * math.pi * signed_frequencies(Ny) / Ly
    k2 = kx[:, None] ** 2 + ky[None, :] ** 2
    s = (kappa * kappa + k2) ** (-(nu + 1.0))
    N = Nx * Ny
    return var * N * s / s.sum()


def spectrum_for(cfg) -> np.ndarray:
    return matern_spectrum(cfg.Nx, cfg.Ny, cfg.Lx, cfg.Ly, cfg.nu, cfg.ell, cfg.var)


def dft_matrix(n: int) -> np.ndarray:
    """W[p, a] = exp(-2 pi i p a / n).

    The phase index p*a is reduced mod n first (exact: the exponential is
    n-periodic); otherwise rounding of the phase argument 2 pi p a / n, which
    grows with p*a up to n^2, costs ~1e-16 * 2 pi n absolute accuracy.
    """
    p = np.arange(n)
    return np.exp(-2j * math.pi * (np.outer(p, p) % n) / n)


def prior_apply(x: np.ndarray, lam: np.ndarray, power: float = 1.0) -> np.ndarray:
    """Apply C^power to every spatial field in x (shape [..., Nx*Ny])."""
    Nx, Ny = lam.shape
    X = x.reshape(-1, Nx, Ny)
    Wx = dft_matrix(Nx)
    Wy = dft_matrix(Ny)
    Xh = Wx @ X @ Wy.T                      # forward 2D DFT of each field
    Xh = Xh * (lam ** power)
    Y = np.conj(Wx) @ Xh @ np.conj(Wy).T    # inverse 2D DFT (times N)
    return (Y.real / (Nx * Ny)).reshape(x.shape)


def dense_prior(lam: np.ndarray, Lx: float = 1.0, Ly: float = 1.0) -> np.ndarray:
    """The explicit Nm x Nm matrix C[k1, k2] = (1/N) sum_k lambda_k cos(k . (x_k1 - x_k2))."""
    Nx, Ny = lam.shape
    N = Nx * Ny
    a = np.repeat(np.arange(Nx), Ny)          # grid index a of flat k
    b = np.tile(np.arange(Ny), Nx)
    da = a[:, None] - a[None, :]
    db = b[:, None] - b[None, :]
    C = np.zeros((N, N))
    for p in range(Nx):
        for q in range(Ny):
            C += lam[p, q] * np.cos(2.0 * math.pi * (p * da / Nx + q * db / Ny))
    return C / N


def gamma_pr_apply(x: np.ndarray, lam: np.ndarray, power: float = 1.0) -> np.ndarray:
    """Gamma_pr^power = I_Nt (x) C^power applied to time-major x [Nt, Nm] (or [..., Nt, Nm])."""
    return prior_apply(x, lam, power)
