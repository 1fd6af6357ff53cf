"""Data-space posterior mean, forecast, windows and samples (oracle, FP64).

Test infrastructure only (see the package docstring).

Definitions (Sec. "State of the art" and Sec. "Real-time Bayesian inference
and prediction framework" of arXiv 2504.16344), with m_prior = 0:

* noise covariance Gamma_n = sigma^2 I (one sigma for the whole network; the
  synthetic data carry 1% relative noise, sigma = 0.01 rms(F m_true));
* data-space Hessian K = Gamma_n + F Gamma_pr F*, time-major, formed as the
  plain block product that only skips F's zero blocks:
      K_(i,j) = sigma^2 delta_ij I + sum_{s=0}^{min(i,j)} F_{i-s} C F_{j-s}^T;
* K = L L^T (Cholesky), y = K^{-1} d, posterior mean m = Gamma_pr F* y, and
  forecast q = F_q m (Phase 4);
* parameter-space MAP system (Eq. mmap-problem):
      (F* Gamma_n^{-1} F + Gamma_pr^{-1}) m = F* Gamma_n^{-1} d,
  and posterior covariance Gamma_post = H^{-1} (Eq. Hessian); the two are
  equal by the Sherman-Morrison-Woodbury identity of Phase 2;
* observation window Nt' <= Nt: the data are the leading Nt' blocks of d, the
  map F' is the leading Nt' block rows of F, and K' = K[:n', :n'] with
  n' = Nd Nt' (Cholesky factors nest, so L' = L[:n', :n']);
* posterior sample (perturb-then-condition, exact for a linear-Gaussian
  model): s = m_pr + Gamma_pr F'* K'^{-1} (d' - F' m_pr - sigma z_n) with
  m_pr = Gamma_pr^{1/2} z_m, whose covariance is Gamma_post.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from .prior import prior_apply, dense_prior
from .toeplitz import dense_p2o, p2o_adjoint, p2o_apply


# --------------------------------------------------------------------------- K

def block_products(Fcol: np.ndarray, lam: np.ndarray, Nt: int | None = None) -> np.ndarray:
    """P[u*Nd + a, v*Nd + b] = (F_u C F_v^T)[a, b] for u, v < Nt."""
    Nt = Fcol.shape[0] if Nt is None else Nt
    _, Nd, Nm = Fcol.shape
    Phi = Fcol[:Nt].reshape(Nt * Nd, Nm)
    # rows F_u C (C is symmetric), filtered a bounded number of rows at a time
    # (each row's filter is independent; this only limits host memory)
    H = np.empty_like(Phi)
    for r0 in range(0, Phi.shape[0], 512):
        H[r0:r0 + 512] = prior_apply(Phi[r0:r0 + 512], lam)
    return H @ Phi.T


def form_K(Fcol: np.ndarray, lam: np.ndarray, sigma2: float, Nt: int | None = None) -> np.ndarray:
    """K = sigma^2 I + F Gamma_pr F^T for the leading Nt blocks (time-major)."""
    Nt = Fcol.shape[0] if Nt is None else Nt
    Nd = Fcol.shape[1]
    P = block_products(Fcol, lam, Nt)
    K = np.zeros((Nt * Nd, Nt * Nd))
    for i in range(Nt):
        for j in range(Nt):
            acc = np.zeros((Nd, Nd))
            for s in range(min(i, j) + 1):
                u, v = i - s, j - s
                acc += P[u * Nd:(u + 1) * Nd, v * Nd:(v + 1) * Nd]
            K[i * Nd:(i + 1) * Nd, j * Nd:(j + 1) * Nd] = acc
    K[np.diag_indices_from(K)] += sigma2
    return K


def form_K_dense(Fcol: np.ndarray, lam: np.ndarray, sigma2: float) -> np.ndarray:
    """K from the explicit dense F and Gamma_pr = I (x) C (small cases only)."""
    Nt = Fcol.shape[0]
    F = dense_p2o(Fcol)
    G = np.kron(np.eye(Nt), dense_prior(lam))
    return sigma2 * np.eye(F.shape[0]) + F @ G @ F.T


def cholesky(K: np.ndarray) -> np.ndarray:
    """Lower Cholesky factor (library primitive)."""
    return np.linalg.cholesky(K)


def solve_K(L: np.ndarray, rhs: np.ndarray) -> np.ndarray:
    """y = (L L^T)^{-1} rhs; rhs flat [n] or [n, k]."""
    t = scipy.linalg.solve_triangular(L, rhs, lower=True)
    return scipy.linalg.solve_triangular(L.T, t, lower=False)


# ---------------------------------------------------------------- Phase 4

def posterior_mean(Fcol, lam: np.ndarray, L: np.ndarray, d: np.ndarray,
                   Nt: int, nt_window: int | None = None):
    """m = Gamma_pr F'^T K'^{-1} d' for window Nt' (default Nt).

    d: [>=Nt', Nd] time-major data (rows >= Nt' ignored).  Returns
    (m [Nt, Nm], y [Nt', Nd]); rows t >= Nt' of m equal the prior mean 0.
    """
    w = Nt if nt_window is None else nt_window
    Nd = d.shape[1]
    n_w = Nd * w
    y = solve_K(L[:n_w, :n_w], d[:w].reshape(n_w)).reshape(w, Nd)
    x = p2o_adjoint(Fcol, y)              # lags 0..w-1 only
    m = np.zeros((Nt, x.shape[1]))
    m[:w] = prior_apply(x, lam)
    return m, y


def forecast(Fqcol, m: np.ndarray) -> np.ndarray:
    """q = F_q m over all Nt steps.  m: [Nt, Nm] -> q: [Nt, Nq]."""
    return p2o_apply(Fqcol, m)


def noise_sigma(d_clean: np.ndarray, rel: float = 0.01) -> float:
    """sigma = rel * rms over all entries of the noise-free data F m_true."""
    return rel * float(np.sqrt(np.mean(d_clean * d_clean)))


def synthetic_event(Fcol, lam: np.ndarray, z: np.ndarray, z_n: np.ndarray,
                    sigma: float | None = None, rel: float = 0.01):
    """m_true = Gamma_pr^{1/2} z, d = F m_true + sigma z_n.

    Returns (m_true, d, sigma); sigma defaults to rel * rms(F m_true).
    """
    m_true = prior_apply(z, lam, 0.5)
    d_clean = p2o_apply(Fcol, m_true)
    if sigma is None:
        sigma = noise_sigma(d_clean, rel)
    return m_true, d_clean + sigma * z_n, sigma


def posterior_sample(Fcol, lam: np.ndarray, L: np.ndarray, sigma: float,
                     d: np.ndarray, z_m: np.ndarray, z_n: np.ndarray,
                     nt_window: int | None = None) -> np.ndarray:
    """s = m_pr + Gamma_pr F'^T K'^{-1} (d' - F' m_pr - sigma z_n), m_pr = Gamma_pr^{1/2} z_m."""
    Nt = z_m.shape[0]
    w = Nt if nt_window is None else nt_window
    Nd = d.shape[1]
    m_pr = prior_apply(z_m, lam, 0.5)
    r = d[:w] - p2o_apply(Fcol, m_pr[:w]) - sigma * z_n[:w]
    n_w = Nd * w
    y = solve_K(L[:n_w, :n_w], r.reshape(n_w)).reshape(w, Nd)
    x = p2o_adjoint(Fcol, y)
    s = m_pr.copy()
    s[:w] += prior_apply(x, lam)
    return s


# ------------------------------------------------- parameter-space cross-check

def hessian_dense(Fcol: np.ndarray, lam: np.ndarray, sigma2: float) -> np.ndarray:
    """H = F^T Gamma_n^{-1} F + Gamma_pr^{-1} (Eq. Hessian), dense."""
    Nt = Fcol.shape[0]
    F = dense_p2o(Fcol)
    Cinv = dense_prior(1.0 / lam)
    return F.T @ F / sigma2 + np.kron(np.eye(Nt), Cinv)


def map_parameter_space(Fcol: np.ndarray, lam: np.ndarray, sigma2: float,
                        d: np.ndarray) -> np.ndarray:
    """Solve (F^T Gamma_n^{-1} F + Gamma_pr^{-1}) m = F^T Gamma_n^{-1} d (Eq. mmap-problem)."""
    Nt, _, Nm = Fcol.shape
    F = dense_p2o(Fcol)
    H = hessian_dense(Fcol, lam, sigma2)
    m = np.linalg.solve(H, F.T @ d.reshape(-1) / sigma2)
    return m.reshape(Nt, Nm)


def posterior_covariance_dense(Fcol: np.ndarray, lam: np.ndarray, sigma2: float) -> np.ndarray:
    """Gamma_post = H^{-1} (Eq. Hessian), dense."""
    return np.linalg.inv(hessian_dense(Fcol, lam, sigma2))


def condition_number_K(K: np.ndarray) -> float:
    """2-norm condition number of K from its extreme eigenvalues (symmetric)."""
    ev = np.linalg.eigvalsh(K)
    return float(ev[-1] / ev[0])
