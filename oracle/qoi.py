"""Data-to-QoI map and QoI posterior covariance (oracle, FP64).

Test infrastructure only (see the package docstring).

Phase 3 of the paper's framework precomputes, for the QoI q = F_q m,
  * the posterior covariance of the QoI, Gamma_post(q) = F_q Gamma_post F_q^*,
  * the data-to-QoI map Q = F_q Gamma_post F^* Gamma_n^{-1},
so that Phase 4 predicts q = Q d directly from data (Sec. "Real-time Bayesian
inference and prediction framework", Phases 3 and 4; the predictive
distribution of q is N(F_q m_map, F_q Gamma_post F_q^*), Sec. "State of the
art").  With the data-space Hessian K = Gamma_n + F Gamma_pr F^* (Phase 2)
the Woodbury form Gamma_post = Gamma_pr - Gamma_pr F^* K^{-1} F Gamma_pr gives
  Q = F_q Gamma_pr F^* K^{-1}                       (push-through identity),
  Gamma_post(q) = F_q Gamma_pr F_q^* - W^T K^{-1} W,  W = F Gamma_pr F_q^*.
Both are formed here column by column from the QoI unit vectors, as the paper
does (Nq Nt actions on unit vectors), with the oracle's own applies and
solves.  The dense parameter-space forms (`*_dense`) are the definitions
written out, for tiny cases.  Indices: QoI entry j = t*Nq + i, data entry
t*Nd + s (time-major, as K).
"""
from __future__ import annotations

import numpy as np

from .posterior import solve_K
from .prior import dense_prior, prior_apply
from .toeplitz import dense_p2o, p2o_adjoint, p2o_apply


def _unit(Nt: int, R: int, j: int) -> np.ndarray:
    e = np.zeros((Nt, R))
    e[j // R, j % R] = 1.0
    return e


def qoi_columns(Fcol, Fqcol, lam: np.ndarray, L: np.ndarray):
    """For every QoI unit vector e_j: (w_j = F Gamma_pr F_q^T e_j, K^{-1} w_j, F_q Gamma_pr F_q^T e_j).

    Returns W [Nq Nt, Nd Nt], Y [Nq Nt, Nd Nt] (rows), Cqq [Nq Nt, Nq Nt].
    """
    Nt, Nd, _ = Fcol.shape
    Nq = Fqcol.shape[1]
    nq, n = Nq * Nt, Nd * Nt
    W = np.zeros((nq, n))
    Y = np.zeros((nq, n))
    C = np.zeros((nq, nq))
    for j in range(nq):
        u = prior_apply(p2o_adjoint(Fqcol, _unit(Nt, Nq, j)), lam)   # Gamma_pr F_q^T e_j
        w = p2o_apply(Fcol, u).ravel()
        W[j] = w
        Y[j] = solve_K(L, w)
        C[:, j] = p2o_apply(Fqcol, u).ravel()
    return W, Y, C


def qoi_map(Fcol, Fqcol, lam: np.ndarray, L: np.ndarray) -> np.ndarray:
    """Q = F_q Gamma_pr F^T K^{-1}, [Nq Nt, Nd Nt]: row j is (K^{-1} F Gamma_pr F_q^T e_j)^T (K symmetric)."""
    return qoi_columns(Fcol, Fqcol, lam, L)[1]


def qoi_covariance(Fcol, Fqcol, lam: np.ndarray, L: np.ndarray) -> np.ndarray:
    """Gamma_post(q) = F_q Gamma_pr F_q^T - W^T K^{-1} W, [Nq Nt, Nq Nt]."""
    W, Y, C = qoi_columns(Fcol, Fqcol, lam, L)
    return C - W @ Y.T


def qoi_map_dense(Fcol, Fqcol, lam: np.ndarray, sigma2: float) -> np.ndarray:
    """Q = F_q Gamma_post F^T Gamma_n^{-1} with Gamma_post = (F^T F / sigma2 + Gamma_pr^{-1})^{-1}, dense."""
    F, Fq = dense_p2o(Fcol), dense_p2o(Fqcol)
    Nt = Fcol.shape[0]
    Cinv = np.kron(np.eye(Nt), dense_prior(1.0 / lam))
    H = F.T @ F / sigma2 + Cinv
    return Fq @ np.linalg.solve(H, F.T) / sigma2


def qoi_covariance_dense(Fcol, Fqcol, lam: np.ndarray, sigma2: float) -> np.ndarray:
    """F_q Gamma_post F_q^T with Gamma_post the inverse of the parameter-space Hessian, dense."""
    F, Fq = dense_p2o(Fcol), dense_p2o(Fqcol)
    Nt = Fcol.shape[0]
    Cinv = np.kron(np.eye(Nt), dense_prior(1.0 / lam))
    H = F.T @ F / sigma2 + Cinv
    return Fq @ np.linalg.solve(H, Fq.T)
