"""Pins of the CPU oracle against facts fixed by the paper or by mathematics.

Each test checks the oracle against something other than itself: the explicit
matrices of the paper's block Toeplitz form, a library FFT, closed forms
(pointwise variance, the continuum Matern correlation), the parameter-space
MAP system (Woodbury), exact recovery on a square toy, nesting of windows,
and the exact covariance of the posterior sampler.
"""
import math

import numpy as np
import pytest
import scipy.special

import synth
from oracle import posterior as Q
from oracle import prior as P
from oracle import toeplitz as T

C1 = synth.CONFIGS[1]


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.fixture(scope="module")
def c1():
    F = synth.block_column(C1, "F")
    Fq = synth.block_column(C1, "Fq")
    lam = P.spectrum_for(C1)
    m_true, d, sigma = Q.synthetic_event(F, lam, synth.event_z(C1), synth.noise_z(C1))
    return dict(F=F, Fq=Fq, lam=lam, m_true=m_true, d=d, sigma=sigma)


def tiny_cfg(Nd=3, Nx=4, Ny=3, Nt=5, Nq=2):
    return synth.small_config(Nd=Nd, Nx=Nx, Ny=Ny, Nt=Nt, Nq=Nq, cid=91, ell=0.4)


# ------------------------------------------------------------------ Toeplitz

def test_direct_sum_equals_dense_block_toeplitz(c1):
    m = synth.white((C1.Nt, C1.Nm), 11)
    d = T.p2o_apply(c1["F"], m)
    dd = T.dense_p2o(c1["F"]) @ m.reshape(-1)
    assert _rel(d, dd) < 1e-14


def test_direct_sum_equals_fft_convolution(c1):
    # independent computation: zero-padded circular convolution with numpy.fft
    F, Nt = c1["F"], C1.Nt
    m = synth.white((Nt, C1.Nm), 12)
    L = 2 * Nt
    Fh = np.fft.rfft(F, n=L, axis=0)                     # [Nf, Nd, Nm]
    mh = np.fft.rfft(m, n=L, axis=0)                     # [Nf, Nm]
    yh = np.einsum("wsk,wk->ws", Fh, mh)
    d_fft = np.fft.irfft(yh, n=L, axis=0)[:Nt]
    assert _rel(T.p2o_apply(F, m), d_fft) < 1e-13


def test_impulse_response_is_block_column(c1):
    F = c1["F"]
    for j, k in [(0, 0), (0, 77), (5, 200)]:
        m = np.zeros((C1.Nt, C1.Nm))
        m[j, k] = 1.0
        d = T.p2o_apply(F, m)
        assert np.all(d[:j] == 0.0)
        np.testing.assert_allclose(d[j:], F[:C1.Nt - j, :, k], rtol=0, atol=0)


def test_single_step_is_plain_gemv(c1):
    F0 = c1["F"][:1]
    m = synth.white((1, C1.Nm), 13)
    np.testing.assert_allclose(T.p2o_apply(F0, m)[0], F0[0] @ m[0], rtol=1e-15)


def test_adjoint_identity_and_dense_transpose(c1):
    F = c1["F"]
    m = synth.white((C1.Nt, C1.Nm), 14)
    y = synth.white((C1.Nt, C1.Nd), 15)
    Fm = T.p2o_apply(F, m)
    Fty = T.p2o_adjoint(F, y)
    lhs, rhs = np.vdot(Fm, y), np.vdot(m, Fty)
    assert abs(lhs - rhs) / (np.linalg.norm(Fm) * np.linalg.norm(y)) < 1e-12
    assert _rel(Fty, T.dense_p2o(F).T @ y.reshape(-1)) < 1e-14


def test_entry_forms_match_full_applies(c1):
    F = c1["F"]
    m = synth.white((C1.Nt, C1.Nm), 16)
    y = synth.white((C1.Nt, C1.Nd), 17)
    d = T.p2o_apply(F, m)
    x = T.p2o_adjoint(F, y)
    rows = [0, 5]
    cols = [3, 100, 255]
    for i in [0, 7, C1.Nt - 1]:
        got = T.p2o_apply_entry(lambda l: F[l][rows], m, i)
        np.testing.assert_allclose(got, d[i, rows], rtol=1e-13)
    for j in [0, 9, C1.Nt - 1]:
        got = T.p2o_adjoint_entry(lambda l: F[l][:, cols], y, j)
        np.testing.assert_allclose(got, x[j, cols], rtol=1e-12, atol=1e-14)


# --------------------------------------------------------------------- prior

def test_prior_matches_library_fft2():
    cfg = synth.small_config(Nd=2, Nx=12, Ny=10, Nt=3, Nq=1)
    lam = P.spectrum_for(cfg)
    x = synth.white((cfg.Nt, cfg.Nm), 21)
    ref = np.fft.ifft2(np.fft.fft2(x.reshape(-1, 12, 10)) * lam).real.reshape(x.shape)
    for power in (1.0, 0.5, -1.0):
        ref = np.fft.ifft2(np.fft.fft2(x.reshape(-1, 12, 10)) * lam ** power).real
        assert _rel(P.prior_apply(x, lam, power), ref.reshape(x.shape)) < 1e-13


def test_prior_matches_library_fft2_at_full_grid_to_rounding():
    # the 200 x 250 grid of the 100-sensor workload: agreement to FP64 rounding
    cfg = synth.CONFIGS[2]
    lam = P.spectrum_for(cfg)
    x = synth.white((2, cfg.Nm), 24)
    ref = np.fft.ifft2(np.fft.fft2(x.reshape(-1, cfg.Nx, cfg.Ny)) * lam).real.reshape(x.shape)
    assert _rel(P.prior_apply(x, lam), ref) < 2e-15


def test_prior_dense_circulant_variance_and_spd(c1):
    lam = c1["lam"]
    C = P.dense_prior(lam)
    x = synth.white(C1.Nm, 22)
    assert _rel(P.prior_apply(x, lam), C @ x) < 1e-13
    np.testing.assert_allclose(np.diag(C), C1.var, rtol=1e-13)   # pointwise variance
    np.testing.assert_allclose(C, C.T, atol=1e-15)
    assert np.linalg.eigvalsh(C).min() > 0.0


def test_prior_constant_field_scaled_by_zero_mode(c1):
    lam = c1["lam"]
    one = np.ones(C1.Nm)
    np.testing.assert_allclose(P.prior_apply(one, lam), lam[0, 0] * one, rtol=1e-13)


def test_prior_square_root_squares(c1):
    lam = c1["lam"]
    x = synth.white((2, C1.Nm), 23)
    half = P.prior_apply(P.prior_apply(x, lam, 0.5), lam, 0.5)
    assert _rel(half, P.prior_apply(x, lam)) < 1e-13


def test_prior_matches_continuum_matern_correlation():
    # nu = 1 Matern covariance in 2D: c(r) = var * (kappa r) K_1(kappa r), kappa = sqrt(2 nu)/ell.
    cfg = synth.CONFIGS[2]
    lam = P.spectrum_for(cfg)
    e = np.zeros(cfg.Nm)
    e[0] = 1.0
    row = P.prior_apply(e, lam)
    kappa = math.sqrt(2.0 * cfg.nu) / cfg.ell
    for a in (2, 5, 10, 20, 40):
        r = a / cfg.Nx
        ref = kappa * r * scipy.special.kv(1, kappa * r)
        assert abs(row[a * cfg.Ny] / ref - 1.0) < 2e-3, (a, row[a * cfg.Ny], ref)
    for b in (5, 25, 50):
        r = b / cfg.Ny
        ref = kappa * r * scipy.special.kv(1, kappa * r)
        assert abs(row[b] / ref - 1.0) < 2e-3


# ----------------------------------------------------------------- posterior

def test_K_block_sum_equals_dense_product(c1):
    K = Q.form_K(c1["F"], c1["lam"], c1["sigma"] ** 2)
    Kd = Q.form_K_dense(c1["F"], c1["lam"], c1["sigma"] ** 2)
    assert _rel(K, Kd) < 1e-13
    np.testing.assert_allclose(K, K.T, rtol=0, atol=1e-12 * np.abs(K).max())


def test_noise_level_is_one_percent_of_rms(c1):
    d_clean = T.p2o_apply(c1["F"], c1["m_true"])
    assert c1["sigma"] == pytest.approx(0.01 * np.sqrt(np.mean(d_clean ** 2)), rel=1e-15)


@pytest.mark.parametrize("cfgname", ["tiny", "c1"])
def test_woodbury_data_space_equals_parameter_space(c1, cfgname):
    if cfgname == "tiny":
        cfg = synth.small_config(Nd=4, Nx=8, Ny=8, Nt=8, Nq=2, cid=92)
        F = synth.block_column(cfg, "F")
        lam = P.spectrum_for(cfg)
        _, d, sigma = Q.synthetic_event(F, lam, synth.event_z(cfg), synth.noise_z(cfg))
    else:
        cfg, F, lam, d, sigma = C1, c1["F"], c1["lam"], c1["d"], c1["sigma"]
    L = Q.cholesky(Q.form_K(F, lam, sigma ** 2))
    m_data, _ = Q.posterior_mean(F, lam, L, d, cfg.Nt)
    m_param = Q.map_parameter_space(F, lam, sigma ** 2, d)
    assert _rel(m_data, m_param) < 1e-9


def test_map_point_is_stationary(c1):
    # gradient of 1/2|Fm-d|^2/sigma^2 + 1/2|m|^2_{Gamma_pr^-1} vanishes at the MAP point
    F, lam, d, sigma = c1["F"], c1["lam"], c1["d"], c1["sigma"]
    L = Q.cholesky(Q.form_K(F, lam, sigma ** 2))
    m, _ = Q.posterior_mean(F, lam, L, d, C1.Nt)
    g_like = T.p2o_adjoint(F, T.p2o_apply(F, m) - d) / sigma ** 2
    g_prior = P.prior_apply(m, lam, -1.0)
    assert np.linalg.norm(g_like + g_prior) / np.linalg.norm(g_prior) < 1e-6


def test_exact_recovery_square_toy_without_noise():
    # Nd = Nm and an invertible lag-0 block: Gamma_pr F^T (F Gamma_pr F^T)^{-1} = F^{-1}.
    Nt, Nx, Ny = 6, 2, 2
    Nm = Nx * Ny
    g = synth.rng(424242)
    F = 0.3 * g.standard_normal((Nt, Nm, Nm)) / math.sqrt(Nm)
    F[0] = np.eye(Nm) + 0.1 * g.standard_normal((Nm, Nm)) / math.sqrt(Nm)
    lam = P.matern_spectrum(Nx, Ny, ell=0.5)
    m_true = g.standard_normal((Nt, Nm))
    d = T.p2o_apply(F, m_true)
    L = Q.cholesky(Q.form_K(F, lam, 0.0))
    m, _ = Q.posterior_mean(F, lam, L, d, Nt)
    assert _rel(m, m_true) < 1e-11


def test_windows_nest_and_match_fresh_subproblem(c1):
    F, lam, d, sigma = c1["F"], c1["lam"], c1["d"], c1["sigma"]
    K = Q.form_K(F, lam, sigma ** 2)
    L = Q.cholesky(K)
    for w in (1, 7, 20):
        n_w = C1.Nd * w
        Kw = Q.form_K(F, lam, sigma ** 2, Nt=w)
        np.testing.assert_allclose(K[:n_w, :n_w], Kw, rtol=0, atol=1e-13 * np.abs(K).max())
        Lw = Q.cholesky(Kw)
        np.testing.assert_allclose(L[:n_w, :n_w], Lw, rtol=0, atol=1e-10 * np.abs(L).max())
        m_nest, _ = Q.posterior_mean(F, lam, L, d, C1.Nt, nt_window=w)
        m_fresh, _ = Q.posterior_mean(F[:w], lam, Lw, d[:w], w)
        assert np.all(m_nest[w:] == 0.0)
        assert _rel(m_nest[:w], m_fresh) < 1e-10


@pytest.mark.parametrize("w", [5, 3])
def test_sampler_covariance_equals_posterior_covariance(w):
    cfg = tiny_cfg()
    F = synth.block_column(cfg, "F")
    lam = P.spectrum_for(cfg)
    _, d, sigma = Q.synthetic_event(F, lam, synth.event_z(cfg), synth.noise_z(cfg))
    L = Q.cholesky(Q.form_K(F, lam, sigma ** 2))
    n_m, n_d = cfg.Nt * cfg.Nm, w * cfg.Nd
    zero_m, zero_n = np.zeros((cfg.Nt, cfg.Nm)), np.zeros((w, cfg.Nd))
    mean = Q.posterior_sample(F, lam, L, sigma, d, zero_m, zero_n, w)
    m_map, _ = Q.posterior_mean(F, lam, L, d, cfg.Nt, nt_window=w)
    assert _rel(mean, m_map) < 1e-10
    A_m = np.zeros((n_m, n_m))
    for i in range(n_m):
        z = zero_m.copy()
        z.flat[i] = 1.0
        A_m[:, i] = (Q.posterior_sample(F, lam, L, sigma, d, z, zero_n, w) - mean).ravel()
    A_n = np.zeros((n_m, n_d))
    for i in range(n_d):
        z = zero_n.copy()
        z.flat[i] = 1.0
        A_n[:, i] = (Q.posterior_sample(F, lam, L, sigma, d, zero_m, z, w) - mean).ravel()
    cov = A_m @ A_m.T + A_n @ A_n.T
    # windowed posterior covariance from the parameter-space Hessian of the first w block rows
    Fd = T.dense_p2o(F)[:n_d]
    H = Fd.T @ Fd / sigma ** 2 + np.kron(np.eye(cfg.Nt), P.dense_prior(1.0 / lam))
    post = np.linalg.inv(H)
    assert np.abs(cov - post).max() / np.abs(post).max() < 1e-9


def test_forecast_matches_dense_p2q(c1):
    m = synth.white((C1.Nt, C1.Nm), 31)
    q = Q.forecast(c1["Fq"], m)
    assert _rel(q, T.dense_p2o(c1["Fq"]) @ m.reshape(-1)) < 1e-14
    assert q.shape == (C1.Nt, C1.Nq)


# ------------------------------------------------------- Phase 3: QoI map and covariance

from oracle import qoi as QO  # noqa: E402


@pytest.fixture(scope="module")
def tiny_qoi():
    cfg = synth.small_config(Nd=4, Nx=8, Ny=8, Nt=8, Nq=2, cid=92)
    F = synth.block_column(cfg, "F")
    Fq = synth.block_column(cfg, "Fq")
    lam = P.spectrum_for(cfg)
    _, d, sigma = Q.synthetic_event(F, lam, synth.event_z(cfg), synth.noise_z(cfg))
    L = Q.cholesky(Q.form_K(F, lam, sigma ** 2))
    return dict(cfg=cfg, F=F, Fq=Fq, lam=lam, d=d, sigma=sigma, L=L)


def test_qoi_map_reproduces_forecast_of_posterior_mean(c1):
    # Phase 4: q_map = F_q m_map = Q d, for the event and for an unrelated data vector
    F, Fq, lam, sigma = c1["F"], c1["Fq"], c1["lam"], c1["sigma"]
    L = Q.cholesky(Q.form_K(F, lam, sigma ** 2))
    Qm = QO.qoi_map(F, Fq, lam, L)
    for d in (c1["d"], synth.white((C1.Nt, C1.Nd), 4242)):
        m, _ = Q.posterior_mean(F, lam, L, d, C1.Nt)
        assert _rel(Qm @ d.ravel(), Q.forecast(Fq, m).ravel()) < 1e-11


def test_qoi_map_equals_parameter_space_definition(tiny_qoi):
    t = tiny_qoi
    Qd = QO.qoi_map(t["F"], t["Fq"], t["lam"], t["L"])
    Qp = QO.qoi_map_dense(t["F"], t["Fq"], t["lam"], t["sigma"] ** 2)
    assert _rel(Qd, Qp) < 1e-9


def test_qoi_covariance_equals_parameter_space_definition(tiny_qoi):
    t = tiny_qoi
    Cd = QO.qoi_covariance(t["F"], t["Fq"], t["lam"], t["L"])
    Cp = QO.qoi_covariance_dense(t["F"], t["Fq"], t["lam"], t["sigma"] ** 2)
    assert _rel(Cd, Cp) < 1e-8


def test_qoi_covariance_symmetric_positive_and_below_prior(tiny_qoi):
    t = tiny_qoi
    W, Y, C = QO.qoi_columns(t["F"], t["Fq"], t["lam"], t["L"])
    G = C - W @ Y.T
    assert _rel(G, G.T) < 1e-10
    assert np.linalg.eigvalsh(0.5 * (G + G.T)).min() > 0.0
    assert np.all(np.diag(G) <= np.diag(C) * (1 + 1e-12))     # data never add variance
