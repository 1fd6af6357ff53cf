"""GPU parity of K's factorisation, the posterior mean, windows and the forecast.

The oracle forms K by the block product, factors it with LAPACK and solves;
the GPU forms K as G G^T plus block-diagonal prefix sums, factors it in
FP64 (FP64 path) or FP32 + FP64-residual refinement (mixed path).
Tolerances: FP64 path 1e-11 relative L2 on m and q (the oracle's own error
against an extended-precision refinement is 3e-13 .. 3e-12 on these sizes,
so 1e-11 leaves room for both); complex64 path 1e-5 on m and q; bf16 hi+lo
storage 1e-5 or twice its rounded-operator floor.
"""
import json
import os

import numpy as np
import pytest

import synth
from oracle import posterior as Q
from oracle import prior as P
from oracle import toeplitz as T

from gpu_util import adjoint_rounded, make_context, mixed_bound, rel

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
SIGMA_C1 = json.load(open(os.path.join(HERE, "golden", "sigma_c1.json")))["sigma"]

CASES = {
    "c1": synth.CONFIGS[1],
    # n = 800: 12.5 blocks of 64 -> ragged last block
    "mid": synth.small_config(Nd=20, Nx=40, Ny=50, Nt=40, Nq=5, cid=84),
    # n = 2002 (odd Nt, Nd not a divisor of 64)
    "wide": synth.small_config(Nd=26, Nx=60, Ny=75, Nt=77, Nq=3, cid=85),
    # the 316 x 316 grid of the serving workload (prior filter with radix-79 passes)
    "grid316": synth.small_config(Nd=4, Nx=316, Ny=316, Nt=6, Nq=2, cid=87),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    import torch
    from paper_2504_16344_gb300 import tw
    cfg = CASES[request.param]
    F = synth.block_column(cfg, "F")
    Fq = synth.block_column(cfg, "Fq")
    lam = P.spectrum_for(cfg)
    if request.param == "c1":
        m_true, d, sigma = Q.synthetic_event(F, lam, synth.event_z(cfg), synth.noise_z(cfg), SIGMA_C1)
    else:
        m_true, d, sigma = Q.synthetic_event(F, lam, synth.event_z(cfg), synth.noise_z(cfg))
    K = Q.form_K(F, lam, sigma ** 2)
    L = Q.cholesky(K)
    ctx = make_context(cfg, keep=tw.KEEP_FP64 | tw.KEEP_C64 | tw.KEEP_BF16X2)
    ctx.factor_K(sigma ** 2)
    yield dict(cfg=cfg, ctx=ctx, F=F, Fq=Fq, lam=lam, d=d, sigma=sigma, K=K, L=L,
               dev=torch.device("cuda", 0))
    ctx.close()


def _t(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def test_K_apply_matches_oracle(case):
    cfg, ctx = case["cfg"], case["ctx"]
    x = synth.white((cfg.Nt, cfg.Nd), 3001)
    got = ctx.apply_K(_t(x, case["dev"]))[0].cpu().numpy()
    err = rel(got, case["K"] @ x.ravel())
    print(f"{cfg.cid}: K x rel err {err:.2e}")
    assert err < 1e-13


def test_solve_K_matches_oracle(case):
    from paper_2504_16344_gb300 import tw
    cfg, ctx = case["cfg"], case["ctx"]
    y_ref = Q.solve_K(case["L"], case["d"].ravel())
    y = ctx.solve_K(tw.PREC_FP64, _t(case["d"], case["dev"]))[0].cpu().numpy()
    # m from the oracle's y through the GPU applies (isolates the apply stage)
    m_ref, _ = Q.posterior_mean(case["F"], case["lam"], case["L"], case["d"], cfg.Nt)
    m_via = ctx.prior_apply(ctx.p2o_adjoint(tw.MAP_F, tw.PREC_FP64, _t(y_ref.reshape(cfg.Nt, cfg.Nd), case["dev"])))
    ey, em = rel(y, y_ref), rel(m_via[0].cpu().numpy(), m_ref)
    print(f"{cfg.cid}: y rel err {ey:.2e}; m from oracle y through GPU applies {em:.2e}")
    assert em < 1e-11


def test_posterior_mean_fp64_full_window(case):
    from paper_2504_16344_gb300 import tw
    cfg = case["cfg"]
    m_ref, _ = Q.posterior_mean(case["F"], case["lam"], case["L"], case["d"], cfg.Nt)
    m, st = case["ctx"].infer(tw.PREC_FP64, _t(case["d"], case["dev"]), stats=True)
    case["ctx"].check()
    err = rel(m[0].cpu().numpy(), m_ref)
    print(f"{cfg.cid}: FP64 m rel err {err:.2e}")
    assert err < 1e-11


@pytest.mark.parametrize("frac", [0.03, 0.25, 0.5, 0.77])
def test_posterior_mean_fp64_windows(case, frac):
    from paper_2504_16344_gb300 import tw
    cfg = case["cfg"]
    w = max(1, int(round(frac * cfg.Nt)))
    m_ref, _ = Q.posterior_mean(case["F"], case["lam"], case["L"], case["d"], cfg.Nt, nt_window=w)
    m = case["ctx"].infer(tw.PREC_FP64, _t(case["d"], case["dev"]), windows=[w])[0].cpu().numpy()
    case["ctx"].check()
    assert np.all(m[w:] == 0.0)
    assert rel(m, m_ref) < 1e-11


def test_batched_uneven_windows_equal_single_calls(case):
    from paper_2504_16344_gb300 import tw
    cfg = case["cfg"]
    ws = [cfg.Nt, max(1, cfg.Nt // 3), max(1, cfg.Nt // 2 + 1)]
    d3 = np.stack([case["d"], case["d"] * 0.5, -case["d"]])
    mb = case["ctx"].infer(tw.PREC_FP64, _t(d3, case["dev"]), windows=ws).cpu().numpy()
    for r, w in enumerate(ws):
        m_ref, _ = Q.posterior_mean(case["F"], case["lam"], case["L"], d3[r], cfg.Nt, nt_window=w)
        assert rel(mb[r], m_ref) < 1e-11


def test_forecast_of_posterior_mean(case):
    from paper_2504_16344_gb300 import tw
    cfg, ctx = case["cfg"], case["ctx"]
    m_ref, _ = Q.posterior_mean(case["F"], case["lam"], case["L"], case["d"], cfg.Nt)
    q_ref = Q.forecast(case["Fq"], m_ref)
    m = ctx.infer(tw.PREC_FP64, _t(case["d"], case["dev"]))
    q = ctx.forecast(tw.PREC_FP64, m)[0].cpu().numpy()
    ctx.check()
    assert rel(q, q_ref) < 1e-11


@pytest.mark.parametrize("solver", [0, 1])
@pytest.mark.parametrize("prec", [1, 2])
def test_posterior_mean_mixed_precision(case, prec, solver):
    # solver 0: FP64 factor; 1: FP32 factor + FP64-residual refinement
    from paper_2504_16344_gb300 import tw
    cfg, ctx = case["cfg"], case["ctx"]
    m_ref, _ = Q.posterior_mean(case["F"], case["lam"], case["L"], case["d"], cfg.Nt)
    q_ref = Q.forecast(case["Fq"], m_ref)
    ctx.set_solver(solver)
    try:
        m, st = ctx.infer(prec, _t(case["d"], case["dev"]), stats=True)
        q = ctx.forecast(prec, m)[0].cpu().numpy()
        q64 = ctx.forecast(tw.PREC_FP64, m)[0].cpu().numpy()
    finally:
        ctx.set_solver(0)
    ctx.check()
    em, eq, eq64 = rel(m[0].cpu().numpy(), m_ref), rel(q, q_ref), rel(q64, q_ref)
    print(f"{cfg.cid}: prec {prec} solver {solver} ir {ctx.refinement_steps()} m err {em:.2e} "
          f"q err {eq:.2e} (FP64 forecast of this m: {eq64:.2e}) resid {st.resid_rel:.2e}")
    assert st.resid_rel < 1e-10
    if prec == 1:
        assert em < 1e-5 and eq < 1e-5
    else:
        # bf16 hi+lo storage: 1e-5 or twice its rounded-operator floor
        _, y = Q.posterior_mean(case["F"], case["lam"], case["L"], case["d"], cfg.Nt)
        m_fl = P.prior_apply(adjoint_rounded(case["F"], y, "BF16X2"), case["lam"])
        fl, flq = rel(m_fl, m_ref), rel(T.p2o_apply(case["Fq"], m_fl), q_ref)
        print(f"{cfg.cid}: bf16x2 floors m {fl:.2e} q {flq:.2e}")
        assert em < mixed_bound(fl) and eq < mixed_bound(flq)


def test_solve_residual_certificate_fp64(case):
    # backward-stable solve: |d - K y| / |d| small (the oracle's own: 2e-14 .. 3e-13)
    from paper_2504_16344_gb300 import tw
    cfg, ctx = case["cfg"], case["ctx"]
    _, st = ctx.infer(tw.PREC_FP64, _t(case["d"], case["dev"]), stats=True)
    print(f"{cfg.cid}: FP64 residual {st.resid_rel:.2e}")
    assert 0.0 <= st.resid_rel < 1e-11


@pytest.mark.parametrize("frac", [1.0, 0.4])
def test_posterior_samples_match_oracle(case, frac):
    # same draws on both sides: the perturb-then-condition sample is deterministic given z
    cfg, ctx = case["cfg"], case["ctx"]
    w = max(1, int(round(frac * cfg.Nt)))
    zs = [synth.sample_z(cfg, k, cfg.Nt) for k in range(2)]
    z_m = np.stack([z[0] for z in zs])
    z_n = np.stack([z[1] for z in zs])
    d2 = np.stack([case["d"], case["d"]])
    got = ctx.sample_posterior(_t(d2, case["dev"]), _t(z_m, case["dev"]), _t(z_n, case["dev"]),
                               case["sigma"], windows=[w, w]).cpu().numpy()
    ctx.check()
    for k in range(2):
        ref = Q.posterior_sample(case["F"], case["lam"], case["L"], case["sigma"], case["d"],
                                 z_m[k], z_n[k], w)
        m_pr = P.prior_apply(z_m[k], case["lam"], 0.5)
        err = rel(got[k], ref)
        err_c = rel(got[k] - m_pr, ref - m_pr)      # the conditioning update alone
        print(f"{cfg.cid}: sample {k} window {w} rel err {err:.2e}, update {err_c:.2e}")
        assert err < 1e-11 and err_c < 1e-10
