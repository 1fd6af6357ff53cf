"""Full-size (Nd=100, 200x250 grid, Nt=400, Nq=20) checks in the benchmark's launch configuration.

The oracle cannot form the 40,000 x 40,000 K on the CPU in test time, so at
this size the tests compare outputs the oracle can compute one by one
(entries of F m, F^T y, F_q m, single time steps of the prior), the
posterior mean of an observation window the oracle can factor
(Nt' = 12, n' = 1,200), and properties that hold at any size: the adjoint
identity and the MAP stationarity  m = Gamma_pr F^T (d - F m) / sigma^2.
"""
import json
import os

import numpy as np
import pytest

import synth
from oracle import posterior as Q
from oracle import prior as P
from oracle import toeplitz as T

from gpu_util import make_context, rel

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CFG = synth.CONFIGS[2]


@pytest.fixture(scope="module")
def c2():
    import torch
    from paper_2504_16344_gb300 import tw
    sigma = json.load(open(os.path.join(HERE, "golden", "sigma_c2.json")))["sigma"]
    d = np.load(os.path.join(HERE, "golden", "event_c2.npy"))
    ctx = make_context(CFG, keep=tw.KEEP_FP64 | tw.KEEP_C64 | tw.KEEP_BF16X2,
                       on_device_columns=True, chunk_rows=10)
    ctx.factor_K(sigma ** 2)
    yield dict(ctx=ctx, sigma=sigma, d=d, lam=P.spectrum_for(CFG), dev=torch.device("cuda", 0))
    ctx.close()


def _t(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def _rows(rows):
    return lambda lag: synth.block_column(CFG, "F", rows=rows, lags=[lag])[0]


def test_sampled_forward_entries(c2):
    from paper_2504_16344_gb300 import tw
    m = synth.white((CFG.Nt, CFG.Nm), 2001)
    d = c2["ctx"].p2o_apply(tw.MAP_F, tw.PREC_FP64, _t(m, c2["dev"]))[0].cpu().numpy()
    for i, rows in [(0, [0, 99]), (137, [3, 64]), (399, [17, 98, 99])]:
        ref = T.p2o_apply_entry(_rows(rows), m, i)
        assert rel(d[i, rows], ref) < 1e-11


def test_sampled_adjoint_entries(c2):
    from paper_2504_16344_gb300 import tw
    y = synth.white((CFG.Nt, CFG.Nd), 2002)
    x = c2["ctx"].p2o_adjoint(tw.MAP_F, tw.PREC_FP64, _t(y, c2["dev"]))[0].cpu().numpy()
    cols = [0, 777, 49_999]
    for j in (0, 211, 399):
        ref = T.p2o_adjoint_entry(lambda lag: synth.block_column(CFG, "F", lags=[lag], cols=cols)[0], y, j)
        assert rel(x[j, cols], ref) < 1e-11


def test_sampled_forecast_entries(c2):
    from paper_2504_16344_gb300 import tw
    m = synth.white((CFG.Nt, CFG.Nm), 2003)
    q = c2["ctx"].forecast(tw.PREC_FP64, _t(m, c2["dev"]))[0].cpu().numpy()
    for i in (5, 399):
        ref = T.p2o_apply_entry(lambda lag: synth.block_column(CFG, "Fq", lags=[lag])[0], m, i)
        assert rel(q[i], ref) < 1e-11


def test_prior_single_steps(c2):
    x = synth.white((CFG.Nt, CFG.Nm), 2004)
    y = c2["ctx"].prior_apply(_t(x, c2["dev"]))[0].cpu().numpy()
    for t in (0, 199, 399):
        assert rel(y[t], P.prior_apply(x[t], c2["lam"])) < 1e-11


def test_adjoint_identity_fullsize(c2):
    from paper_2504_16344_gb300 import tw
    m = synth.white((CFG.Nt, CFG.Nm), 2005)
    y = synth.white((CFG.Nt, CFG.Nd), 2006)
    Fm = c2["ctx"].p2o_apply(tw.MAP_F, tw.PREC_FP64, _t(m, c2["dev"]))[0].cpu().numpy()
    Fty = c2["ctx"].p2o_adjoint(tw.MAP_F, tw.PREC_FP64, _t(y, c2["dev"]))[0].cpu().numpy()
    gap = abs(np.vdot(Fm, y) - np.vdot(m, Fty)) / (np.linalg.norm(Fm) * np.linalg.norm(y))
    assert gap < 1e-12


def test_windowed_posterior_mean_matches_oracle(c2):
    from paper_2504_16344_gb300 import tw
    w = 12
    Fw = synth.block_column(CFG, "F", lags=range(w))            # [w][Nd][Nm]
    Kw = Q.form_K(Fw, c2["lam"], c2["sigma"] ** 2)
    m_ref, _ = Q.posterior_mean(Fw, c2["lam"], Q.cholesky(Kw), c2["d"][:w], w)
    m = c2["ctx"].infer(tw.PREC_FP64, _t(c2["d"], c2["dev"]), windows=[w])[0].cpu().numpy()
    c2["ctx"].check()
    assert np.all(m[w:] == 0.0)
    err = rel(m[:w], m_ref)
    print(f"window {w}: FP64 m rel err {err:.2e}")
    assert err < 1e-11


def _stationarity(ctx, d, m, sigma, prec):
    import torch
    from paper_2504_16344_gb300 import tw
    Fm = ctx.p2o_apply(tw.MAP_F, prec, m)
    r = (d - Fm) / sigma ** 2
    g = ctx.prior_apply(ctx.p2o_adjoint(tw.MAP_F, prec, r))
    return float(torch.linalg.norm(g - m) / torch.linalg.norm(m))


def test_full_window_map_stationarity_and_mixed_agreement(c2):
    from paper_2504_16344_gb300 import tw
    ctx, dev = c2["ctx"], c2["dev"]
    d = _t(c2["d"], dev).unsqueeze(0)
    m64, st = ctx.infer(tw.PREC_FP64, d, stats=True)
    s64 = _stationarity(ctx, d, m64, c2["sigma"], tw.PREC_FP64)
    print(f"FP64: stationarity {s64:.2e} residual {st.resid_rel:.2e}")
    assert s64 < 1e-6
    q64 = ctx.forecast(tw.PREC_FP64, m64)
    for prec in (tw.PREC_C64, tw.PREC_BF16X2):
        for solver in (0, 1):
            ctx.set_solver(solver)
            m32, st32 = ctx.infer(prec, d, stats=True)
            ctx.set_solver(0)
            q32 = ctx.forecast(prec, m32)
            em = rel(m32.cpu().numpy(), m64.cpu().numpy())
            eq = rel(q32.cpu().numpy(), q64.cpu().numpy())
            print(f"prec {prec} solver {solver}: m vs FP64 {em:.2e}, q vs FP64 {eq:.2e}, "
                  f"residual {st32.resid_rel:.2e}, refinement steps {ctx.refinement_steps()}")
            assert em < 1e-5 and eq < 5e-5
    ctx.check()
