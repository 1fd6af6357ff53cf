"""GPU parity with G^ = F^ C kept (the paper's G* = Gamma_pr F*, Phase 2).

With TW_KEEP_G the posterior mean is one adjoint apply of G* (no prior filter
online) on the FP64 and complex64 paths; the bf16x2 path keeps F* + prior.
Results must match the oracle as the F* + prior path does: FP64 1e-11
(single, windows, batched, samples); complex64 1e-5 on m and q; bf16 hi+lo
1e-5 or twice its rounded-operator floor.
"""
import json
import os

import numpy as np
import pytest

import synth
from oracle import posterior as Q
from oracle import prior as P
from oracle import toeplitz as T

from gpu_util import adjoint_rounded, make_context, mixed_bound, pad_window, rel

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
SIGMA_C1 = json.load(open(os.path.join(HERE, "golden", "sigma_c1.json")))["sigma"]

CASES = {
    "c1": synth.CONFIGS[1],
    "wide": synth.small_config(Nd=26, Nx=60, Ny=75, Nt=77, Nq=3, cid=85),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    import torch
    from paper_2504_16344_gb300 import tw
    cfg = CASES[request.param]
    F = synth.block_column(cfg, "F")
    Fq = synth.block_column(cfg, "Fq")
    lam = P.spectrum_for(cfg)
    sigma0 = SIGMA_C1 if request.param == "c1" else None
    _, d, sigma = Q.synthetic_event(F, lam, synth.event_z(cfg), synth.noise_z(cfg), sigma0)
    L = Q.cholesky(Q.form_K(F, lam, sigma ** 2))
    ctx = make_context(cfg, keep=tw.KEEP_FP64 | tw.KEEP_C64 | tw.KEEP_BF16X2 | tw.KEEP_G)
    ctx.factor_K(sigma ** 2)
    ctx.reserve_batch(8)
    yield dict(cfg=cfg, ctx=ctx, F=F, Fq=Fq, lam=lam, L=L, d=d, sigma=sigma,
               dev=torch.device("cuda", 0))
    ctx.close()


def _t(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


@pytest.mark.parametrize("frac", [1.0, 0.3])
def test_single_fp64_with_gstar(case, frac):
    from paper_2504_16344_gb300 import tw
    cfg = case["cfg"]
    w = max(1, int(round(frac * cfg.Nt)))
    m_ref, _ = Q.posterior_mean(case["F"], case["lam"], case["L"], case["d"], cfg.Nt, nt_window=w)
    m = case["ctx"].infer(tw.PREC_FP64, _t(case["d"], case["dev"]), windows=[w])[0].cpu().numpy()
    case["ctx"].check()
    err = rel(m, m_ref)
    print(f"{cfg.cid}: G* path FP64 window {w}: m rel err {err:.2e}")
    assert np.all(m[w:] == 0.0) and err < 1e-11


def _bounds(case, prec, y, nt_window, m_ref, q_ref):
    """(m bound, q bound): 1e-5 for complex64; for bf16 hi+lo 1e-5 or twice
    the floor of its rounded operator (the F* + prior path it keeps)."""
    if prec != "BF16X2":
        return 1e-5, 1e-5
    cfg = case["cfg"]
    m_fl = P.prior_apply(adjoint_rounded(case["F"], pad_window(y, cfg.Nt, cfg.Nd), "BF16X2"), case["lam"])
    m_fl[nt_window:] = 0.0
    return mixed_bound(rel(m_fl, m_ref)), mixed_bound(rel(T.p2o_apply(case["Fq"], m_fl), q_ref))


@pytest.mark.parametrize("prec", ["C64", "BF16X2"])
def test_single_mixed_with_gstar(case, prec):
    from paper_2504_16344_gb300 import tw
    cfg, ctx = case["cfg"], case["ctx"]
    p = getattr(tw, "PREC_" + prec)
    m_ref, y = Q.posterior_mean(case["F"], case["lam"], case["L"], case["d"], cfg.Nt)
    q_ref = T.p2o_apply(case["Fq"], m_ref)
    m = ctx.infer(p, _t(case["d"], case["dev"]))
    q = ctx.forecast(p, m)[0].cpu().numpy()
    ctx.check()
    em, eq = rel(m[0].cpu().numpy(), m_ref), rel(q, q_ref)
    bm, bq = _bounds(case, prec, y, cfg.Nt, m_ref, q_ref)
    print(f"{cfg.cid}: G* path {prec}: m rel err {em:.2e} q {eq:.2e} (bounds {bm:.1e} {bq:.1e})")
    assert em < bm and eq < bq


@pytest.mark.parametrize("prec", ["FP64", "C64", "BF16X2"])
def test_batched_with_gstar(case, prec):
    import torch
    from paper_2504_16344_gb300 import tw
    cfg, ctx = case["cfg"], case["ctx"]
    ws = [cfg.Nt, max(1, cfg.Nt // 3), 1, cfg.Nt - 1]
    ds = np.stack([case["d"], 0.5 * case["d"], -case["d"], case["d"]])
    win = torch.tensor(ws, dtype=torch.int32, device=case["dev"])
    m, q = ctx.infer_batch(getattr(tw, "PREC_" + prec), _t(ds, case["dev"]), win)
    ctx.check()
    m, q = m.cpu().numpy(), q.cpu().numpy()
    for r, w in enumerate(ws):
        m_ref, y = Q.posterior_mean(case["F"], case["lam"], case["L"], ds[r], cfg.Nt, nt_window=w)
        q_ref = T.p2o_apply(case["Fq"], m_ref)
        em, eq = rel(m[r], m_ref), rel(q[r], q_ref)
        bm, bq = (1e-11, 1e-11) if prec == "FP64" else _bounds(case, prec, y, w, m_ref, q_ref)
        print(f"{cfg.cid}: G* batched {prec} window {w}: m {em:.2e} q {eq:.2e} (bounds {bm:.1e} {bq:.1e})")
        assert em < bm and eq < bq


def test_batched_samples_with_gstar(case):
    from paper_2504_16344_gb300 import tw
    cfg, ctx = case["cfg"], case["ctx"]
    ns = 3
    ws = [cfg.Nt, cfg.Nt // 2, 2]
    zm = np.stack([synth.sample_z(cfg, k, cfg.Nt)[0] for k in range(ns)])
    zn = np.stack([synth.sample_z(cfg, k, cfg.Nt)[1] for k in range(ns)])
    d = np.stack([case["d"]] * ns)
    got = ctx.sample_posterior(_t(d, case["dev"]), _t(zm, case["dev"]), _t(zn, case["dev"]),
                               case["sigma"], windows=ws).cpu().numpy()
    ctx.check()
    for k in range(ns):
        ref = Q.posterior_sample(case["F"], case["lam"], case["L"], case["sigma"], d[k], zm[k],
                                 zn[k], ws[k])
        m_pr = P.prior_apply(zm[k], case["lam"], 0.5)
        assert rel(got[k], ref) < 1e-11 and rel(got[k] - m_pr, ref - m_pr) < 1e-10


@pytest.mark.parametrize("prec", ["FP64", "C64", "BF16X2"])
@pytest.mark.parametrize("frac", [1.0, 0.3])
def test_infer_forecast_in_one_call(case, prec, frac):
    """tw_infer_forecast: with G^ kept, m's inverse time FFT also takes the
    forecast's forward FFT of m in the same kernel.  m must be the bits
    tw_infer gives; q must match the oracle as tw_forecast's does (FP64 at
    1e-11 and within 1e-13 of tw_forecast, whose m^ comes from m rounded to
    FP64) and be the very bits of tw_forecast on the reduced paths."""
    from paper_2504_16344_gb300 import tw
    cfg, ctx, dev = case["cfg"], case["ctx"], case["dev"]
    p = getattr(tw, "PREC_" + prec)
    w = max(1, int(round(frac * cfg.Nt)))
    d = _t(case["d"], dev)
    m1 = ctx.infer(p, d, windows=[w])
    q1 = ctx.forecast(p, m1)
    m2, q2 = ctx.infer_forecast(p, d, windows=[w])
    ctx.check()
    m1, q1, m2, q2 = (a[0].cpu().numpy() for a in (m1, q1, m2, q2))
    assert np.array_equal(m1, m2)
    m_ref, _ = Q.posterior_mean(case["F"], case["lam"], case["L"], case["d"], cfg.Nt, nt_window=w)
    q_ref = T.p2o_apply(case["Fq"], m_ref)
    e_sep, e_ref = rel(q2, q1), rel(q2, q_ref)
    print(f"{cfg.cid}: {prec} window {w}: fused q vs separate {e_sep:.2e}, vs oracle {e_ref:.2e}")
    if prec == "FP64":
        assert e_sep < 1e-13 and e_ref < 1e-11
    else:
        assert np.array_equal(q1, q2)
