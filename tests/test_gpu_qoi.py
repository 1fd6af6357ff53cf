"""GPU parity of the Phase 3 QoI precomputations and the Phase 4 map q = Q d.

The oracle forms Q and the QoI posterior covariance column by column from
QoI unit vectors with its own applies and LAPACK solves (pinned against the
dense parameter-space definitions).  Bars: Q and q = Q d 1e-11 relative L2;
the covariance C - W^T K^-1 W cancels (the posterior variance is far below
the prior's), so it is compared relative to C's norm at 1e-11 and each
variance relative to its prior variance C_jj at 1e-11.
"""
import json
import os

import numpy as np
import pytest

import synth
from oracle import posterior as Q
from oracle import prior as P
from oracle import qoi as QO

from gpu_util import make_context, rel

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
SIGMA_C1 = json.load(open(os.path.join(HERE, "golden", "sigma_c1.json")))["sigma"]

CASES = {
    "c1": synth.CONFIGS[1],
    "mid": synth.small_config(Nd=20, Nx=40, Ny=50, Nt=40, Nq=5, cid=84),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    import torch
    cfg = CASES[request.param]
    F = synth.block_column(cfg, "F")
    Fq = synth.block_column(cfg, "Fq")
    lam = P.spectrum_for(cfg)
    sigma0 = SIGMA_C1 if request.param == "c1" else None
    _, d, sigma = Q.synthetic_event(F, lam, synth.event_z(cfg), synth.noise_z(cfg), sigma0)
    L = Q.cholesky(Q.form_K(F, lam, sigma ** 2))
    W, Y, C = QO.qoi_columns(F, Fq, lam, L)
    ctx = make_context(cfg)
    ctx.factor_K(sigma ** 2)
    ctx.reserve_batch(16)
    ctx.qoi_build()
    yield dict(cfg=cfg, ctx=ctx, F=F, Fq=Fq, lam=lam, L=L, d=d, sigma=sigma, W=W, Y=Y, C=C,
               dev=torch.device("cuda", 0))
    ctx.close()


def _t(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def test_q_map_apply_matches_oracle(case):
    """Model data (events): 1e-11.  A white vector, which is not data of the model,
    makes Q d cancel; it is held entrywise to kappa(K) u of |Q| |d| instead."""
    cfg, ctx = case["cfg"], case["ctx"]
    F, lam = case["F"], case["lam"]
    sigma = case["sigma"]
    events = [case["d"]] + [Q.synthetic_event(F, lam, synth.event_z(cfg, e), synth.noise_z(cfg, e),
                                              sigma)[1] for e in (1, 2)]
    white = synth.white((cfg.Nt, cfg.Nd), 515)
    ds = np.stack(events + [white])
    q = ctx.qoi_apply(_t(ds, case["dev"])).cpu().numpy()
    ctx.check()
    for r in range(len(events)):
        ref = case["Y"] @ ds[r].ravel()                     # oracle Q d
        m, _ = Q.posterior_mean(F, lam, case["L"], ds[r], cfg.Nt)
        ref2 = Q.forecast(case["Fq"], m).ravel()            # F_q m_map (Phase 4)
        e1, e2 = rel(q[r], ref), rel(q[r], ref2)
        print(f"{cfg.cid}: event {r}: q = Q d rel err vs oracle Q d {e1:.2e}, vs F_q m_map {e2:.2e}")
        assert e1 < 1e-11 and e2 < 1e-11
    # two backward-stable FP64 solvers of K may differ by ~kappa(K) u entrywise
    kappa = Q.condition_number_K(Q.form_K(F, lam, sigma ** 2))
    scale = np.abs(case["Y"]) @ np.abs(white.ravel())
    ew = np.max(np.abs(q[-1].ravel() - case["Y"] @ white.ravel()) / scale)
    bound = max(1e-12, kappa * 2.0 ** -53)
    print(f"{cfg.cid}: white vector: error / (|Q||d|) {ew:.2e}, kappa(K) u = {kappa * 2.0 ** -53:.1e}")
    assert ew < bound



def test_qoi_variance_matches_oracle(case):
    cfg, ctx = case["cfg"], case["ctx"]
    var = ctx.qoi_variance().cpu().numpy().ravel()
    ref = np.diag(case["C"] - case["W"] @ case["Y"].T)
    e = np.max(np.abs(var - ref) / ref)
    # the variance is C_jj - w_j . y_j, two terms of the prior variance's size
    # that cancel: its error is bounded at the FP64 tolerance of that scale
    ec = np.max(np.abs(var - ref) / np.diag(case["C"]))
    print(f"{cfg.cid}: QoI variance max rel err {e:.2e} (of the prior variance {ec:.2e}); "
          f"posterior/prior variance {np.median(ref / np.diag(case['C'])):.2e} (median)")
    assert np.all(var > 0) and ec < 1e-11


def test_qoi_covariance_matches_oracle(case):
    cfg, ctx = case["cfg"], case["ctx"]
    G = ctx.qoi_covariance().cpu().numpy()
    ctx.check()
    ref = case["C"] - case["W"] @ case["Y"].T
    e = np.linalg.norm(G - ref) / np.linalg.norm(case["C"])
    print(f"{cfg.cid}: QoI covariance error / |C| {e:.2e}; asymmetry {rel(G, G.T):.2e}")
    assert e < 1e-11
