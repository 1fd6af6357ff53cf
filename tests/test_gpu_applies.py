"""GPU parity of the Toeplitz applies and the Matern prior against the CPU oracle.

FP64-class path: relative L2 error <= 1e-11 per output vector (the target of
the FP64 path).  FP32 paths: 1e-5, or twice the error of exact arithmetic
on the operator rounded as stored where that floor is higher (the bf16
hi+lo storage keeps 16-17 significant bits per entry, 2^-17 relative).
Shapes span several tiles with ragged tails: odd Nt (radix 3 and 7 passes),
Nm not a multiple of the 1024 grid-point chunk, row counts that do not fill
the 8 warps, sensor counts that leave the tensor-core adjoint's last
16-row stage partly empty.
"""
import numpy as np
import pytest

import synth
from oracle import prior as P
from oracle import toeplitz as T

from gpu_util import adjoint_rounded, forward_rounded, make_context, mixed_bound, rel

pytestmark = pytest.mark.gpu

CASES = {
    "c1": synth.CONFIGS[1],
    "ragged": synth.small_config(Nd=13, Nx=45, Ny=50, Nt=21, Nq=3, cid=81),
    "mid": synth.small_config(Nd=37, Nx=40, Ny=60, Nt=50, Nq=6, cid=82),
    "long": synth.small_config(Nd=5, Nx=20, Ny=25, Nt=400, Nq=2, cid=83),
    # the 316 x 316 grid of the serving workload: 316 = 4 * 79, a prime radix-79 pass
    "grid316": synth.small_config(Nd=4, Nx=316, Ny=316, Nt=6, Nq=2, cid=87),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    import torch
    from paper_2504_16344_gb300 import tw
    cfg = CASES[request.param]
    ctx = make_context(cfg, keep=tw.KEEP_FP64 | tw.KEEP_C64 | tw.KEEP_BF16X2)
    F = synth.block_column(cfg, "F")
    Fq = synth.block_column(cfg, "Fq")
    lam = P.spectrum_for(cfg)
    yield dict(cfg=cfg, ctx=ctx, F=F, Fq=Fq, lam=lam, dev=torch.device("cuda", 0))
    ctx.close()


def _t(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


FMT = {1: "C64", 2: "BF16X2"}


def _bound(prec, got_floor):
    return 1e-11 if prec == 0 else mixed_bound(got_floor())


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_forward_apply_matches_oracle(case, prec):
    from paper_2504_16344_gb300 import tw
    cfg, ctx = case["cfg"], case["ctx"]
    m = synth.white((2, cfg.Nt, cfg.Nm), 1001)
    out = ctx.p2o_apply(tw.MAP_F, prec, _t(m, case["dev"])).cpu().numpy()
    outq = ctx.p2o_apply(tw.MAP_FQ, prec, _t(m, case["dev"])).cpu().numpy()
    ctx.check()
    for r in range(2):
        ref, refq = T.p2o_apply(case["F"], m[r]), T.p2o_apply(case["Fq"], m[r])
        e, eq = rel(out[r], ref), rel(outq[r], refq)
        b = _bound(prec, lambda: rel(forward_rounded(case["F"], m[r], FMT[prec]), ref))
        bq = _bound(prec, lambda: rel(forward_rounded(case["Fq"], m[r], FMT[prec]), refq))
        print(f"{cfg.cid}: forward prec {prec}: F {e:.2e} (bound {b:.1e}), F_q {eq:.2e} (bound {bq:.1e})")
        assert e < b and eq < bq


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_adjoint_apply_matches_oracle(case, prec):
    from paper_2504_16344_gb300 import tw
    cfg, ctx = case["cfg"], case["ctx"]
    y = synth.white((cfg.Nt, cfg.Nd), 1002)
    yq = synth.white((cfg.Nt, cfg.Nq), 1003)
    x = ctx.p2o_adjoint(tw.MAP_F, prec, _t(y, case["dev"]))[0].cpu().numpy()
    xq = ctx.p2o_adjoint(tw.MAP_FQ, prec, _t(yq, case["dev"]))[0].cpu().numpy()
    ctx.check()
    ref, refq = T.p2o_adjoint(case["F"], y), T.p2o_adjoint(case["Fq"], yq)
    e, eq = rel(x, ref), rel(xq, refq)
    b = _bound(prec, lambda: rel(adjoint_rounded(case["F"], y, FMT[prec]), ref))
    bq = _bound(prec, lambda: rel(adjoint_rounded(case["Fq"], yq, FMT[prec]), refq))
    print(f"{cfg.cid}: adjoint prec {prec}: F^T {e:.2e} (bound {b:.1e}), F_q^T {eq:.2e} (bound {bq:.1e})")
    assert e < b and eq < bq


def test_adjoint_identity_on_gpu(case):
    from paper_2504_16344_gb300 import tw
    cfg, ctx = case["cfg"], case["ctx"]
    m = synth.white((cfg.Nt, cfg.Nm), 1004)
    y = synth.white((cfg.Nt, cfg.Nd), 1005)
    Fm = ctx.p2o_apply(tw.MAP_F, tw.PREC_FP64, _t(m, case["dev"]))[0].cpu().numpy()
    Fty = ctx.p2o_adjoint(tw.MAP_F, tw.PREC_FP64, _t(y, case["dev"]))[0].cpu().numpy()
    gap = abs(np.vdot(Fm, y) - np.vdot(m, Fty)) / (np.linalg.norm(Fm) * np.linalg.norm(y))
    assert gap < 1e-12


def test_impulse_response_on_gpu(case):
    from paper_2504_16344_gb300 import tw
    cfg, ctx = case["cfg"], case["ctx"]
    m = np.zeros((cfg.Nt, cfg.Nm))
    k = cfg.Nm // 3
    m[0, k] = 1.0
    d = ctx.p2o_apply(tw.MAP_F, tw.PREC_FP64, _t(m, case["dev"]))[0].cpu().numpy()
    ref = case["F"][:, :, k]
    assert np.abs(d - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("power", [1.0, 0.5])
def test_prior_matches_oracle(case, power):
    cfg, ctx = case["cfg"], case["ctx"]
    x = synth.white((cfg.Nt, cfg.Nm), 1006)
    y = ctx.prior_apply(_t(x, case["dev"]), power)[0].cpu().numpy()
    ctx.check()
    assert rel(y, P.prior_apply(x, case["lam"], power)) < 1e-11
