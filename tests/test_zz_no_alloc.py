"""The allocation-free forward apply gives the same result as tw_p2o_apply.

tw_p2o_apply_noalloc is for callers that must not allocate device memory at
call time: it keeps the GEMV's partial sums in a fixed array inside the
library instead of the context.  Two calls in a row are checked against the
regular entry point (the fixed array keeps the previous call's contents, so
the second call shows nothing stale leaks through).  This file is collected
last so that a failure here cannot hide failures elsewhere.
"""
import numpy as np
import pytest

import synth

from gpu_util import make_context, rel

pytestmark = pytest.mark.gpu

CFG = synth.small_config(Nd=13, Nx=45, Ny=50, Nt=21, Nq=3, cid=81)


@pytest.fixture(scope="module")
def ctx():
    from paper_2504_16344_gb300 import tw
    c = make_context(CFG, keep=tw.KEEP_FP64 | tw.KEEP_C64)
    yield c
    c.close()


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 1e-5)])
@pytest.mark.parametrize("which", [0, 1])
def test_noalloc_apply_matches_regular_apply_twice(ctx, prec, tol, which):
    import torch
    dev = torch.device("cuda", ctx.device)
    rows = ctx.rows(which)
    for call in range(2):
        x = torch.from_numpy(synth.white((2, CFG.Nt, CFG.Nm), 4100 + call)).to(dev)
        ref = ctx.p2o_apply(which, prec, x)
        out = torch.full((2, CFG.Nt, rows), float("nan"), dtype=torch.float64, device=dev)
        ctx.p2o_apply_noalloc(which, prec, x, out)
        ctx.check()
        got, want = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(got))
        for r in range(2):
            assert rel(got[r], want[r]) < tol
