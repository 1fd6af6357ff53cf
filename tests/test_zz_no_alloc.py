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
    c = make_context(CFG, keep=tw.KEEP_FP64 | tw.KEEP_C64 | tw.KEEP_BF16X2)
    yield c
    c.close()


# the same kernels run on both entry points, so the tolerance is the one the
# precision's own tests use against the oracle
@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 1e-5), (2, 1e-5)])
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


def test_noalloc_zero_rhs_launches_nothing(ctx):
    import ctypes
    from paper_2504_16344_gb300 import tw
    before = tw.kernel_launches()
    assert ctx.lib.tw_p2o_apply_noalloc(ctx.h, 0, 0, 0, None, None, None) == tw.OK
    assert tw.kernel_launches() == before


def test_noalloc_rejects_sizes_beyond_the_fixed_scratch():
    """(Nt+1) * ceil(Nm/1024) * rows * 16 bytes above 32 MiB: 2,048 sensors,
    1,100 steps, one grid point (36 MB of partial sums, a 36 MB operator).
    The call returns TW_ERR_ARG with a message before any launch."""
    import torch
    from paper_2504_16344_gb300 import tw
    big = synth.small_config(Nd=2048, Nx=1, Ny=1, Nt=1100, Nq=1, cid=82)
    c = make_context(big, keep=tw.KEEP_FP64, prior=False)
    try:
        dev = torch.device("cuda", c.device)
        x = torch.zeros((1, big.Nt, big.Nm), dtype=torch.float64, device=dev)
        out = torch.zeros((1, big.Nt, big.Nd), dtype=torch.float64, device=dev)
        before = tw.kernel_launches()
        with pytest.raises(tw.TwError) as ei:
            c.p2o_apply_noalloc(0, 0, x, out)
        assert ei.value.status == tw.ERR_ARG and "scratch" in str(ei.value)
        assert tw.kernel_launches() == before
        # the regular entry point serves the same call
        c.p2o_apply(0, 0, x)
        c.check()
    finally:
        c.close()
