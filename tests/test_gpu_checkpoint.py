"""Phase-2 checkpoint (tw_save_factor / tw_load_factor) and TW_KEEP_FACTOR64.

The offline-online split (Sec. "Real-time Bayesian inference and prediction
framework": Phases 1-3 once, Phase 4 per event) lets a context load K's
factor instead of forming it.  A loaded factor must give bit-for-bit the
results of the context that formed it, single and batched; a complex64
context that forms only the FP64 factor (TW_KEEP_FACTOR64) must solve exactly
as a context that also keeps the FP64 operator; and every mismatch between
checkpoint and context is refused.
"""
import json
import os

import numpy as np
import pytest

import synth
from oracle import posterior as Q
from oracle import prior as P

from gpu_util import make_context, rel

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
SIGMA_C1 = json.load(open(os.path.join(HERE, "golden", "sigma_c1.json")))["sigma"]

CASES = {
    "c1": synth.CONFIGS[1],
    "wide": synth.small_config(Nd=26, Nx=60, Ny=75, Nt=77, Nq=3, cid=85),
}


def _t(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    import torch
    from paper_2504_16344_gb300 import tw
    cfg = CASES[request.param]
    F = synth.block_column(cfg, "F")
    lam = P.spectrum_for(cfg)
    sigma0 = SIGMA_C1 if request.param == "c1" else None
    _, d, sigma = Q.synthetic_event(F, lam, synth.event_z(cfg), synth.noise_z(cfg), sigma0)
    L = Q.cholesky(Q.form_K(F, lam, sigma ** 2))
    # the context that forms K (FP64 and complex64 operators, both factors)
    ref = make_context(cfg, keep=tw.KEEP_FP64 | tw.KEEP_C64)
    ref.factor_K(sigma ** 2)
    buf = ref.save_factor()
    yield dict(cfg=cfg, ref=ref, buf=buf, F=F, lam=lam, L=L, d=d, sigma=sigma,
               dev=torch.device("cuda", 0))
    ref.close()


def _loaded(case, keep):
    """A context that loads the checkpoint: columns first, then the prior (no G is kept)."""
    cfg = case["cfg"]
    ctx = make_context(cfg, keep=keep, prior=False)
    ctx.set_prior(cfg.nu, cfg.ell, cfg.var)
    ctx.load_factor(case["buf"])
    return ctx


def test_checkpoint_size_and_header(case):
    cfg = case["cfg"]
    NB = -(-cfg.Nd * cfg.Nt // 64)
    nblk = NB * (NB + 1) // 2
    buf = case["buf"]
    assert buf.size == case["ref"].factor_bytes() == 96 + 8 * 64 * 64 * (nblk + NB)
    assert bytes(buf[:8]) == b"TWLFAC02"
    hdr = np.frombuffer(buf[8:32].tobytes(), dtype=np.int32)
    assert list(hdr) == [cfg.Nd, cfg.Nt, cfg.Nx, cfg.Ny, NB, 64]
    assert np.frombuffer(buf[40:48].tobytes(), dtype=np.float64)[0] == case["sigma"] ** 2


def test_loaded_factor_bitwise_single_and_windows(case):
    from paper_2504_16344_gb300 import tw
    cfg, dev = case["cfg"], case["dev"]
    ctx = _loaded(case, tw.KEEP_FP64 | tw.KEEP_C64)
    try:
        d = _t(case["d"], dev)
        for w in (cfg.Nt, max(1, cfg.Nt // 3)):
            for prec in (tw.PREC_FP64, tw.PREC_C64):
                a = case["ref"].infer(prec, d, windows=[w])[0].cpu().numpy()
                b = ctx.infer(prec, d, windows=[w])[0].cpu().numpy()
                assert np.array_equal(a, b), (w, prec)
        m_ref, _ = Q.posterior_mean(case["F"], case["lam"], case["L"], case["d"], cfg.Nt)
        assert rel(ctx.infer(tw.PREC_FP64, d)[0].cpu().numpy(), m_ref) < 1e-11
        ctx.check()
    finally:
        ctx.close()


def test_loaded_factor_bitwise_batched(case):
    import torch
    from paper_2504_16344_gb300 import tw
    cfg, dev = case["cfg"], case["dev"]
    ctx = _loaded(case, tw.KEEP_FP64 | tw.KEEP_C64)
    try:
        B = 5
        d = _t(np.stack([case["d"] * (1.0 + 0.1 * k) for k in range(B)]), dev)
        win = torch.tensor([max(1, cfg.Nt - 7 * k) for k in range(B)], dtype=torch.int32, device=dev)
        outs = []
        for c in (case["ref"], ctx):
            c.reserve_batch(B)
            m = torch.empty((B, cfg.Nt, cfg.Nm), dtype=torch.float64, device=dev)
            q = torch.empty((B, cfg.Nt, cfg.Nq), dtype=torch.float64, device=dev)
            for prec in (tw.PREC_FP64, tw.PREC_C64):
                c.infer_batch(prec, d, win, m, q)
                outs.append((m.cpu().numpy(), q.cpu().numpy()))
            c.check()
            c.reserve_batch(0)
        for (ma, qa), (mb, qb) in zip(outs[:2], outs[2:]):
            assert np.array_equal(ma, mb) and np.array_equal(qa, qb)
    finally:
        ctx.close()


def test_checkpoint_file_roundtrip(case, tmp_path):
    from paper_2504_16344_gb300 import tw
    cfg, dev = case["cfg"], case["dev"]
    path = str(tmp_path / "factor.bin")
    case["ref"].save_factor(path)
    ctx = make_context(cfg, keep=tw.KEEP_FP64, prior=False)
    try:
        ctx.set_prior(cfg.nu, cfg.ell, cfg.var)
        ctx.load_factor(path)
        d = _t(case["d"], dev)
        a = case["ref"].infer(tw.PREC_FP64, d)[0].cpu().numpy()
        assert np.array_equal(a, ctx.infer(tw.PREC_FP64, d)[0].cpu().numpy())
    finally:
        ctx.close()


def test_no_K_after_load(case):
    from paper_2504_16344_gb300 import tw
    cfg, dev = case["cfg"], case["dev"]
    ctx = _loaded(case, tw.KEEP_FP64)
    try:
        x = _t(case["d"], dev)
        with pytest.raises(tw.TwError) as ei:
            ctx.apply_K(x)
        assert ei.value.status == 4
        _, st = ctx.infer(tw.PREC_FP64, x, stats=True)
        assert st.resid_rel == -1.0
    finally:
        ctx.close()


def test_checkpoint_mismatch_refused(case):
    from paper_2504_16344_gb300 import tw
    cfg = case["cfg"]
    buf = case["buf"]

    def status_of(fn):
        with pytest.raises(tw.TwError) as ei:
            fn()
        return ei.value.status

    # other sizes
    other = synth.small_config(Nd=cfg.Nd, Nx=cfg.Nx, Ny=cfg.Ny, Nt=cfg.Nt - 1, Nq=cfg.Nq, cid=86)
    c2 = make_context(other, keep=tw.KEEP_FP64, prior=False)
    try:
        c2.set_prior(other.nu, other.ell, other.var)
        assert status_of(lambda: c2.load_factor(buf)) == 1
    finally:
        c2.close()
    ctx = make_context(cfg, keep=tw.KEEP_FP64, prior=False)
    try:
        # no factor yet, no prior yet
        assert status_of(lambda: ctx.save_factor()) == 4
        assert status_of(lambda: ctx.load_factor(buf)) == 4
        # another prior
        ctx.set_prior(cfg.nu, 2.0 * cfg.ell, cfg.var)
        assert status_of(lambda: ctx.load_factor(buf)) == 1
        ctx.set_prior(cfg.nu, cfg.ell, cfg.var)
        bad = buf.copy()
        bad[0] ^= 0xFF
        assert status_of(lambda: ctx.load_factor(bad)) == 1
        assert status_of(lambda: ctx.load_factor(buf[:-8])) == 1
        assert status_of(lambda: ctx.load_factor(buf[:50])) == 1
        ctx.load_factor(buf)       # the intact checkpoint still loads
        ctx.check()
    finally:
        ctx.close()


def test_factor_of_another_block_column_refused(case):
    """Same sizes, prior and domain, but another synthetic operator (other
    sensor positions): the checkpoint's block-column fingerprint differs and
    the factor is refused instead of giving wrong posterior means."""
    from paper_2504_16344_gb300 import tw
    cfg = case["cfg"]
    other = synth.small_config(Nd=cfg.Nd, Nx=cfg.Nx, Ny=cfg.Ny, Nt=cfg.Nt, Nq=cfg.Nq, cid=cfg.cid + 50)
    ctx = make_context(other, keep=tw.KEEP_FP64, prior=False)
    try:
        ctx.set_prior(cfg.nu, cfg.ell, cfg.var)
        with pytest.raises(tw.TwError) as ei:
            ctx.load_factor(case["buf"])
        assert ei.value.status == 1 and "block column" in str(ei.value)
    finally:
        ctx.close()


def test_factor64_only_mixed_context(case):
    """keep = C64 | FACTOR64: the FP64 factor without the FP64 operator gives
    the mixed results of the context that keeps both, bit for bit; no FP32
    factor is formed, so the FP32-refinement solver has nothing to select."""
    import torch
    from paper_2504_16344_gb300 import tw
    cfg, dev = case["cfg"], case["dev"]
    ctx = make_context(cfg, keep=tw.KEEP_C64 | tw.KEEP_FACTOR64)
    try:
        ctx.factor_K(case["sigma"] ** 2)
        assert ctx.device_bytes() < case["ref"].device_bytes()
        d = _t(case["d"], dev)
        a = case["ref"].infer(tw.PREC_C64, d)[0].cpu().numpy()
        b = ctx.infer(tw.PREC_C64, d)[0].cpu().numpy()
        assert np.array_equal(a, b)
        ctx.set_solver(tw.SOLVE_FP32_IR)
        assert np.array_equal(a, ctx.infer(tw.PREC_C64, d)[0].cpu().numpy())
        ctx.set_solver(tw.SOLVE_FACTOR64)
        # its checkpoint is the FP64 context's checkpoint
        assert np.array_equal(ctx.save_factor(), case["buf"])
        with pytest.raises(tw.TwError):
            ctx.infer(tw.PREC_FP64, d)
        m_ref, _ = Q.posterior_mean(case["F"], case["lam"], case["L"], case["d"], cfg.Nt)
        assert rel(b, m_ref) < 1e-5
        ctx.reserve_batch(2)
        m = torch.empty((2, cfg.Nt, cfg.Nm), dtype=torch.float64, device=dev)
        q = torch.empty((2, cfg.Nt, cfg.Nq), dtype=torch.float64, device=dev)
        win = torch.tensor([cfg.Nt, cfg.Nt], dtype=torch.int32, device=dev)
        ctx.infer_batch(tw.PREC_C64, torch.stack([d, d]), win, m, q)
        ctx.check()
        assert rel(m[1].cpu().numpy(), m_ref) < 1e-5
    finally:
        ctx.close()


def test_factor64_without_fp64_operator_needs_prior_first(case):
    from paper_2504_16344_gb300 import tw
    cfg = case["cfg"]
    ctx = make_context(cfg, keep=tw.KEEP_C64 | tw.KEEP_FACTOR64, prior=False)
    try:
        ctx.set_prior(cfg.nu, cfg.ell, cfg.var)
        with pytest.raises(tw.TwError) as ei:
            ctx.factor_K(case["sigma"] ** 2)
        assert ei.value.status == 4
    finally:
        ctx.close()
