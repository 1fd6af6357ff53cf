"""GPU serving loop: replay a request trace with continuous batching over lanes.

Requests arrive in bursts much faster than a batch completes, and the loop
keeps several batches in flight on separate lanes (streams and workspaces),
so requests that arrive while batches run start before those batches end
and their kernels overlap on the device.  Every request's posterior mean and
forecast must match the oracle for its event and window (FP64 path 1e-11,
complex64 path 1e-5), must be bitwise what the request gets when served
alone, and the loop must have run batches side by side.
"""
import numpy as np
import pytest

import synth
from oracle import posterior as Q
from oracle import prior as P
from oracle import toeplitz as T

from gpu_util import make_context, rel

pytestmark = pytest.mark.gpu

CFG = synth.small_config(Nd=20, Nx=40, Ny=50, Nt=40, Nq=5, cid=84)
NEV, NREQ, BMAX, LANES = 5, 64, 8, 3
TOL = {"FP64": 1e-11, "C64": 1e-5}


@pytest.fixture(scope="module")
def setup():
    import torch
    from paper_2504_16344_gb300 import tw
    cfg = CFG
    F = synth.block_column(cfg, "F")
    Fq = synth.block_column(cfg, "Fq")
    lam = P.spectrum_for(cfg)
    _, d0, sigma = Q.synthetic_event(F, lam, synth.event_z(cfg, 0), synth.noise_z(cfg, 0))
    ds = np.stack([d0] + [Q.synthetic_event(F, lam, synth.event_z(cfg, e), synth.noise_z(cfg, e),
                                            sigma)[1] for e in range(1, NEV)])
    L = Q.cholesky(Q.form_K(F, lam, sigma ** 2))
    ctx = make_context(cfg, keep=tw.KEEP_FP64 | tw.KEEP_C64)
    ctx.factor_K(sigma ** 2)
    ctx.reserve_batch(BMAX)
    g = np.random.default_rng(4242)
    # bursts: requests arrive much faster than a batch completes
    arr = np.cumsum(g.exponential(1.0 / 5000.0, size=NREQ))
    ev = g.integers(0, NEV, size=NREQ)
    win = g.integers(1, cfg.Nt + 1, size=NREQ)
    dev = torch.device("cuda", 0)
    bank = torch.from_numpy(ds).to(dev)
    refs = []
    for i in range(NREQ):
        m_ref, _ = Q.posterior_mean(F, lam, L, ds[int(ev[i])], cfg.Nt, nt_window=int(win[i]))
        refs.append((m_ref, T.p2o_apply(Fq, m_ref)))
    yield dict(ctx=ctx, cfg=cfg, arr=arr, ev=ev, win=win, bank=bank, dev=dev, refs=refs)
    ctx.close()


@pytest.fixture(scope="module", params=["FP64", "C64"])
def served(setup, request):
    import torch
    from paper_2504_16344_gb300 import tw
    ctx, arr, ev, win, bank = setup["ctx"], setup["arr"], setup["ev"], setup["win"], setup["bank"]
    prec = getattr(tw, "PREC_" + request.param)
    stream = torch.cuda.Stream(device=setup["dev"])
    # warm-up replay (kernel attributes, first-launch costs), then the measured one
    ctx.serve_replay(prec, arr[:4], ev[:4], win[:4], bank, BMAX, stream, lanes=LANES)
    lat, q, m, st = ctx.serve_replay(prec, arr, ev, win, bank, BMAX, stream, m_out=True, lanes=LANES)
    return dict(setup, name=request.param, prec=prec, lat=lat, q=q, m=m, st=st)


def test_every_request_matches_oracle(served):
    errs_m = [rel(served["m"][i], served["refs"][i][0]) for i in range(NREQ)]
    errs_q = [rel(served["q"][i], served["refs"][i][1]) for i in range(NREQ)]
    print(f"{served['name']}: served {NREQ} requests: max m err {max(errs_m):.2e}, "
          f"q err {max(errs_q):.2e}")
    assert max(errs_m) < TOL[served["name"]] and max(errs_q) < TOL[served["name"]]


def test_alone_equals_in_mix(served):
    """Served alone (one request, the reserved lane) or inside a batch of any
    lane while other batches run: identical bits."""
    import torch
    ctx = served["ctx"]
    for i in (0, 7, NREQ // 2, NREQ - 1):
        e, w = int(served["ev"][i]), int(served["win"][i])
        winv = torch.tensor([w], dtype=torch.int32, device=served["dev"])
        m1, q1 = ctx.infer_batch(served["prec"], served["bank"][e:e + 1].contiguous(), winv)
        assert np.array_equal(m1[0].cpu().numpy(), served["m"][i])
        assert np.array_equal(q1[0].cpu().numpy(), served["q"][i])


def test_batches_overlap(served):
    st, lat = served["st"], served["lat"]
    print(f"{served['name']}: lanes {st.lanes}, at most {st.max_in_flight} batches in flight, "
          f"batches {st.batches} (max {st.max_batch}, mean {st.mean_batch:.2f}), "
          f"p50 {np.percentile(lat, 50):.2f} ms, p99 {np.percentile(lat, 99):.2f} ms, "
          f"busy {st.busy_s * 1e3:.1f} ms over a makespan of {st.makespan_s * 1e3:.1f} ms")
    assert st.lanes == LANES
    assert st.max_in_flight >= 2                  # batches ran side by side
    assert st.batches >= 3 and 1 < st.max_batch <= BMAX
    assert st.mean_batch == pytest.approx(NREQ / st.batches)
    assert np.all(lat > 0)
    # overlapping batches: their summed durations may exceed the makespan, but
    # never the lanes' combined time
    assert st.busy_s <= st.lanes * st.makespan_s + 1e-3
