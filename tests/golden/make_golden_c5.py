"""Write tests/golden/posterior_c5.npz: oracle posterior means and forecasts of the
200-sensor serving workload (Nd=200, 316x316 grid, Nt=420, Nq=50) for
observation windows the CPU can afford.

Calls only `oracle/` (and the seeded input generator `synth`).  For each case
(event e, window Nt'), with sigma from tests/golden/sigma_c5.json (written by
make_golden.py 5: 1% of rms(F m_true) of event 0 over the full window):

  m_true = Gamma_pr^{1/2} z_e,  d' = F' m_true + sigma z_n,e   (leading Nt' blocks)
  K' = sigma^2 I + F' Gamma_pr F'^T,  m = Gamma_pr F'^T K'^{-1} d'  (Phase 4)
  q = F_q m over all Nt steps

(Sec. "Real-time Bayesian inference and prediction framework").  Stored per
case: d' ([Nt'][Nd]), q ([Nt][Nq]), ||m||, and m at 20,000 entries drawn
with a seeded generator (the full m is 40 MB per case); the benchmark
compares its results with these, relative L2 over q and over the sampled m.

usage: python tests/golden/make_golden_c5.py     (about 15 minutes, ~40 GB of host memory)
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import synth  # noqa: E402
from oracle import posterior as Q  # noqa: E402
from oracle import prior as P  # noqa: E402
from oracle import toeplitz as T  # noqa: E402

CASES = ((0, 20), (1, 60))        # (event, observation window Nt')
NSAMPLE = 20_000
SAMPLE_SEED = 5_020


def sample_index(cfg, window):
    """Flat indices into m [Nt][Nm] of the stored entries (inside the window)."""
    return synth.sample_entries(window * cfg.Nm, NSAMPLE, SAMPLE_SEED + window)


def main():
    cfg = synth.CONFIGS[5]
    sigma = json.load(open(os.path.join(HERE, "sigma_c5.json")))["sigma"]
    lam = P.spectrum_for(cfg)
    out = {"sigma": np.float64(sigma), "cases": np.array(CASES, dtype=np.int64)}
    for e, w in CASES:
        t0 = time.time()
        Fw = synth.block_column(cfg, "F", lags=range(w))                 # [w][Nd][Nm]
        m_true = P.prior_apply(synth.event_z(cfg, e)[:w], lam, 0.5)
        d = T.p2o_apply(Fw, m_true) + sigma * synth.noise_z(cfg, e)[:w]
        L = Q.cholesky(Q.form_K(Fw, lam, sigma ** 2))
        m, _ = Q.posterior_mean(Fw, lam, L, d, cfg.Nt, nt_window=w)
        del Fw, L

        def fq(lag):
            return synth.block_column(cfg, "Fq", lags=[lag])[0]

        q = T.p2o_apply(fq, m, Nt=cfg.Nt)
        idx = sample_index(cfg, w)
        out[f"d_e{e}_w{w}"] = d
        out[f"q_e{e}_w{w}"] = q
        out[f"msample_e{e}_w{w}"] = m.reshape(-1)[idx]
        out[f"mnorm_e{e}_w{w}"] = np.float64(np.linalg.norm(m))
        print(f"event {e} window {w}: |m| {np.linalg.norm(m):.4e} |q| {np.linalg.norm(q):.4e} "
              f"({time.time() - t0:.0f} s)", flush=True)
    np.savez_compressed(os.path.join(HERE, "posterior_c5.npz"), **out)


if __name__ == "__main__":
    main()
