"""Write tests/golden/sigma_c<N>.json: the noise level of each synthetic workload.

Also writes tests/golden/event_c<N>.npy: the event-0 data
d = F m_true + sigma z_n ([Nt][Nd] FP64) of each large workload, so GPU
tests and the benchmark use oracle-made data without a full CPU apply.

Calls only `oracle/` (and the seeded input generator `synth`).  The paper adds
1% relative noise to its synthetic observations (Sec. "Application to the
Cascadia subduction zone"), read here as one global level,
sigma = 0.01 * rms(F m_true) over all Nd*Nt entries of event 0 with
m_true = Gamma_pr^{1/2} z.  Both the GPU tests and the benchmark take sigma
from these files, so K = sigma^2 I + F Gamma_pr F^T is the same on both sides.

usage: python tests/golden/make_golden.py 1 2 5
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


def sigma_for(cid: int) -> dict:
    cfg = synth.CONFIGS[cid]
    t0 = time.time()
    lam = P.spectrum_for(cfg)
    m_true = P.prior_apply(synth.event_z(cfg, 0), lam, 0.5)

    def block(lag):
        return synth.block_column(cfg, "F", lags=[lag])[0]

    d_clean = T.p2o_apply(block, m_true, Nt=cfg.Nt)
    rms = float(np.sqrt(np.mean(d_clean * d_clean)))
    sigma = Q.noise_sigma(d_clean, cfg.noise_rel)
    if cid != 1:
        np.save(os.path.join(HERE, f"event_c{cid}.npy"), d_clean + sigma * synth.noise_z(cfg, 0))
    return {
        "config": cid,
        "sigma": sigma,
        "rms_clean": rms,
        "norm_m_true": float(np.linalg.norm(m_true)),
        "recipe": "sigma = 0.01 * rms(F m_true), event 0, m_true = Gamma_pr^{1/2} z; "
                  "1% relative noise of Sec. 'Application to the Cascadia subduction zone'",
        "seconds": round(time.time() - t0, 1),
    }


if __name__ == "__main__":
    for arg in sys.argv[1:] or ["1"]:
        out = sigma_for(int(arg))
        with open(os.path.join(HERE, f"sigma_c{arg}.json"), "w") as f:
            json.dump(out, f, indent=1)
        print(out)
