"""Shared helpers of the GPU tests: build the library, fill a context from `synth`."""
import numpy as np

import synth


def rel(a, b) -> float:
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def make_context(cfg, keep=None, on_device_columns=False, chunk_rows=None, prior=True):
    """Context for `cfg` with both block columns loaded and the prior set.

    Small configs copy the numpy block column (the oracle's exact input); large
    ones generate it with torch on the GPU (identical formula).
    """
    import torch
    from paper_2504_16344_gb300 import build, tw

    build.build()
    keep = tw.KEEP_FP64 if keep is None else keep
    ctx = tw.Context(cfg.Nd, cfg.Nq, cfg.Nx, cfg.Ny, cfg.Nt, cfg.Lx, cfg.Ly, keep=keep)
    dev = torch.device("cuda", ctx.device)
    if prior:
        # prior first: the context then forms K's factor G from the exact column
        ctx.set_prior(cfg.nu, cfg.ell, cfg.var)
    for which, name, rows in ((tw.MAP_F, "F", cfg.Nd), (tw.MAP_FQ, "Fq", cfg.Nq)):
        step = chunk_rows or rows
        for r0 in range(0, rows, step):
            nr = min(step, rows - r0)
            if on_device_columns:
                col = synth.block_column_torch(cfg, name, dev, r0, nr)
            else:
                col = torch.from_numpy(synth.block_column(cfg, name, rows=range(r0, r0 + nr))).to(dev)
            ctx.set_block_column(which, r0, col)
            del col
    torch.cuda.synchronize()
    return ctx
