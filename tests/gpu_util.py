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


# ---- floors of the reduced-precision storages --------------------------------
# A reduced-precision operator is stored rounded (complex64, or each real
# part as bf16 hi + bf16 lo); no arithmetic after that can recover the
# rounding.  These helpers give the result of EXACT (FP64) arithmetic on the
# rounded operator, through the circulant embedding of Sec. "FFT-based
# Hessian matvecs" (zero-pad time to 2Nt, one product per frequency, inverse
# transform, first Nt steps); with the unrounded operator they equal the
# oracle's direct sums (checked by the callers' FP64 tests).

def bf16_rn(x32: np.ndarray) -> np.ndarray:
    """float32 -> bf16 (round to nearest even), returned as float32."""
    u = x32.astype(np.float32).view(np.uint32)
    u = (u + (((u >> 16) & 1) + 0x7FFF)) & np.uint32(0xFFFF0000)
    return u.view(np.float32)


def round_operator(Fh: np.ndarray, fmt: str) -> np.ndarray:
    """Frequency-domain operator rounded as stored: "C64" complex64, or
    "BF16X2" each real part as float32 split into bf16 hi + bf16 lo."""
    if fmt == "C64":
        return Fh.astype(np.complex64).astype(np.complex128)
    out = []
    for part in (Fh.real, Fh.imag):
        v = part.astype(np.float32)
        hi = bf16_rn(v)
        lo = bf16_rn((v - hi).astype(np.float32))
        out.append(hi.astype(np.float64) + lo.astype(np.float64))
    return out[0] + 1j * out[1]


def forward_rounded(F: np.ndarray, x: np.ndarray, fmt: str) -> np.ndarray:
    """F x ([Nt][Nm] -> [Nt][rows]) with F^ rounded to `fmt`, exact arithmetic."""
    Nt = F.shape[0]
    Fh = round_operator(np.fft.rfft(F, n=2 * Nt, axis=0), fmt)
    xh = np.fft.rfft(x, n=2 * Nt, axis=0)
    return np.fft.irfft(np.einsum("wsk,wk->ws", Fh, xh), n=2 * Nt, axis=0)[:Nt]


def adjoint_rounded(F: np.ndarray, y: np.ndarray, fmt: str) -> np.ndarray:
    """F^T y ([Nt][rows] -> [Nt][Nm]) with F^ rounded to `fmt`, exact arithmetic."""
    Nt = F.shape[0]
    Fh = round_operator(np.fft.rfft(F, n=2 * Nt, axis=0), fmt)
    yh = np.fft.rfft(y, n=2 * Nt, axis=0)
    return np.fft.irfft(np.einsum("wsk,ws->wk", Fh.conj(), yh), n=2 * Nt, axis=0)[:Nt]


def pad_window(y: np.ndarray, Nt: int, rows: int) -> np.ndarray:
    """A window's solution (its leading rows * Nt' entries) as [Nt][rows], zero beyond."""
    out = np.zeros(Nt * rows)
    out[:y.size] = np.ravel(y)
    return out.reshape(Nt, rows)


def mixed_bound(floor: float) -> float:
    """Bound of a reduced-precision result: the 1e-5 target, or twice the
    error that rounding the stored operator alone causes where that floor is
    higher (the bf16 hi+lo storage on ill-conditioned cases)."""
    return max(1e-5, 2.0 * floor)
