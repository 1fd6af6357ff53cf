"""Thin ctypes binding of libtw.so (argument marshalling only).

Every step of the online path runs in the library's CUDA kernels; this module
only checks tensor shapes, dtypes and devices and passes raw device pointers
and the current CUDA stream.  Importing it does not need a GPU; creating a
Context does, and fails loudly if libtw.so has not been built.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libtw.so")

# tw_status
OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_STATE, ERR_NOT_SPD, ERR_NOT_CONVERGED, ERR_TIMEOUT = range(8)
STATUS_NAMES = ["TW_OK", "TW_ERR_ARG", "TW_ERR_OOM", "TW_ERR_CUDA", "TW_ERR_STATE",
                "TW_ERR_NOT_SPD", "TW_ERR_NOT_CONVERGED", "TW_ERR_TIMEOUT"]
# tw_phase
PHASES = ["trsv_fwd", "trsv_bwd", "residual", "rfft_data", "gemv_adj", "irfft_param", "prior",
          "rfft_param", "gemv_fwd", "irfft_data", "form_K", "cholesky", "cholesky32", "solve_setup",
          "form_gstar"]
# tw_map
MAP_F, MAP_FQ = 0, 1
# tw_prec
PREC_FP64, PREC_C64, PREC_BF16X2 = 0, 1, 2
KEEP_FP64, KEEP_C64, KEEP_BF16X2, KEEP_G, KEEP_FACTOR64 = 1, 2, 4, 8, 16
# tw_solver
SOLVE_FACTOR64, SOLVE_FP32_IR = 0, 1

_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_U = ctypes.c_uint
_S = ctypes.c_int  # tw_status

# name -> (restype, argtypes); the names are those declared in include/tw.h
SIGNATURES = {
    "tw_create": (_S, [ctypes.POINTER(_P), _I, _I, _I, _I, _I, _D, _D, _U, _I]),
    "tw_destroy": (None, [_P]),
    "tw_last_error": (ctypes.c_char_p, [_P]),
    "tw_set_block_column": (_S, [_P, _I, _I, _I, _P, _P]),
    "tw_set_prior": (_S, [_P, _D, _D, _D]),
    "tw_p2o_apply": (_S, [_P, _I, _I, _I, _P, _P, _P]),
    "tw_p2o_adjoint": (_S, [_P, _I, _I, _I, _P, _P, _P]),
    "tw_prior_apply": (_S, [_P, _D, _I, _P, _P, _P]),
    "tw_factor_K": (_S, [_P, _D, _P]),
    "tw_factor_bytes": (ctypes.c_size_t, [_P]),
    "tw_save_factor": (_S, [_P, _P, ctypes.c_size_t, _P]),
    "tw_load_factor": (_S, [_P, _P, ctypes.c_size_t, _P]),
    "tw_infer": (_S, [_P, _I, _I, _P, _P, _P, _P, _P]),
    "tw_forecast": (_S, [_P, _I, _I, _P, _P, _P]),
    "tw_infer_forecast": (_S, [_P, _I, _I, _P, _P, _P, _P, _P, _P]),
    "tw_solve_K": (_S, [_P, _I, _I, _P, _P, _P, _P]),
    "tw_apply_K": (_S, [_P, _I, _P, _P, _P, _P]),
    "tw_sample_posterior": (_S, [_P, _I, _P, _P, _P, _P, _D, _P, _P]),
    "tw_set_refinement": (_S, [_P, _I]),
    "tw_refinement_steps": (_I, [_P]),
    "tw_set_solver": (_S, [_P, _I]),
    "tw_profile_enable": (_S, [_P, _I]),
    "tw_profile_read": (_S, [_P, _P, _P, _I]),
    "tw_kernel_launches": (ctypes.c_longlong, []),
    "tw_p2o_apply_noalloc": (_S, [_P, _I, _I, _I, _P, _P, _P]),
    "tw_check": (_S, [_P, _P]),
    "tw_device_bytes": (ctypes.c_size_t, [_P]),
    "tw_reserve_batch": (_S, [_P, _I]),
    "tw_batch_tiles": (_S, [_P, _P]),
    "tw_set_batch_tiles": (_S, [_P, _P]),
    "tw_autotune_pick": (_I, [_I, _P]),
    "tw_autotune_clear_cache": (None, []),
    "tw_batch_capacity": (_I, [_P]),
    "tw_infer_batch": (_S, [_P, _I, _I, _P, _P, _P, _P, _P]),
    "tw_sample_posterior_batch": (_S, [_P, _I, _I, _P, _P, _P, _P, _D, _P, _P]),
    "tw_forecast_batch": (_S, [_P, _I, _I, _P, _P, _P, _P]),
    "tw_capture_begin": (_S, [_P, _P]),
    "tw_capture_end": (_S, [_P, _P, ctypes.POINTER(_P)]),
    "tw_graph_launch": (_S, [_P, _P]),
    "tw_graph_kernel_count": (_I, [_P]),
    "tw_graph_destroy": (None, [_P]),
    "tw_serve_replay": (_S, [_P, _I, _I, _P, _P, _P, _I, _P, _I, _I, _P, _P, _P, _P, _P]),
    "tw_serve_simulate": (_S, [_I, _P, _I, _I, _D, _D, _P, _P]),
    "tw_qoi_build": (_S, [_P, _P]),
    "tw_qoi_apply": (_S, [_P, _I, _P, _P, _P]),
    "tw_qoi_variance": (_S, [_P, _P, _P]),
    "tw_qoi_covariance": (_S, [_P, _P, _P]),
}

_lib = None


class InferStats(ctypes.Structure):
    _fields_ = [("ir_iters", ctypes.c_int), ("resid_rel", ctypes.c_double)]


class ServeStats(ctypes.Structure):
    _fields_ = [("batches", ctypes.c_int), ("max_batch", ctypes.c_int),
                ("mean_batch", ctypes.c_double), ("makespan_s", ctypes.c_double),
                ("busy_s", ctypes.c_double), ("lanes", ctypes.c_int),
                ("max_in_flight", ctypes.c_int)]


class Tiles(ctypes.Structure):
    """Tiles of the batched products (tw_tiles)."""
    _fields_ = [("adj_tile", ctypes.c_int), ("adj_rw", ctypes.c_int), ("fwd_lanes", ctypes.c_int),
                ("adj_tile_ms", ctypes.c_double), ("adj_rw_ms", ctypes.c_double),
                ("fwd_lanes_ms", ctypes.c_double), ("tuned", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TwError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")


def lib_path() -> str:
    return LIB_PATH


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libtw.so and declare the C signatures.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "(the CUDA library is required; there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _stream_ptr(stream) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _dev(t, dtype=None, shape=None, name="tensor"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """An online-inversion context on one GPU (wraps tw_ctx)."""

    def __init__(self, Nd, Nq, Nx, Ny, Nt, Lx=1.0, Ly=1.0, keep=KEEP_FP64, device=0):
        self.lib = load()
        self.Nd, self.Nq, self.Nx, self.Ny, self.Nt = Nd, Nq, Nx, Ny, Nt
        self.Nm = Nx * Ny
        self.device = device
        self.keep = keep
        h = ctypes.c_void_p()
        st = self.lib.tw_create(ctypes.byref(h), Nd, Nq, Nx, Ny, Nt, Lx, Ly, keep, device)
        if st != OK:
            raise TwError(st, "tw_create failed")
        self.h = h

    # ------------------------------------------------------------ util
    def _check(self, st):
        if st != OK:
            raise TwError(st, self.lib.tw_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.tw_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def rows(self, which):
        return self.Nd if which == MAP_F else self.Nq

    def device_bytes(self) -> int:
        return int(self.lib.tw_device_bytes(self.h))

    def check(self, stream=None):
        """Synchronise and raise on errors recorded by kernels."""
        self._check(self.lib.tw_check(self.h, _stream_ptr(stream)))

    # ----------------------------------------------------------- setup
    def set_block_column(self, which, row0, col, stream=None):
        import torch
        nrows = col.shape[1]
        p = _dev(col, torch.float64, (self.Nt, nrows, self.Nm), "col")
        self._check(self.lib.tw_set_block_column(self.h, which, row0, nrows, p, _stream_ptr(stream)))

    def set_prior(self, nu=1.0, ell=0.1, var=1.0):
        self._check(self.lib.tw_set_prior(self.h, nu, ell, var))

    # ---------------------------------------------------------- applies
    def p2o_apply(self, which, prec, x, out=None, stream=None):
        import torch
        x = x if x.dim() == 3 else x.unsqueeze(0)
        nrhs = x.shape[0]
        px = _dev(x, torch.float64, (nrhs, self.Nt, self.Nm), "x")
        if out is None:
            out = torch.empty((nrhs, self.Nt, self.rows(which)), dtype=torch.float64, device=x.device)
        po = _dev(out, torch.float64, (nrhs, self.Nt, self.rows(which)), "out")
        self._check(self.lib.tw_p2o_apply(self.h, which, prec, nrhs, px, po, _stream_ptr(stream)))
        return out

    def p2o_apply_noalloc(self, which, prec, x, out, stream=None):
        """F x like p2o_apply, through the entry point that allocates nothing.

        `out` must be given: this call path creates no tensors either.
        """
        import torch
        nrhs = x.shape[0]
        px = _dev(x, torch.float64, (nrhs, self.Nt, self.Nm), "x")
        po = _dev(out, torch.float64, (nrhs, self.Nt, self.rows(which)), "out")
        self._check(self.lib.tw_p2o_apply_noalloc(self.h, which, prec, nrhs, px, po,
                                                  _stream_ptr(stream)))
        return out

    def p2o_adjoint(self, which, prec, y, out=None, stream=None):
        import torch
        y = y if y.dim() == 3 else y.unsqueeze(0)
        nrhs = y.shape[0]
        py = _dev(y, torch.float64, (nrhs, self.Nt, self.rows(which)), "y")
        if out is None:
            out = torch.empty((nrhs, self.Nt, self.Nm), dtype=torch.float64, device=y.device)
        po = _dev(out, torch.float64, (nrhs, self.Nt, self.Nm), "out")
        self._check(self.lib.tw_p2o_adjoint(self.h, which, prec, nrhs, py, po, _stream_ptr(stream)))
        return out

    def prior_apply(self, x, power=1.0, out=None, stream=None):
        import torch
        x = x if x.dim() == 3 else x.unsqueeze(0)
        nrhs = x.shape[0]
        px = _dev(x, torch.float64, (nrhs, self.Nt, self.Nm), "x")
        if out is None:
            out = torch.empty_like(x)
        po = _dev(out, torch.float64, (nrhs, self.Nt, self.Nm), "out")
        self._check(self.lib.tw_prior_apply(self.h, power, nrhs, px, po, _stream_ptr(stream)))
        return out

    # ------------------------------------------------------------ solve
    def factor_K(self, noise_var, stream=None):
        self._check(self.lib.tw_factor_K(self.h, float(noise_var), _stream_ptr(stream)))

    def factor_bytes(self) -> int:
        return int(self.lib.tw_factor_bytes(self.h))

    def save_factor(self, path=None, stream=None):
        """Phase-2 checkpoint of the FP64 factor: a numpy uint8 array (also
        written to `path` when given)."""
        import numpy as np
        n = self.factor_bytes()
        if n == 0:
            raise TwError(4, "no FP64 factor to save (factor_K first)")
        buf = np.empty(n, dtype=np.uint8)
        self._check(self.lib.tw_save_factor(self.h, buf.ctypes.data, n, _stream_ptr(stream)))
        if path is not None:
            buf.tofile(path)
        return buf

    def load_factor(self, src, stream=None):
        """Load a checkpoint written by save_factor (array or file path)."""
        import numpy as np
        buf = np.fromfile(src, dtype=np.uint8) if isinstance(src, (str, os.PathLike)) else src
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        self._check(self.lib.tw_load_factor(self.h, buf.ctypes.data, buf.size, _stream_ptr(stream)))

    def set_refinement(self, steps):
        self._check(self.lib.tw_set_refinement(self.h, int(steps)))

    def set_solver(self, solver):
        self._check(self.lib.tw_set_solver(self.h, int(solver)))

    def refinement_steps(self) -> int:
        return int(self.lib.tw_refinement_steps(self.h))

    def infer(self, prec, d, windows=None, out=None, stats=False, stream=None):
        """Posterior mean for d [nrhs][Nt][Nd]; windows: per-rhs Nt' (None = Nt)."""
        import torch
        d = d if d.dim() == 3 else d.unsqueeze(0)
        nrhs = d.shape[0]
        pd = _dev(d, torch.float64, (nrhs, self.Nt, self.Nd), "d")
        if out is None:
            out = torch.empty((nrhs, self.Nt, self.Nm), dtype=torch.float64, device=d.device)
        po = _dev(out, torch.float64, (nrhs, self.Nt, self.Nm), "m")
        win = None
        if windows is not None:
            if len(windows) != nrhs:
                raise ValueError("one window per right-hand side")
            win = (ctypes.c_int * nrhs)(*[int(w) for w in windows])
        st = InferStats() if stats else None
        self._check(self.lib.tw_infer(self.h, prec, nrhs, win, pd, po,
                                      ctypes.byref(st) if st is not None else None,
                                      _stream_ptr(stream)))
        return (out, st) if stats else out

    def _windows(self, windows, nrhs):
        if windows is None:
            return None
        if len(windows) != nrhs:
            raise ValueError("one window per right-hand side")
        return (ctypes.c_int * nrhs)(*[int(w) for w in windows])

    def solve_K(self, prec, d, windows=None, out=None, stream=None):
        """y = K'^{-1} d' for d [nrhs][Nt][Nd]."""
        import torch
        d = d if d.dim() == 3 else d.unsqueeze(0)
        nrhs = d.shape[0]
        pd = _dev(d, torch.float64, (nrhs, self.Nt, self.Nd), "d")
        out = torch.empty_like(d) if out is None else out
        po = _dev(out, torch.float64, (nrhs, self.Nt, self.Nd), "y")
        self._check(self.lib.tw_solve_K(self.h, prec, nrhs, self._windows(windows, nrhs), pd, po,
                                        _stream_ptr(stream)))
        return out

    def apply_K(self, x, windows=None, out=None, stream=None):
        """K' x with the stored K."""
        import torch
        x = x if x.dim() == 3 else x.unsqueeze(0)
        nrhs = x.shape[0]
        px = _dev(x, torch.float64, (nrhs, self.Nt, self.Nd), "x")
        out = torch.empty_like(x) if out is None else out
        po = _dev(out, torch.float64, (nrhs, self.Nt, self.Nd), "out")
        self._check(self.lib.tw_apply_K(self.h, nrhs, self._windows(windows, nrhs), px, po,
                                        _stream_ptr(stream)))
        return out

    def sample_posterior(self, d, z_m, z_n, sigma, windows=None, out=None, stream=None):
        """Perturb-then-condition posterior samples; d, z_n [ns][Nt][Nd], z_m [ns][Nt][Nm]."""
        import torch
        ns = z_m.shape[0]
        pd = _dev(d, torch.float64, (ns, self.Nt, self.Nd), "d")
        pzm = _dev(z_m, torch.float64, (ns, self.Nt, self.Nm), "z_m")
        pzn = _dev(z_n, torch.float64, (ns, self.Nt, self.Nd), "z_n")
        out = torch.empty_like(z_m) if out is None else out
        po = _dev(out, torch.float64, (ns, self.Nt, self.Nm), "samples")
        self._check(self.lib.tw_sample_posterior(self.h, ns, self._windows(windows, ns), pd, pzm,
                                                 pzn, float(sigma), po, _stream_ptr(stream)))
        return out

    def infer_forecast(self, prec, d, windows=None, m=None, q=None, stream=None):
        """Posterior means m and forecasts q = F_q m of d [nrhs][Nt][Nd] in one call."""
        import torch
        d = d if d.dim() == 3 else d.unsqueeze(0)
        nrhs = d.shape[0]
        pd = _dev(d, torch.float64, (nrhs, self.Nt, self.Nd), "d")
        if m is None:
            m = torch.empty((nrhs, self.Nt, self.Nm), dtype=torch.float64, device=d.device)
        if q is None:
            q = torch.empty((nrhs, self.Nt, self.Nq), dtype=torch.float64, device=d.device)
        pm = _dev(m, torch.float64, (nrhs, self.Nt, self.Nm), "m")
        pq = _dev(q, torch.float64, (nrhs, self.Nt, self.Nq), "q")
        win = None
        if windows is not None:
            if len(windows) != nrhs:
                raise ValueError("one window per right-hand side")
            win = (ctypes.c_int * nrhs)(*[int(w) for w in windows])
        self._check(self.lib.tw_infer_forecast(self.h, prec, nrhs, win, pd, pm, pq, None,
                                               _stream_ptr(stream)))
        return m, q

    def forecast(self, prec, m, out=None, stream=None):
        import torch
        m = m if m.dim() == 3 else m.unsqueeze(0)
        nrhs = m.shape[0]
        pm = _dev(m, torch.float64, (nrhs, self.Nt, self.Nm), "m")
        if out is None:
            out = torch.empty((nrhs, self.Nt, self.Nq), dtype=torch.float64, device=m.device)
        po = _dev(out, torch.float64, (nrhs, self.Nt, self.Nq), "q")
        self._check(self.lib.tw_forecast(self.h, prec, nrhs, pm, po, _stream_ptr(stream)))
        return out

    # -------------------------------------------------------- batches
    def reserve_batch(self, bmax: int):
        """Workspaces for batches of up to bmax right-hand sides (after factor_K)."""
        self._check(self.lib.tw_reserve_batch(self.h, int(bmax)))

    def batch_capacity(self) -> int:
        return int(self.lib.tw_batch_capacity(self.h))

    def batch_tiles(self) -> Tiles:
        """The tiles of the batched products (measured at reserve_batch)."""
        t = Tiles()
        self._check(self.lib.tw_batch_tiles(self.h, ctypes.byref(t)))
        return t

    def set_batch_tiles(self, adj_tile: int, adj_rw: int, fwd_lanes: int):
        t = Tiles(int(adj_tile), int(adj_rw), int(fwd_lanes), -1.0, -1.0, -1.0, 0)
        self._check(self.lib.tw_set_batch_tiles(self.h, ctypes.byref(t)))

    def infer_batch(self, prec, d, windows_dev, m=None, q=None, forecast=True, stream=None):
        """Posterior means (and forecasts) of d [B][Nt][Nd]; windows_dev: int32 CUDA tensor [B]."""
        import torch
        B = d.shape[0]
        pd = _dev(d, torch.float64, (B, self.Nt, self.Nd), "d")
        pw = _dev(windows_dev, torch.int32, (B,), "windows")
        if m is None:
            m = torch.empty((B, self.Nt, self.Nm), dtype=torch.float64, device=d.device)
        pm = _dev(m, torch.float64, (B, self.Nt, self.Nm), "m")
        pq = None
        if forecast:
            if q is None:
                q = torch.empty((B, self.Nt, self.Nq), dtype=torch.float64, device=d.device)
            pq = _dev(q, torch.float64, (B, self.Nt, self.Nq), "q")
        self._check(self.lib.tw_infer_batch(self.h, prec, B, pw, pd, pm, pq, _stream_ptr(stream)))
        return (m, q) if forecast else m

    def sample_posterior_batch(self, prec, d, z_m, z_n, sigma, windows_dev, out=None, stream=None):
        import torch
        ns = z_m.shape[0]
        pd = _dev(d, torch.float64, (ns, self.Nt, self.Nd), "d")
        pzm = _dev(z_m, torch.float64, (ns, self.Nt, self.Nm), "z_m")
        pzn = _dev(z_n, torch.float64, (ns, self.Nt, self.Nd), "z_n")
        pw = _dev(windows_dev, torch.int32, (ns,), "windows")
        out = torch.empty_like(z_m) if out is None else out
        po = _dev(out, torch.float64, (ns, self.Nt, self.Nm), "samples")
        self._check(self.lib.tw_sample_posterior_batch(self.h, prec, ns, pw, pd, pzm, pzn,
                                                       float(sigma), po, _stream_ptr(stream)))
        return out

    def forecast_batch(self, prec, m, windows_dev=None, out=None, stream=None):
        import torch
        B = m.shape[0]
        pm = _dev(m, torch.float64, (B, self.Nt, self.Nm), "m")
        pw = None if windows_dev is None else _dev(windows_dev, torch.int32, (B,), "windows")
        if out is None:
            out = torch.empty((B, self.Nt, self.Nq), dtype=torch.float64, device=m.device)
        po = _dev(out, torch.float64, (B, self.Nt, self.Nq), "q")
        self._check(self.lib.tw_forecast_batch(self.h, prec, B, pw, pm, po, _stream_ptr(stream)))
        return out

    def serve_replay(self, prec, arrival_s, event, window, event_data, max_batch, stream,
                     q_out=True, m_out=False, lanes=0):
        """Replay a request trace (host arrays) with continuous batching over
        up to `lanes` batches in flight (0: as many as device memory allows, <= 4).

        Returns (latency_ms [n], q [n][Nt][Nq] or None, m [n][Nt][Nm] or None, ServeStats)."""
        import numpy as np
        import torch
        n = len(arrival_s)
        arr = np.ascontiguousarray(arrival_s, dtype=np.float64)
        ev = np.ascontiguousarray(event, dtype=np.int32)
        win = np.ascontiguousarray(window, dtype=np.int32)
        ne = event_data.shape[0]
        pe = _dev(event_data, torch.float64, (ne, self.Nt, self.Nd), "event_data")
        lat = np.zeros(n, dtype=np.float64)
        q = np.zeros((n, self.Nt, self.Nq), dtype=np.float64) if q_out else None
        m = np.zeros((n, self.Nt, self.Nm), dtype=np.float64) if m_out else None
        st = ServeStats()
        ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p) if a is not None else None
        self._check(self.lib.tw_serve_replay(self.h, prec, n, ptr(arr), ptr(ev), ptr(win), ne, pe,
                                             int(max_batch), int(lanes), ptr(lat), ptr(q), ptr(m),
                                             ctypes.byref(st), _stream_ptr(stream)))
        return lat, q, m, st

    # -------------------------------------------------------- QoI (Phase 3 / 4)
    def qoi_build(self, stream=None):
        """Precompute the data-to-QoI map, W, C and the QoI posterior variances."""
        self._check(self.lib.tw_qoi_build(self.h, _stream_ptr(stream)))

    def qoi_apply(self, d, out=None, stream=None):
        """q = Q d for d [nrhs][Nt][Nd]."""
        import torch
        d = d if d.dim() == 3 else d.unsqueeze(0)
        nrhs = d.shape[0]
        pd = _dev(d, torch.float64, (nrhs, self.Nt, self.Nd), "d")
        if out is None:
            out = torch.empty((nrhs, self.Nt, self.Nq), dtype=torch.float64, device=d.device)
        po = _dev(out, torch.float64, (nrhs, self.Nt, self.Nq), "q")
        self._check(self.lib.tw_qoi_apply(self.h, nrhs, pd, po, _stream_ptr(stream)))
        return out

    def qoi_variance(self, stream=None):
        import torch
        out = torch.empty((self.Nt, self.Nq), dtype=torch.float64, device=torch.device("cuda", self.device))
        self._check(self.lib.tw_qoi_variance(self.h, _dev(out, torch.float64), _stream_ptr(stream)))
        return out

    def qoi_covariance(self, stream=None):
        import torch
        nq = self.Nq * self.Nt
        out = torch.empty((nq, nq), dtype=torch.float64, device=torch.device("cuda", self.device))
        self._check(self.lib.tw_qoi_covariance(self.h, _dev(out, torch.float64), _stream_ptr(stream)))
        return out

    def capture(self, stream):
        """Context manager: batched calls on `stream` inside it are recorded into a Graph."""
        return _Capture(self, stream)

    # -------------------------------------------------------- profiling
    def profile(self, on=True):
        self._check(self.lib.tw_profile_enable(self.h, 1 if on else 0))

    def profile_read(self, reset=True):
        """{phase: (ms, launches)} of the timed phases since the last reset (synchronises)."""
        n = len(PHASES)
        ms = (ctypes.c_double * n)()
        calls = (ctypes.c_longlong * n)()
        self._check(self.lib.tw_profile_read(self.h, ms, calls, 1 if reset else 0))
        return {PHASES[i]: (ms[i], calls[i]) for i in range(n)}


class Graph:
    """An instantiated CUDA graph of batched calls (tw_graph)."""

    def __init__(self, lib, handle):
        self.lib, self.h = lib, handle

    def launch(self, stream=None):
        st = self.lib.tw_graph_launch(self.h, _stream_ptr(stream))
        if st != OK:
            raise TwError(st, "tw_graph_launch failed")

    def kernel_count(self) -> int:
        return int(self.lib.tw_graph_kernel_count(self.h))

    def close(self):
        if self.h:
            self.lib.tw_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Capture:
    def __init__(self, ctx, stream):
        self.ctx, self.stream, self.graph = ctx, stream, None

    def __enter__(self):
        self.ctx._check(self.ctx.lib.tw_capture_begin(self.ctx.h, _stream_ptr(self.stream)))
        return self

    def __exit__(self, et, ev, tb):
        h = ctypes.c_void_p()
        st = self.ctx.lib.tw_capture_end(self.ctx.h, _stream_ptr(self.stream), ctypes.byref(h))
        if et is None:
            self.ctx._check(st)
            self.graph = Graph(self.ctx.lib, h)
        elif h:
            self.ctx.lib.tw_graph_destroy(h)
        return False


def serve_simulate(arrival_s, max_batch, cost_ms, cost_ms_per_req, lanes=1):
    """The serving policy on a virtual clock with `lanes` batch lanes:
    (latency_ms [n], batch index [n] in start order).  Host only."""
    import numpy as np
    arr = np.ascontiguousarray(arrival_s, dtype=np.float64)
    n = len(arr)
    lat = np.zeros(n, dtype=np.float64)
    bid = np.zeros(n, dtype=np.int32)
    st = load().tw_serve_simulate(n, arr.ctypes.data_as(ctypes.c_void_p), int(max_batch), int(lanes),
                                  float(cost_ms), float(cost_ms_per_req),
                                  lat.ctypes.data_as(ctypes.c_void_p),
                                  bid.ctypes.data_as(ctypes.c_void_p))
    if st != OK:
        raise TwError(st, "tw_serve_simulate failed")
    return lat, bid


def autotune_pick(ms) -> int:
    """The tile tuner's selection rule on a list of times (host only)."""
    import numpy as np
    a = np.ascontiguousarray(ms, dtype=np.float64)
    return int(load().tw_autotune_pick(len(a), a.ctypes.data_as(ctypes.c_void_p)))


def autotune_clear_cache():
    load().tw_autotune_clear_cache()


def kernel_launches() -> int:
    """Kernels enqueued by libtw.so in this process."""
    return int(load().tw_kernel_launches())
