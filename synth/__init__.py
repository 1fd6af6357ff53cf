"""Seeded synthetic inputs for the online Bayesian inversion (both sides use these).

This module is the only code shared by the CPU oracle and the GPU path.  It
produces inputs and nothing else: sensor and forecast-point positions, the
parameter grid, the synthetic p2o / p2q first block column that stands in for
the offline adjoint wave propagations (Sec. "FFT-based Hessian matvecs": the
first block column {F_i1} of the block lower-triangular Toeplitz map), white
Gaussian vectors z, and the request traces of the serving workload.  None of
the method's arithmetic (Toeplitz applies, the Matern prior, K, its factor,
the solves) lives here.

Workload recipe (synthetic stand-ins for the Cascadia workload of the paper's
Sec. "Application to the Cascadia subduction zone", whose rupture scenario,
bathymetry and mesh are not available):

* Nd sensors and Nq forecast points drawn uniformly in [0, 1]^2 (PCG64);
* Nm = Nx * Ny parameter points on a periodic grid over [0, Lx) x [0, Ly)
  with Lx = Ly = 1, point (a, b) at (a Lx/Nx, b Ly/Ny), flat index a*Ny + b;
* Nt time steps, dt = 1/Nt, lag i = 0 .. Nt-1 (lag 0 is the paper's F_11);
* block column F_i[j, k] = exp(-((i dt - r_jk/1.5) / (2 dt))^2) / (1 + 10 r_jk)
  with r_jk the Euclidean (non-periodic) distance from point j to grid point k;
  the p2q column uses the same formula at the forecast points;
* seeds are 1000 * config + stream, one stream per kind of input.
"""
from __future__ import annotations

import dataclasses

import numpy as np

# Seed streams: seed = 1000 * config + stream (+ an index for per-event draws).
STREAM_SENSORS = 1
STREAM_QOI = 2
STREAM_EVENT_Z = 100      # + event index: white z with m_true = Gamma_pr^{1/2} z
STREAM_NOISE = 300        # + event index: white noise z_n for d = F m_true + sigma z_n
STREAM_SAMPLE_ZM = 500    # + sample index: prior draw of a posterior sample
STREAM_SAMPLE_ZN = 700    # + sample index: noise draw of a posterior sample
STREAM_TRACE = 900        # request trace of the serving workload
STREAM_WINDOWS = 901      # observation windows of the batched workload


@dataclasses.dataclass(frozen=True)
class Config:
    """Shapes of one synthetic workload (prior: Matern nu=1, length 0.1, var 1)."""

    cid: int
    Nd: int
    Nx: int
    Ny: int
    Nt: int
    Nq: int
    Lx: float = 1.0
    Ly: float = 1.0
    nu: float = 1.0
    ell: float = 0.1
    var: float = 1.0
    noise_rel: float = 0.01       # noise std = 1% of rms(F m_true) of event 0
    events: int = 1
    samples: int = 0
    operator_cid: int = 0         # configs that reuse another config's operator

    @property
    def Nm(self) -> int:
        return self.Nx * self.Ny

    @property
    def dt(self) -> float:
        return 1.0 / self.Nt

    @property
    def n(self) -> int:
        """Data-space dimension Nd * Nt (size of K)."""
        return self.Nd * self.Nt

    @property
    def op(self) -> int:
        """Config id whose seeds define sensors, forecast points and events."""
        return self.operator_cid or self.cid

    def seed(self, stream: int, index: int = 0) -> int:
        return 1000 * self.op + stream + index


CONFIGS = {
    # tiny plain FP64 case
    1: Config(1, Nd=8, Nx=16, Ny=16, Nt=32, Nq=4),
    # plain FP64 medium case
    2: Config(2, Nd=100, Nx=200, Ny=250, Nt=400, Nq=20),
    # mixed precision on the operator and data of case 2
    3: Config(3, Nd=100, Nx=200, Ny=250, Nt=400, Nq=20, operator_cid=2),
    # batched uneven windows: 64 events + 32 posterior samples, operator of case 2
    4: Config(4, Nd=100, Nx=200, Ny=250, Nt=400, Nq=20, events=64, samples=32,
              operator_cid=2),
    # serving at scale: 16 events, Poisson requests with growing windows
    5: Config(5, Nd=200, Nx=316, Ny=316, Nt=420, Nq=50, events=16),
}


def small_config(Nd: int, Nx: int, Ny: int, Nt: int, Nq: int, cid: int = 90,
                 **kw) -> Config:
    """A reduced workload with the same recipe (parity tests, profiling cases)."""
    return Config(cid, Nd=Nd, Nx=Nx, Ny=Ny, Nt=Nt, Nq=Nq, **kw)


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def sensors(cfg: Config) -> np.ndarray:
    """[Nd, 2] sensor positions, uniform in [0,1]^2."""
    return rng(cfg.seed(STREAM_SENSORS)).random((cfg.Nd, 2))


def qoi_points(cfg: Config) -> np.ndarray:
    """[Nq, 2] forecast-point positions, uniform in [0,1]^2."""
    return rng(cfg.seed(STREAM_QOI)).random((cfg.Nq, 2))


def grid_points(cfg: Config) -> np.ndarray:
    """[Nm, 2] parameter-grid coordinates, flat index a*Ny + b."""
    a = np.arange(cfg.Nx, dtype=np.float64) * (cfg.Lx / cfg.Nx)
    b = np.arange(cfg.Ny, dtype=np.float64) * (cfg.Ly / cfg.Ny)
    ga, gb = np.meshgrid(a, b, indexing="ij")
    return np.stack([ga.ravel(), gb.ravel()], axis=1)


def _kernel_np(lags: np.ndarray, r: np.ndarray, dt: float) -> np.ndarray:
    # lags [L], r [P, K] -> [L, P, K]
    t = lags.astype(np.float64)[:, None, None] * dt
    arg = (t - r[None] / 1.5) / (2.0 * dt)
    return np.exp(-arg * arg) / (1.0 + 10.0 * r[None])


def distances(points: np.ndarray, cfg: Config, cols: np.ndarray | None = None) -> np.ndarray:
    """[P, K] Euclidean distance from each point to grid points (all, or `cols`)."""
    g = grid_points(cfg)
    if cols is not None:
        g = g[np.asarray(cols)]
    diff = points[:, None, :] - g[None, :, :]
    return np.sqrt(np.sum(diff * diff, axis=2))


def block_column(cfg: Config, which: str = "F", rows=None, lags=None, cols=None) -> np.ndarray:
    """First block column, numpy FP64: [len(lags), len(rows), len(cols)].

    which: "F" (sensors, the p2o map) or "Fq" (forecast points, the p2q map).
    rows / lags / cols select sensors, lags and grid points (default: all).
    """
    pts = sensors(cfg) if which == "F" else qoi_points(cfg)
    if rows is not None:
        pts = pts[np.asarray(rows)]
    lag = np.arange(cfg.Nt) if lags is None else np.asarray(lags)
    r = distances(pts, cfg, cols)
    return _kernel_np(lag, r, cfg.dt)


def block_column_torch(cfg: Config, which: str, device, row0: int = 0, nrows: int | None = None):
    """Same block column, generated with torch on `device`: [Nt, nrows, Nm] float64.

    Used to fill large operators quickly; values agree with `block_column`
    to a few ulps (exp is evaluated by a different library).
    """
    import torch

    pts = sensors(cfg) if which == "F" else qoi_points(cfg)
    nrows = pts.shape[0] - row0 if nrows is None else nrows
    p = torch.as_tensor(pts[row0:row0 + nrows], dtype=torch.float64, device=device)
    g = torch.as_tensor(grid_points(cfg), dtype=torch.float64, device=device)
    r = torch.sqrt(((p[:, None, :] - g[None, :, :]) ** 2).sum(-1))      # [P, Nm]
    out = torch.empty((cfg.Nt, nrows, cfg.Nm), dtype=torch.float64, device=device)
    w = 1.0 / (1.0 + 10.0 * r)
    rr = r / 1.5
    for i in range(cfg.Nt):
        arg = (i * cfg.dt - rr) / (2.0 * cfg.dt)
        torch.mul(torch.exp(-arg * arg), w, out=out[i])
    return out


def white(shape, seed: int) -> np.ndarray:
    """Standard normal FP64 array from PCG64(seed)."""
    return rng(seed).standard_normal(shape)


def event_z(cfg: Config, e: int = 0) -> np.ndarray:
    """[Nt, Nm] white field of event e (m_true = Gamma_pr^{1/2} z)."""
    return white((cfg.Nt, cfg.Nm), cfg.seed(STREAM_EVENT_Z, e))


def noise_z(cfg: Config, e: int = 0) -> np.ndarray:
    """[Nt, Nd] white noise of event e (d = F m_true + sigma z_n)."""
    return white((cfg.Nt, cfg.Nd), cfg.seed(STREAM_NOISE, e))


def sample_z(cfg: Config, k: int, nt_window: int):
    """White draws (z_m [Nt, Nm], z_n [nt_window, Nd]) of posterior sample k."""
    zm = white((cfg.Nt, cfg.Nm), cfg.seed(STREAM_SAMPLE_ZM, k))
    zn = white((nt_window, cfg.Nd), cfg.seed(STREAM_SAMPLE_ZN, k))
    return zm, zn


def batch_windows(cfg: Config) -> np.ndarray:
    """Observation windows Nt' of the batched workload: uniform on {100,150,...,Nt}."""
    choices = np.arange(100, cfg.Nt + 1, 50)
    return rng(cfg.seed(STREAM_WINDOWS)).choice(choices, size=cfg.events)


@dataclasses.dataclass
class Request:
    t_arrival: float   # seconds since trace start
    event: int
    window: int        # Nt' in [lo, Nt]


def request_trace(cfg: Config, n: int = 10_000, rate: float = 200.0, lo: int = 60) -> list:
    """Poisson arrivals (mean `rate`/s), event uniform, window uniform in [lo, Nt]."""
    g = rng(cfg.seed(STREAM_TRACE))
    gaps = g.exponential(1.0 / rate, size=n)
    t = np.cumsum(gaps)
    ev = g.integers(0, cfg.events, size=n)
    win = g.integers(lo, cfg.Nt + 1, size=n)
    return [Request(float(t[i]), int(ev[i]), int(win[i])) for i in range(n)]


def sample_entries(n_total: int, count: int, seed: int) -> np.ndarray:
    """Sorted distinct flat indices in [0, n_total) drawn with a seeded
    generator: the entries at which a stored reference vector is compared."""
    g = np.random.default_rng(seed)
    return np.sort(g.choice(n_total, size=min(count, n_total), replace=False))


def nbytes_gb(x) -> float:
    return float(x) / 1e9


def check_sizes(cfg: Config) -> dict:
    """Sizes (bytes) of the main operator objects, for planning and reports."""
    Nf = cfg.Nt + 1
    return {
        "Fhat_c128": 16 * Nf * cfg.Nd * cfg.Nm,
        "Fhat_c64": 8 * Nf * cfg.Nd * cfg.Nm,
        "Fqhat_c128": 16 * Nf * cfg.Nq * cfg.Nm,
        "K_f64_full": 8 * cfg.n * cfg.n,
        "L_f64_tri": 8 * cfg.n * (cfg.n + 1) // 2,
    }

