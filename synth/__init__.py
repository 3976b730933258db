"""Seeded synthetic workloads shared by the FP64 oracle and the CUDA path.

This package only *draws and evaluates inputs*: acquisition geometry, the
parameters of the hyperbolic-event kernel, Ricker wavelets, virtual points,
the Marchenko window cut-offs and the direct-arrival focusing function.  It
holds none of the multi-dimensional-convolution or LSQR arithmetic; the
oracle and the GPU library both receive what it returns as plain inputs.

The paper's benchmark kernel is a finite-difference reflection response of a
3D density model with 9801 co-located sources and receivers on a regular
grid, truncated to the first ``n_wmax`` frequencies and stored as complex64
(Section "Benchmarking the Multi-Dimensional Convolution operator", Table 1).
That dataset is not available, so the kernel here is a sum of hyperbolic
events with a 15 Hz Ricker spectrum on the same kind of co-located square
grid, frequency-major ``[nf][nr][ns]`` complex, which keeps the paper's
shapes and structure:

    G[k, r, s] = scale * sum_e a_e W(f_k) exp(-i 2 pi f_k sqrt(t0_e^2 + |x_r - x_s|^2 / v_e^2))

with f_k = k / (nt dt), W the Ricker amplitude spectrum, t0_e ~ U(0.2, 0.8) s,
v_e ~ U(1500, 3000) m/s and a_e ~ N(0, 1), drawn from NumPy's PCG64 with the
seed ``20201122 + config number`` in that order (all t0, then all v, then all
a, then virtual-point positions).
"""
from __future__ import annotations

import dataclasses
import json
import math
import os
from typing import Optional

import numpy as np

SEED_BASE = 20201122
RICKER_FP = 15.0          # Hz, dominant frequency of the Ricker wavelet
GRID_DX = 20.0            # m, grid spacing of sources and receivers
POINT_SPEED = 2000.0      # m/s, speed used for virtual-point travel times

_MANIFEST = os.path.join(os.path.dirname(os.path.abspath(__file__)), "manifest.json")


# --------------------------------------------------------------------------- wavelets
def ricker_spectrum(f, fp: float = RICKER_FP):
    """Amplitude spectrum of a Ricker wavelet, W(f) = 2/sqrt(pi) f^2/fp^3 exp(-f^2/fp^2)."""
    f = np.asarray(f, dtype=np.float64)
    return (2.0 / math.sqrt(math.pi)) * f * f / fp ** 3 * np.exp(-(f * f) / (fp * fp))


def ricker(t, fp: float = RICKER_FP):
    """Zero-phase Ricker wavelet r(t) = (1 - 2 pi^2 fp^2 t^2) exp(-pi^2 fp^2 t^2)."""
    t = np.asarray(t, dtype=np.float64)
    a = (math.pi * fp * t) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


# --------------------------------------------------------------------------- geometry
def grid_xy(n_side: int, dx: float = GRID_DX):
    """Co-located source/receiver grid; flat index = iy * n_side + ix (x fastest)."""
    ix = np.arange(n_side * n_side) % n_side
    iy = np.arange(n_side * n_side) // n_side
    return np.stack([ix * dx, iy * dx], axis=1).astype(np.float64)


def irregular_subset(n_side: int, fraction: float = 0.5, seed: int = 0):
    """Sorted flat indices of a random subset of the n_side x n_side grid (an irregular geometry,
    as in the paper's example that keeps half of the regular sources and receivers)."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 7919 + seed))
    n = n_side * n_side
    return np.sort(rng.choice(n, size=max(1, int(round(fraction * n))), replace=False))


def voronoi_areas(xy: np.ndarray, lo: float, hi: float, res: int = 2048):
    """Areal extent of each point's Voronoi cell inside the square [lo, hi]^2 (m^2), from a
    res x res raster of cell centres assigned to their nearest point.  Input weights for the
    spatial integration of irregular geometries; they sum to (hi - lo)^2."""
    xy = np.asarray(xy, np.float64)
    h = (hi - lo) / res
    c = lo + h * (np.arange(res) + 0.5)
    counts = np.zeros(len(xy), np.int64)
    for r0 in range(0, res, 64):                  # rows of the raster in blocks
        px, py = np.meshgrid(c, c[r0:r0 + 64], indexing="xy")
        d2 = (px[..., None] - xy[:, 0]) ** 2 + (py[..., None] - xy[:, 1]) ** 2
        counts += np.bincount(np.argmin(d2, axis=-1).ravel(), minlength=len(xy))
    return counts * h * h


def signed_time_index(nt: int):
    """Signed circular time sample tau(t) = t for t < nt/2, else t - nt."""
    t = np.arange(nt)
    return np.where(t < nt // 2, t, t - nt)


# --------------------------------------------------------------------------- configs
@dataclasses.dataclass
class Config:
    number: int
    name: str
    n_side: int
    nt: int
    dt: float
    nf: int
    n_events: int
    nv: int
    z_point: float
    point_grid: int = 0          # >0: virtual points on a point_grid x point_grid lattice
    normalise: bool = False      # scale G so that ||C||_2 is 0.5 (manifest constant)
    niter: int = 20

    @property
    def nr(self) -> int:
        return self.n_side * self.n_side

    @property
    def ns(self) -> int:
        return self.n_side * self.n_side

    @property
    def dr(self) -> float:
        return GRID_DX * GRID_DX          # areal integration weight of one receiver

    @property
    def seed(self) -> int:
        return SEED_BASE + self.number

    @property
    def freqs(self):
        return np.arange(self.nf, dtype=np.float64) / (self.nt * self.dt)

    def with_(self, **kw) -> "Config":
        return dataclasses.replace(self, **kw)


CONFIGS = {
    1: Config(1, "mdc-441x441-nt256-nf64-c64", 21, 256, 0.004, 64, 5, 1, 600.0),
    2: Config(2, "mdc-3721x3721-nt1024-nf200-c64", 61, 1024, 0.004, 200, 20, 1, 600.0),
    3: Config(3, "mdc-8281x8281-nt1024-nf160", 91, 1024, 0.004, 160, 20, 1, 600.0),
    4: Config(4, "marchenko-1681x1681-nt512-nf150-nv256", 41, 512, 0.004, 150, 20, 256, 800.0,
              point_grid=16, normalise=True, niter=20),
    # serving: the 8281-trace kernel of config 3 (same draws), normalised like the redatuming
    # kernel; virtual points, nv and iterations are drawn per job by the serving workload
    5: Config(3, "serving-8281x8281-nt1024-nf160", 91, 1024, 0.004, 160, 20, 1, 800.0,
              normalise=True, niter=20),
    # the paper's Full geometry (Table 1): 9801 co-located sources and receivers, 300 frequencies;
    # the 1201-sample traces padded to nt = 2048
    6: Config(80, "paper-full-9801x9801-nt2048-nf300", 99, 2048, 0.004, 300, 20, 1, 600.0),
}


def config(number: int, **overrides) -> Config:
    return CONFIGS[number].with_(**overrides) if overrides else CONFIGS[number]


def tiny(n_side=3, nt=32, nf=None, n_events=3, nv=2, z_point=300.0, dt=0.004, number=90,
         point_grid=0, normalise=False) -> Config:
    """A small configuration for brute-force and dense-matrix checks."""
    return Config(number, f"tiny-{n_side}-{nt}", n_side, nt, dt, nf if nf else nt // 4 + 1,
                  n_events, nv, z_point, point_grid=point_grid, normalise=normalise)


# --------------------------------------------------------------------------- draws
@dataclasses.dataclass
class Draw:
    t0: np.ndarray        # [E] s
    vel: np.ndarray       # [E] m/s
    amp: np.ndarray       # [E]
    points: np.ndarray    # [nv, 2] m (x, y) of virtual points
    scale: float          # multiplies G


def draw(cfg: Config) -> Draw:
    rng = np.random.Generator(np.random.PCG64(cfg.seed))
    E = cfg.n_events
    t0 = rng.uniform(0.2, 0.8, size=E)
    vel = rng.uniform(1500.0, 3000.0, size=E)
    amp = rng.standard_normal(size=E)
    extent = GRID_DX * (cfg.n_side - 1)
    if cfg.point_grid > 0:
        g = cfg.point_grid
        off = 0.5 * (extent - GRID_DX * (g - 1))
        px = off + GRID_DX * (np.arange(g * g) % g)
        py = off + GRID_DX * (np.arange(g * g) // g)
        points = np.stack([px, py], axis=1)
        if cfg.nv != g * g:
            points = points[: cfg.nv]
    else:
        points = rng.uniform(0.0, extent, size=(cfg.nv, 2))
    scale = kernel_scale(cfg) if cfg.normalise else 1.0
    return Draw(t0, vel, amp, points, scale)


def kernel_scale(cfg: Config) -> float:
    """Kernel normalisation for the redatuming configurations (stored constant).

    The constant is written by ``synth/normalise_kernel.py`` so that the MDC
    operator built from the scaled kernel has 2-norm 0.5; it is then an input
    like any other drawn parameter.
    """
    if os.path.exists(_MANIFEST):
        with open(_MANIFEST) as fh:
            man = json.load(fh)
        key = _scale_key(cfg)
        if key in man:
            return float(man[key]["scale"])
    raise KeyError(f"no kernel scale stored for {_scale_key(cfg)}; run synth/normalise_kernel.py")


def _scale_key(cfg: Config) -> str:
    return f"n{cfg.n_side}_nt{cfg.nt}_nf{cfg.nf}_E{cfg.n_events}_seed{cfg.seed}"


# --------------------------------------------------------------------------- kernel
def event_times(cfg: Config, d: Draw, rows, cols):
    """Travel times sqrt(t0^2 + |x_r - x_s|^2 / v^2) for each event, [E, len(rows), len(cols)]."""
    xy = grid_xy(cfg.n_side)
    rr = xy[np.asarray(rows)]
    ss = xy[np.asarray(cols)]
    d2 = ((rr[:, None, :] - ss[None, :, :]) ** 2).sum(-1)
    return np.sqrt(d.t0[:, None, None] ** 2 + d2[None] / (d.vel[:, None, None] ** 2))


def kernel(cfg: Config, d: Optional[Draw] = None, ks=None, rows=None, cols=None):
    """Hyperbolic-event kernel G[k, r, s] in complex128, for the requested index subsets."""
    if d is None:
        d = draw(cfg)
    ks = np.arange(cfg.nf) if ks is None else np.asarray(ks)
    rows = np.arange(cfg.nr) if rows is None else np.asarray(rows)
    cols = np.arange(cfg.ns) if cols is None else np.asarray(cols)
    f = ks.astype(np.float64) / (cfg.nt * cfg.dt)
    W = ricker_spectrum(f)
    tau = event_times(cfg, d, rows, cols)                   # [E, R, S]
    out = np.zeros((len(ks), len(rows), len(cols)), dtype=np.complex128)
    for ik in range(len(ks)):
        # phase in cycles, reduced before the trigonometric evaluation
        cyc = f[ik] * tau
        cyc = cyc - np.rint(cyc)
        ph = np.exp(-2j * np.pi * cyc)                      # [E, R, S]
        out[ik] = W[ik] * np.tensordot(d.amp, ph, axes=(0, 0))
    return out * d.scale


def kernel_between(cfg: Config, d: Draw, xy_rows, xy_cols, ks=None):
    """The hyperbolic-event formula of ``kernel`` between two point sets [nr, 2] and [ns, 2] (m),
    e.g. surface receivers x_S by focusing points x_F for a stand-in down-going Green's
    function G+ of Eq. 8; complex128 [len(ks), nr, ns]."""
    ks = np.arange(cfg.nf) if ks is None else np.asarray(ks)
    xr = np.asarray(xy_rows, np.float64)
    xs = np.asarray(xy_cols, np.float64)
    d2 = ((xr[:, None, :] - xs[None, :, :]) ** 2).sum(-1)
    tau = np.sqrt(d.t0[:, None, None] ** 2 + d2[None] / (d.vel[:, None, None] ** 2))
    f = ks.astype(np.float64) / (cfg.nt * cfg.dt)
    W = ricker_spectrum(f)
    out = np.zeros((len(ks), len(xr), len(xs)), dtype=np.complex128)
    for ik in range(len(ks)):
        cyc = f[ik] * tau
        cyc = cyc - np.rint(cyc)
        out[ik] = W[ik] * np.tensordot(d.amp, np.exp(-2j * np.pi * cyc), axes=(0, 0))
    return out * d.scale


def focus_lattice(n: int, spacing: float, centre: float):
    """n x n focusing points [n*n, 2] (m) on a square lattice centred at (centre, centre)."""
    off = centre - 0.5 * spacing * (n - 1)
    i = np.arange(n * n)
    return np.stack([off + spacing * (i % n), off + spacing * (i // n)], axis=1).astype(np.float64)


# --------------------------------------------------------------------------- inputs
def point_times(cfg: Config, d: Draw, z: Optional[float] = None):
    """One-way times from each virtual point (depth z) to each grid location, [ns, nv] s."""
    z = cfg.z_point if z is None else z
    xy = grid_xy(cfg.n_side)
    dd = ((xy[:, None, :] - d.points[None, :, :]) ** 2).sum(-1)
    return np.sqrt(z * z + dd) / POINT_SPEED


def ricker_traces(cfg: Config, d: Optional[Draw] = None):
    """MDC input x[t, s, v] = r(t dt - t_sv), a Ricker at each point's travel time (float32)."""
    if d is None:
        d = draw(cfg)
    tsv = point_times(cfg, d)
    t = np.arange(cfg.nt, dtype=np.float64) * cfg.dt
    x = ricker(t[:, None, None] - tsv[None])
    return x.astype(np.float32)


def random_traces(cfg: Config, nv: int, seed_offset: int = 0, nspace: Optional[int] = None):
    """Gaussian traces [nt, nspace, nv] float32 for dot-product and linearity checks."""
    rng = np.random.Generator(np.random.PCG64(cfg.seed * 1000 + 17 + seed_offset))
    n = cfg.ns if nspace is None else nspace
    return rng.standard_normal(size=(cfg.nt, n, nv)).astype(np.float32)


def direct_times(cfg: Config, d: Optional[Draw] = None):
    """Direct-arrival times t_d(s, v) from each focusing point at z_point, [ns, nv] s."""
    if d is None:
        d = draw(cfg)
    return point_times(cfg, d)


def window_cutoffs(cfg: Config, d: Optional[Draw] = None, margin: int = 4):
    """Marchenko window cut-offs c[s, v] = round(t_d / dt) - margin (int32 samples).

    The window passes a sample when |tau(t)| < c[s, v] in signed circular time.
    """
    td = direct_times(cfg, d)
    return (np.rint(td / cfg.dt).astype(np.int64) - margin).astype(np.int32)


def direct_focusing(cfg: Config, d: Optional[Draw] = None):
    """Initial focusing function f_d+[t, s, v]: the time-reversed direct arrival (float32).

    A Ricker centred at signed time -t_d(s, v), evaluated at the exact delay.
    """
    td = direct_times(cfg, d)
    tau = signed_time_index(cfg.nt).astype(np.float64) * cfg.dt
    return ricker(tau[:, None, None] + td[None]).astype(np.float32)
