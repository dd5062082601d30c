"""Seeded synthetic inputs shared by the CUDA path, the oracle and the bench.

This module holds workload descriptions and random inputs only: screen
samples (pixel centres and sub-rays), source and time grids, source histories
and noise draws.  It contains none of the operator's arithmetic (no ray
tracing, weights, delays, interpolation or hats), so that the oracle and the
CUDA path can both consume its arrays without sharing any of the method.

Workloads (the paper's configurations restated as sizes):
  * ``schw32``   Schwarzschild a=0, i=20 deg, 32x32 image, 8x16 source grid,
                 12 hats, 24 frames at 2 M cadence, history ending at t=0.
  * ``kerr256``  Kerr a=0.5, i=50 deg, 256x256 image with 2x2 sub-rays in the
                 photon-ring annulus, 64x128 grid, 64 hats, 256 frames at 1 M.
  * ``audit12``  12 geometries, spins {0, .5, .75, .94} x incl {20, 50, 75} at
                 the kerr256 sizes (rank audit, Sec. 6.2); ``audit12_paper_sampling``
                 the same geometries with eight frames 2.5 M apart (the paper's
                 audit sampling).
  * ``recovery`` Kerr a=0.94, i=50 deg at kerr256 sizes, 60 held-out histories.
  * ``stress1024`` a in {0, .94}, i=75 deg, 1024x1024, 256x512 grid, 256 hats,
                 1024 frames.
The synthetic histories follow the paper's phenomenological families (Sec. 9):
Gaussian hot spots on Keplerian orbits, flare envelopes and a log-normal level.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

MASK64 = (1 << 64) - 1


# ---------------------------------------------------------------------------
# SplitMix64 (Steele, Lea & Flood 2014) -> uniforms in [0,1) -> Box-Muller.
# Implemented with numpy uint64 arithmetic (wrap-around is the definition).
# ---------------------------------------------------------------------------
def splitmix64(seed: int, n: int) -> np.ndarray:
    """Return n successive SplitMix64 outputs for the given seed (uint64)."""
    with np.errstate(over="ignore"):
        idx = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & MASK64) + idx * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniforms(seed: int, n: int) -> np.ndarray:
    """n uniforms in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def normals(seed: int, n: int) -> np.ndarray:
    """n standard normals by Box-Muller on SplitMix64 uniforms."""
    m = (n + 1) // 2
    u = uniforms(seed, 2 * m)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([rad * np.cos(2 * np.pi * u2), rad * np.sin(2 * np.pi * u2)])
    out = np.empty(2 * m)
    out[0::2] = z[:m]
    out[1::2] = z[m:]
    return out[:n]


# ---------------------------------------------------------------------------
# Workload descriptions
# ---------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class Geometry:
    spin: float
    incl_deg: float
    nx: int
    fov: float = 12.0  # image spans [-fov, fov] M on both axes

    @property
    def incl(self) -> float:
        return math.radians(self.incl_deg)


@dataclasses.dataclass(frozen=True)
class SourceGrid:
    n_r: int
    n_phi: int
    r_in: float = 3.0
    r_out: float = 11.0

    @property
    def n_nodes(self) -> int:
        return self.n_r * self.n_phi

    def radii(self) -> np.ndarray:
        """Node radii, log-spaced on [r_in, r_out]."""
        return self.r_in * (self.r_out / self.r_in) ** (np.arange(self.n_r) / (self.n_r - 1))

    def azimuths(self) -> np.ndarray:
        return 2.0 * np.pi * np.arange(self.n_phi) / self.n_phi


@dataclasses.dataclass(frozen=True)
class TimeGrid:
    n_frames: int
    cadence: float
    n_hats: int
    t_end: float  # time of the youngest hat centre t_0
    t0: float = 0.0  # first observer time
    hat_step: float = 4.0

    def frame_times(self) -> np.ndarray:
        return self.t0 + self.cadence * np.arange(self.n_frames)

    def hat_times(self) -> np.ndarray:
        """t_k = t_end - hat_step * k, k = 0 (youngest) ... K-1 (oldest)."""
        return self.t_end - self.hat_step * np.arange(self.n_hats)


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    geometry: Geometry
    grid: SourceGrid
    time: TimeGrid
    supersample: int = 1  # sub-rays per axis inside the photon-ring annulus
    annulus_pad: float = 1.5  # annulus = critical-curve radius range +- pad

    @property
    def n_dof(self) -> int:
        return self.grid.n_nodes * self.time.n_hats


def schw32() -> Workload:
    return Workload("schw32", Geometry(0.0, 20.0, 32), SourceGrid(8, 16),
                    TimeGrid(24, 2.0, 12, t_end=0.0))


def kerr256(spin: float = 0.5, incl_deg: float = 50.0, name: str = "kerr256") -> Workload:
    return Workload(name, Geometry(spin, incl_deg, 256), SourceGrid(64, 128),
                    TimeGrid(256, 1.0, 64, t_end=255.0), supersample=2)


def audit12() -> list[Workload]:
    out = []
    for a in (0.0, 0.5, 0.75, 0.94):
        for i in (20.0, 50.0, 75.0):
            out.append(kerr256(a, i, name=f"audit_a{a:g}_i{i:g}"))
    return out


def audit12_paper_sampling() -> list[Workload]:
    """The 12 geometries at kerr256 sizes with the paper's audit sampling
    (Sec. 6.2): eight observer times uniformly spanning 20 M, read as
    t_o = 2.5 f, f = 0..7, the youngest hat at the last frame."""
    out = []
    for a in (0.0, 0.5, 0.75, 0.94):
        for i in (20.0, 50.0, 75.0):
            out.append(Workload(f"audit8_a{a:g}_i{i:g}", Geometry(a, i, 256), SourceGrid(64, 128),
                                TimeGrid(8, 2.5, 64, t_end=17.5), supersample=2))
    return out


def recovery() -> Workload:
    return kerr256(0.94, 50.0, name="recovery")


def stress1024(spin: float = 0.94) -> Workload:
    return Workload(f"stress1024_a{spin:g}", Geometry(spin, 75.0, 1024), SourceGrid(256, 512),
                    TimeGrid(1024, 1.0, 256, t_end=1023.0), supersample=1)


def small_kerr(spin=0.5, incl_deg=50.0, nx=48, n_r=12, n_phi=24, n_frames=40, n_hats=12,
               ss=2) -> Workload:
    """A kerr256-shaped workload scaled down so the oracle finishes in seconds;
    several kernel tiles plus ragged tails on every axis."""
    return Workload(f"small_a{spin:g}_i{incl_deg:g}_{nx}", Geometry(spin, incl_deg, nx),
                    SourceGrid(n_r, n_phi), TimeGrid(n_frames, 1.0, n_hats, t_end=n_frames - 1.0),
                    supersample=ss)


# ---------------------------------------------------------------------------
# Screen sampling
# ---------------------------------------------------------------------------
def critical_curve_radius_range(spin: float, incl_deg: float, n: int = 4001) -> tuple[float, float]:
    """Min and max screen radius of the Kerr critical curve (Bardeen 1973),
    used only to place the supersampled annulus on the screen."""
    if spin == 0.0:
        return math.sqrt(27.0), math.sqrt(27.0)
    a = spin
    i = math.radians(incl_deg)
    rm = 2.0 * (1.0 + math.cos(2.0 / 3.0 * math.acos(-a)))
    rp = 2.0 * (1.0 + math.cos(2.0 / 3.0 * math.acos(a)))
    r = np.linspace(rm, rp, n)
    D = r * r - 2.0 * r + a * a
    lam = a + r / a * (r - 2.0 * D / (r - 1.0))
    eta = r ** 3 / a ** 2 * (4.0 * D / (r - 1.0) ** 2 - r)
    al = -lam / math.sin(i)
    b2 = eta + a * a * math.cos(i) ** 2 - lam ** 2 / math.tan(i) ** 2
    ok = b2 >= 0.0
    rho = np.sqrt(al[ok] ** 2 + b2[ok])
    return float(rho.min()), float(rho.max())


@dataclasses.dataclass
class ScreenSamples:
    alpha: np.ndarray  # float64 [n]
    beta: np.ndarray  # float64 [n]
    pixel: np.ndarray  # int32 [n], pixel index = iy * nx + ix
    n_sub: np.ndarray  # int32 [n], number of sub-rays of that pixel
    d_omega_pixel: float  # pixel solid angle (M^2 units)

    def __len__(self) -> int:
        return int(self.alpha.shape[0])


def screen_samples(w: Workload) -> ScreenSamples:
    """Pixel centres alpha_j = -fov + (j + 1/2) (2 fov / N); pixels whose centre
    lies in the photon-ring annulus are split into ss x ss equal-area sub-rays."""
    g = w.geometry
    N = g.nx
    d = 2.0 * g.fov / N
    c = -g.fov + (np.arange(N) + 0.5) * d
    A, Bm = np.meshgrid(c, c)  # [iy, ix]
    alpha = A.ravel()
    beta = Bm.ravel()
    pix = np.arange(N * N, dtype=np.int32)
    ss = w.supersample
    if ss <= 1:
        return ScreenSamples(alpha, beta, pix, np.ones(N * N, np.int32), d * d)
    lo, hi = critical_curve_radius_range(g.spin, g.incl_deg)
    rho = np.hypot(alpha, beta)
    inside = (rho >= lo - w.annulus_pad) & (rho <= hi + w.annulus_pad)
    counts = np.where(inside, ss * ss, 1).astype(np.int64)
    idx = np.repeat(np.arange(N * N), counts)
    starts = np.repeat(np.cumsum(counts) - counts, counts)
    sub = np.arange(idx.shape[0]) - starts
    off = (np.arange(ss) + 0.5) / ss - 0.5  # sub-pixel centre offsets in pixel units
    ins = inside[idx]
    ox = np.where(ins, off[sub % ss], 0.0)
    oy = np.where(ins, off[sub // ss], 0.0)
    return ScreenSamples(alpha[idx] + ox * d, beta[idx] + oy * d, pix[idx],
                         counts[idx].astype(np.int32), d * d)


def screen_band(s: ScreenSamples, nx: int, row_lo: int, row_hi: int) -> ScreenSamples:
    """The samples of the pixel rows iy in [row_lo, row_hi) (a bounded sample
    of a large screen, for timing the CPU oracle)."""
    iy = s.pixel // nx
    m = (iy >= row_lo) & (iy < row_hi)
    return ScreenSamples(s.alpha[m], s.beta[m], s.pixel[m], s.n_sub[m], s.d_omega_pixel)


# ---------------------------------------------------------------------------
# Source histories (nodal coefficients x[s][k], s = i_r * n_phi + j_phi)
# ---------------------------------------------------------------------------
def hotspot_history(w: Workload, seed: int, n_spots: int = 2, sigma: float = 1.0,
                    flare: bool = False, level: bool = False) -> np.ndarray:
    """Gaussian hot spots (sigma = 1 M in equatorial Cartesian distance) on
    prograde Keplerian orbits Omega = 1/(r^1.5 + a), amplitudes U(0.5, 1.5),
    r0 ~ U(4, 10), phi0 ~ U(0, 2 pi).  Optional flare envelope
    exp(-(t - t0)^2 / (2 * 8^2)) with t0 ~ U(0, 200) from the oldest hat, and a
    log-normal (sigma = 0.3) constant level.  Returns float64 [S, K]."""
    g, tg = w.grid, w.time
    u = uniforms(seed, 5 * n_spots + 1)
    z = normals(seed ^ 0x5DEECE66D, 1)[0]
    rs = g.radii()[:, None] * np.ones((1, g.n_phi))
    ps = np.ones((g.n_r, 1)) * g.azimuths()[None, :]
    X = (rs * np.cos(ps)).ravel()
    Y = (rs * np.sin(ps)).ravel()
    tk = tg.hat_times()
    x = np.zeros((g.n_nodes, tg.n_hats))
    for h in range(n_spots):
        r0 = 4.0 + 6.0 * u[5 * h]
        p0 = 2.0 * np.pi * u[5 * h + 1]
        amp = 0.5 + u[5 * h + 2]
        om = 1.0 / (r0 ** 1.5 + w.geometry.spin)
        ang = p0 + om * tk  # [K]
        hx = r0 * np.cos(ang)
        hy = r0 * np.sin(ang)
        d2 = (X[:, None] - hx[None, :]) ** 2 + (Y[:, None] - hy[None, :]) ** 2
        prof = amp * np.exp(-d2 / (2.0 * sigma * sigma))
        if flare:
            t0 = tk[-1] + 200.0 * u[5 * h + 3]
            prof = prof * np.exp(-((tk - t0) ** 2) / (2.0 * 8.0 ** 2))[None, :]
        x += prof
    if level:
        x += math.exp(0.3 * z)
    return x


def history_batch(w: Workload, seeds, **kw) -> np.ndarray:
    """Stack of histories in the library layout x[s][k][b] (float64)."""
    xs = [hotspot_history(w, int(s), **kw) for s in seeds]
    return np.stack(xs, axis=-1)


def recovery_history(w: Workload, seed: int) -> np.ndarray:
    """Held-out recovery history: 1-4 hot spots (count drawn from the seed)
    with flare envelopes and a log-normal baseline level, float64 [S, K]."""
    n_spots = 1 + min(3, int(4.0 * uniforms(seed ^ 0xA5A5A5A5, 1)[0]))
    return hotspot_history(w, seed, n_spots=n_spots, flare=True, level=True)


def recovery_batch(w: Workload, seeds) -> np.ndarray:
    """Stack of recovery histories, layout x[s][k][b] (float64)."""
    return np.stack([recovery_history(w, int(s)) for s in seeds], axis=-1)


def uniform_batch(w: Workload, seeds) -> np.ndarray:
    """x ~ U(0, 1) per coefficient, layout x[s][k][b] (throughput inputs)."""
    n = w.grid.n_nodes * w.time.n_hats
    return np.stack([uniforms(int(s), n).reshape(w.grid.n_nodes, w.time.n_hats) for s in seeds],
                    axis=-1)


def noise(shape, seed: int) -> np.ndarray:
    """i.i.d. N(0, 1) whitened noise of the given shape."""
    n = int(np.prod(shape))
    return normals(seed, n).reshape(shape)
