"""FP64 CPU oracle for the multi-order retarded-time operator -- TEST
INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It shares no code with the CUDA path
(``paper_2609_05528_b300/csrc``): the hot loops are plain C in
``rtt_oracle.c`` (built here with gcc, loaded by ctypes) and everything else
is numpy in FP64.  Inputs come as plain arrays from the seeded generators in
``paper_2609_05528_b300.inputs``; this module never imports the CUDA binding.

Each function cites the passage of the paper it restates.  Declared readings
where the paper is silent are marked "reading:".

Pins: every function here is checked in ``tests/test_oracle_*.py`` against
something other than itself (closed forms, brute force, invariants).
Parity unpinned: the paper's own 12-cell numbers (other grids, other tracer).
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rtt_oracle.c")
SO = os.path.join(HERE, "liboracle.so")
CAPTURE_CUSHION = 0.01
_LIB = None


def build(force: bool = False) -> str:
    """Compile rtt_oracle.c with gcc (plain C, OpenMP)."""
    if force or not os.path.exists(SO) or os.path.getmtime(SO) < os.path.getmtime(SRC):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", SO, SRC, "-lm"])
    return SO


def set_threads(n: int) -> None:
    """Threads of the C oracle's OpenMP loops (timing only: results do not
    depend on the count)."""
    lib().orc_set_threads(int(n))


def max_threads() -> int:
    """Threads the C oracle's OpenMP loops use."""
    return int(lib().orc_max_threads())


class _Grid(ctypes.Structure):
    _fields_ = [("n_r", ctypes.c_int), ("n_phi", ctypes.c_int), ("r_in", ctypes.c_double),
                ("r_out", ctypes.c_double), ("n_frames", ctypes.c_int), ("t0", ctypes.c_double),
                ("cadence", ctypes.c_double), ("n_hats", ctypes.c_int),
                ("hat_step", ctypes.c_double), ("t_end", ctypes.c_double)]


def lib():
    global _LIB
    if _LIB is None:
        build()
        L = ctypes.CDLL(SO)
        dp = ctypes.POINTER(ctypes.c_double)
        i8 = ctypes.POINTER(ctypes.c_int8)
        i64 = ctypes.POINTER(ctypes.c_int64)
        gp = ctypes.POINTER(_Grid)
        L.orc_trace_kerr.restype = ctypes.c_long
        L.orc_trace_kerr.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_long, dp, dp,
                                     ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, dp, dp,
                                     dp, i8]
        L.orc_trace_schw.restype = ctypes.c_long
        L.orc_trace_schw.argtypes = [ctypes.c_double, ctypes.c_long, dp, dp, ctypes.c_int,
                                     ctypes.c_double, dp, dp, dp, dp, i8]
        for nm in ("orc_carlson_rf",):
            getattr(L, nm).restype = ctypes.c_double
            getattr(L, nm).argtypes = [ctypes.c_double] * 3
        for nm in ("orc_schw_psi", "orc_schw_psi_quad"):
            getattr(L, nm).restype = ctypes.c_double
            getattr(L, nm).argtypes = [ctypes.c_double] * 2
        L.orc_schw_turning_u.restype = ctypes.c_double
        L.orc_schw_turning_u.argtypes = [ctypes.c_double]
        L.orc_kerr_fate.restype = ctypes.c_int
        L.orc_kerr_fate.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, dp]
        L.orc_apply_A.restype = None
        L.orc_apply_A.argtypes = [gp, ctypes.c_long, i64, dp, dp, dp, dp, ctypes.c_double,
                                  ctypes.c_int, ctypes.c_int, dp, dp]
        L.orc_apply_AT.restype = None
        L.orc_apply_AT.argtypes = [gp, ctypes.c_long, i64, dp, dp, dp, dp, ctypes.c_double,
                                   ctypes.c_int, ctypes.c_int, dp, dp]
        L.orc_round_bf16.restype = ctypes.c_double
        L.orc_round_bf16.argtypes = [ctypes.c_double]
        L.orc_set_threads.restype = None
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_max_threads.restype = ctypes.c_int
        L.orc_max_threads.argtypes = []
        L.orc_probe_info.restype = None
        L.orc_probe_info.argtypes = [gp, ctypes.c_long, i64, dp, dp, dp, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_int, dp, dp]
        _LIB = L
    return _LIB


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------
# Geodesics (Sec. 3.1 Eq. 2; Sec. 5; Sec. 6.1)
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Trace:
    r: np.ndarray  # [n, n_orders]
    phi: np.ndarray
    T: np.ndarray  # regularised travel time
    sr: np.ndarray  # +1: photon outgoing at emission (forward in time)
    found: np.ndarray  # bool


def trace(spin: float, incl: float, alpha, beta, n_orders: int = 3, r_esc: float = 11.0,
          method: str = "auto", rtol: float = 1e-13) -> Trace:
    """Per screen ray and order n = 0..n_orders-1: the (n+1)-th equatorial
    crossing (the per-order ray maps of Sec. 3.1 Eq. 2; Kerr and the exact
    Schwarzschild branch of Sec. 5).  method "schw" (a = 0 only): exact orbit integral; "kerr":
    Mino-time Carter integration; "auto": schw at a = 0, kerr otherwise."""
    alpha = _c64(alpha)
    beta = _c64(beta)
    n = alpha.shape[0]
    r = np.empty(n * n_orders)
    phi = np.empty_like(r)
    T = np.empty_like(r)
    sr = np.empty_like(r)
    found = np.zeros(n * n_orders, np.int8)
    if method == "auto":
        method = "schw" if spin == 0.0 else "kerr"
    L = lib()
    if method == "schw":
        if spin != 0.0:
            raise ValueError("exact orbit integral is the Schwarzschild (a = 0) branch")
        L.orc_trace_schw(incl, n, _dp(alpha), _dp(beta), n_orders, r_esc, _dp(r), _dp(phi),
                         _dp(T), _dp(sr), found.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)))
    else:
        bad = L.orc_trace_kerr(spin, incl, n, _dp(alpha), _dp(beta), n_orders, r_esc, rtol,
                               _dp(r), _dp(phi), _dp(T), _dp(sr),
                               found.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)))
        if bad:
            raise RuntimeError(f"{bad} rays hit the integrator step limit")
    sh = (n, n_orders)
    return Trace(r.reshape(sh), phi.reshape(sh), T.reshape(sh), sr.reshape(sh),
                 found.reshape(sh).astype(bool))


def kerr_fate(spin: float, incl: float, alpha: float, beta: float):
    """Integrate one ray until capture (-1) or escape (+1); returns (fate, r_min)
    (the Kerr ray maps of Sec. 5; used to pin the critical curve)."""
    rmin = ctypes.c_double(0.0)
    f = lib().orc_kerr_fate(spin, incl, alpha, beta, ctypes.byref(rmin))
    return int(f), float(rmin.value)


def horizon(spin: float) -> float:
    """Outer horizon r_+ = 1 + sqrt(1 - a^2) (Sec. 5, the r_+ check)."""
    return 1.0 + math.sqrt(1.0 - spin * spin)


def isco(spin: float) -> float:
    """ISCO radius of the equatorial circular orbit that co-rotates with the
    sign of `spin` (Bardeen, Press & Teukolsky 1972): spin >= 0 gives the
    prograde orbit, spin < 0 the orbit against a hole of spin |spin|.  The
    boundary of the circular/plunging emitter branch of Sec. 5."""
    a = abs(spin)
    z1 = 1.0 + (1.0 - a * a) ** (1 / 3) * ((1.0 + a) ** (1 / 3) + (1.0 - a) ** (1 / 3))
    z2 = math.sqrt(3.0 * a * a + z1 * z1)
    root = math.sqrt((3.0 - z1) * (3.0 + z1 + 2.0 * z2))
    return 3.0 + z2 - root if spin >= 0 else 3.0 + z2 + root


def circular_EL(spin: float, r):
    """Specific energy and angular momentum of prograde circular equatorial
    orbits (the emitter's circular branch, Sec. 5; redshift factor of Eq. 2)."""
    a = spin
    den = r ** 0.75 * np.sqrt(r ** 1.5 - 3.0 * np.sqrt(r) + 2.0 * a)
    E = (r ** 1.5 - 2.0 * np.sqrt(r) + a) / den
    L = (r * r - 2.0 * a * np.sqrt(r) + a * a) / den
    return E, L



def redshift(spin: float, r, lam, eta, sr):
    """g = 1 / (-p_mu u^mu) with p_t = -1, p_phi = lam and
    p_r = sr sqrt(R(r)) / Delta (photon at emission, forward in time).
    reading: the emitter is on a prograde Keplerian circular orbit outside the
    ISCO and plunges from the ISCO conserving its E, L inside it (the paper's
    circular/plunging branch, Sec. 5).  g^3 enters the transfer weight for
    specific intensity (Sec. 3.1, Eq. 16)."""
    a = spin
    r = np.asarray(r, dtype=np.float64)
    lam = np.broadcast_to(np.asarray(lam, dtype=np.float64), r.shape)
    eta = np.broadcast_to(np.asarray(eta, dtype=np.float64), r.shape)
    sr = np.broadcast_to(np.asarray(sr, dtype=np.float64), r.shape)
    g = np.empty_like(r)
    rI = isco(a)
    out = r >= rI
    ro = r[out]
    Om = 1.0 / (ro ** 1.5 + a)
    ut = (ro ** 1.5 + a) / (ro ** 0.75 * np.sqrt(ro ** 1.5 - 3.0 * np.sqrt(ro) + 2.0 * a))
    g[out] = 1.0 / (ut * (1.0 - Om * lam[out]))
    inn = ~out
    if np.any(inn):
        ri = r[inn]
        li = lam[inn]
        ei = eta[inn]
        E, L = circular_EL(a, rI)
        D = ri * ri - 2.0 * ri + a * a
        A = E * (ri * ri + a * a) - a * L
        ut = ((ri * ri + a * a) * A / D + a * (L - a * E)) / (ri * ri)
        uph = (a * A / D + (L - a * E)) / (ri * ri)
        Rm = A * A - D * (ri * ri + (L - a * E) ** 2)
        ur = -np.sqrt(np.maximum(Rm, 0.0)) / (ri * ri)
        Rph = (ri * ri + a * a - a * li) ** 2 - D * (ei + (li - a) ** 2)
        pr = sr[inn] * np.sqrt(np.maximum(Rph, 0.0)) / D
        g[inn] = 1.0 / (ut - li * uph - pr * ur)
    return g


# ---------------------------------------------------------------------------
# Ray table (Eq. 2 per ray; Eq. 15-16 weights; delays relative to the direct
# minimum, Sec. 3.1 "relative to the repository convention")
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Table:
    order: np.ndarray  # int8 [E]
    pixel: np.ndarray  # int32 [E]
    r: np.ndarray
    phi: np.ndarray
    delay: np.ndarray
    weight: np.ndarray  # w_e = g^3 sqrt(dOmega_p) / S_p
    throughput: np.ndarray  # tau_e = g^3 dOmega_p / S_p
    row_ptr: np.ndarray  # int64 [R+1], rays sorted by (order, pixel, sample)
    row_order: np.ndarray  # int8 [R]
    row_pixel: np.ndarray  # int32 [R]
    sample: np.ndarray  # int64 [E], index of the screen sample of each ray

    @property
    def n_rays(self) -> int:
        return int(self.r.shape[0])

    @property
    def n_rows(self) -> int:
        return int(self.row_order.shape[0])

    def rows_of_order(self, n: int) -> int:
        return int(np.count_nonzero(self.row_order == n))

    def select(self, orders) -> "Table":
        """Sub-table with the rows of the given orders, in the same order
        (the observation arm of Eq. 3 restricted to those blocks)."""
        orders = tuple(orders)
        keep_rows = np.isin(self.row_order, orders)
        rows = np.nonzero(keep_rows)[0]
        counts = self.row_ptr[rows + 1] - self.row_ptr[rows]
        idx = np.concatenate([np.arange(self.row_ptr[i], self.row_ptr[i + 1]) for i in rows]) \
            if rows.size else np.zeros(0, np.int64)
        rp = np.zeros(rows.size + 1, np.int64)
        rp[1:] = np.cumsum(counts)
        return Table(self.order[idx], self.pixel[idx], self.r[idx], self.phi[idx],
                     self.delay[idx], self.weight[idx], self.throughput[idx], rp,
                     self.row_order[rows], self.row_pixel[rows], self.sample[idx])


def build_table(w, samples, method: str = "auto", n_orders: int = 3) -> Table:
    """Trace the screen samples and assemble the raw FP64 ray table.
    validity chi = 1 iff the crossing exists and r in [r_in, r_out] (Eq. 2);
    w_e = chi g_e^3 sqrt(dOmega_p) / S_p for sub-ray e of pixel p (Eq. 16;
    the pixel datum is the average of its S_p sub-rays);
    Delta_e = T_e - min over direct rays of T (reading: zero at the direct
    minimum, Sec. 3.1)."""
    g_ = w.geometry
    grid = w.grid
    tr = trace(g_.spin, g_.incl, samples.alpha, samples.beta, n_orders=n_orders,
               r_esc=grid.r_out, method=method)
    lam = -samples.alpha * math.sin(g_.incl)
    eta = (samples.alpha ** 2 - g_.spin ** 2) * math.cos(g_.incl) ** 2 + samples.beta ** 2
    ent = []
    for n in range(n_orders):
        ok = tr.found[:, n] & (tr.r[:, n] >= grid.r_in) & (tr.r[:, n] <= grid.r_out)
        idx = np.nonzero(ok)[0]
        ent.append((n, idx))
    if ent[0][1].size == 0:
        raise ValueError("no valid direct rays")
    Tmin = np.min(tr.T[ent[0][1], 0])
    cols = {k: [] for k in ("order", "pixel", "r", "phi", "delay", "g", "nsub", "sample")}
    for n, idx in ent:
        cols["order"].append(np.full(idx.size, n, np.int8))
        cols["pixel"].append(samples.pixel[idx])
        cols["r"].append(tr.r[idx, n])
        cols["phi"].append(tr.phi[idx, n])
        cols["delay"].append(tr.T[idx, n] - Tmin)
        cols["g"].append(redshift(g_.spin, tr.r[idx, n], lam[idx], eta[idx], tr.sr[idx, n]))
        cols["nsub"].append(samples.n_sub[idx])
        cols["sample"].append(idx)
    c = {k: np.concatenate(v) for k, v in cols.items()}
    key = np.lexsort((c["sample"], c["pixel"], c["order"]))
    c = {k: v[key] for k, v in c.items()}
    dOm = samples.d_omega_pixel
    weight = c["g"] ** 3 * math.sqrt(dOm) / c["nsub"]
    thr = c["g"] ** 3 * dOm / c["nsub"]
    rowkey = c["order"].astype(np.int64) * (1 << 32) + c["pixel"].astype(np.int64)
    starts = np.nonzero(np.concatenate([[True], rowkey[1:] != rowkey[:-1]]))[0]
    rp = np.concatenate([starts, [rowkey.size]]).astype(np.int64)
    return Table(c["order"].astype(np.int8), c["pixel"].astype(np.int32), c["r"], c["phi"],
                 c["delay"], weight, thr, rp, c["order"][starts].astype(np.int8),
                 c["pixel"][starts].astype(np.int32), c["sample"].astype(np.int64))


# ---------------------------------------------------------------------------
# Mechanism arms of Sec. 6.4, as ray-table transforms (readings 22, 25, 26).
# Plain Python loops over rays: these are the definitions the product's
# library routine (rtt_arm_table) is checked against.
# ---------------------------------------------------------------------------
def pairing_destroyed(table: Table, keys) -> Table:
    """Pairing-destroyed control (Sec. 6.4; reading: each order keeps its
    multiset of delays, and their association with source point and weight is
    broken).  Within each order n, list the rays of order n by ascending
    index, i_0 < i_1 < ...; sort the same rays by (keys, index) into
    j_0, j_1, ...; ray i_m then takes the delay of ray j_m.  `keys` are the
    random numbers the construction draws (one per ray), passed in."""
    keys = [float(k) for k in keys]
    if len(keys) != table.n_rays:
        raise ValueError("one key per ray")
    order = [int(o) for o in table.order]
    new = np.array(table.delay, dtype=np.float64, copy=True)
    for n in sorted(set(order)):
        by_index = [e for e in range(len(order)) if order[e] == n]
        by_key = sorted(by_index, key=lambda e: (keys[e], e))
        for i_m, j_m in zip(by_index, by_key):
            new[i_m] = table.delay[j_m]
    return dataclasses.replace(table, delay=new)


def quantile_partner(table: Table) -> np.ndarray:
    """The direct ray at the same delay quantile as each ray (reading of
    Sec. 6.4's delay-only / spatial-only arms).  Rank the E_0 direct rays by
    (delay, index); within ring order n, rank its E_n rays the same way; the
    ray of rank k in order n has as partner the direct ray of rank
    floor((k + 1/2) E_0 / E_n).  A direct ray is its own partner."""
    order = [int(o) for o in table.order]
    delay = [float(d) for d in table.delay]
    ranked = {}
    for n in sorted(set(order)):
        ranked[n] = sorted((e for e in range(len(order)) if order[e] == n),
                           key=lambda e: (delay[e], e))
    direct = ranked.get(0, [])
    partner = list(range(len(order)))
    for n, rays in ranked.items():
        if n == 0:
            continue
        for k, e in enumerate(rays):
            partner[e] = direct[((2 * k + 1) * len(direct)) // (2 * len(rays))]
    return np.array(partner, dtype=np.int64)


def delay_only(table: Table) -> Table:
    """Delay-only arm (Sec. 6.4, reading 25): the ring rays keep their
    delays, weights and rows and take the source point (r, phi) of their
    direct quantile partner."""
    p = quantile_partner(table)
    return dataclasses.replace(table, r=np.array([table.r[i] for i in p]),
                               phi=np.array([table.phi[i] for i in p]))


def spatial_only(table: Table) -> Table:
    """Spatial-only arm (Sec. 6.4, reading 26): the ring rays keep their
    source points, weights and rows and take the delay of their direct
    quantile partner."""
    p = quantile_partner(table)
    return dataclasses.replace(table, delay=np.array([table.delay[i] for i in p]))


# ---------------------------------------------------------------------------
# Operator (Eq. 2, 3, 16, 47) and its transpose
# ---------------------------------------------------------------------------
def _grid(w) -> _Grid:
    g, t = w.grid, w.time
    return _Grid(g.n_r, g.n_phi, g.r_in, g.r_out, t.n_frames, t.t0, t.cadence, t.n_hats,
                 t.hat_step, t.t_end)


def s_ref(table: Table) -> float:
    """Eq. 17 with j_ref = 1 evaluated directly (reading: not through the hats):
    the direct response of every frame of a row is sum_e w_e, so
    s_ref^2 = (1/m_0) sum_{direct rows, frames} (sum_e w_e)^2 = mean over
    direct rows of (sum_e w_e)^2."""
    d = table.select((0,))
    sums = np.add.reduceat(d.weight, d.row_ptr[:-1]) if d.n_rows else np.zeros(0)
    return float(np.sqrt(np.mean(sums ** 2)))


def scale(table: Table, snr0: float = 100.0) -> float:
    """Whitening scale SNR_0 / s_ref (Eq. 18: sigma_Omega = s_ref / SNR_0)."""
    return snr0 / s_ref(table)


def round_bf16(v: float) -> float:
    """The oracle's BF16 rounding of a weight: to the nearest float, then to
    the nearest BF16 (ties to even)."""
    return float(lib().orc_round_bf16(float(v)))


def apply_A(w, table: Table, x: np.ndarray, scl: float = 1.0, bf16: bool = False) -> np.ndarray:
    """y[row][f][b] = scl * sum_{e in row} w_e sum_c bil_c sum_k B_k(t_o(f) -
    Delta_e) x[node_c][k][b] (Sec. 3.1 Eq. 2-3; the row action of Eq. 47).
    x: [S, K, B] or [S, K].  bf16: each corner weight scl w_e bil_c rounded
    to BF16 (the GPU tables' BF16-weight option)."""
    squeeze = x.ndim == 2
    xx = _c64(x[..., None] if squeeze else x)
    B = xx.shape[-1]
    y = np.empty((table.n_rows, w.time.n_frames, B))
    lib().orc_apply_A(ctypes.byref(_grid(w)), table.n_rows,
                      np.ascontiguousarray(table.row_ptr, np.int64).ctypes.data_as(
                          ctypes.POINTER(ctypes.c_int64)),
                      _dp(_c64(table.r)), _dp(_c64(table.phi)), _dp(_c64(table.delay)),
                      _dp(_c64(table.weight)), scl, int(bool(bf16)), B, _dp(xx), _dp(y))
    return y[..., 0] if squeeze else y


def apply_AT(w, table: Table, y: np.ndarray, scl: float = 1.0, bf16: bool = False) -> np.ndarray:
    """Exact transpose of apply_A (Sec. 5: explicit adjoint action), with
    the same weights (bf16 as in apply_A)."""
    squeeze = y.ndim == 2
    yy = _c64(y[..., None] if squeeze else y)
    B = yy.shape[-1]
    x = np.empty((w.grid.n_nodes, w.time.n_hats, B))
    lib().orc_apply_AT(ctypes.byref(_grid(w)), table.n_rows,
                       np.ascontiguousarray(table.row_ptr, np.int64).ctypes.data_as(
                           ctypes.POINTER(ctypes.c_int64)),
                       _dp(_c64(table.r)), _dp(_c64(table.phi)), _dp(_c64(table.delay)),
                       _dp(_c64(table.weight)), scl, int(bool(bf16)), B, _dp(yy), _dp(x))
    return x[..., 0] if squeeze else x


def dense_A(w, table: Table, scl: float = 1.0) -> np.ndarray:
    """Explicit per-ray assembly of the dense matrix of Eq. 2-3 (tiny cases
    only; the dense/matrix-free parity check of Sec. 5): rows (row, f),
    columns s * K + k.  Written independently of the C loops
    (numpy, evaluating every hat and the bilinear stencil by its definition)."""
    g, t = w.grid, w.time
    K, T = t.n_hats, t.n_frames
    M = np.zeros((table.n_rows * T, g.n_nodes * K))
    lr = np.log(g.r_in), np.log(g.r_out)
    tk = t.hat_times()
    for row in range(table.n_rows):
        for e in range(table.row_ptr[row], table.row_ptr[row + 1]):
            rho = (np.log(table.r[e]) - lr[0]) / (lr[1] - lr[0]) * (g.n_r - 1)
            i0 = min(max(int(np.floor(rho)), 0), g.n_r - 2)
            fr = rho - i0
            ph = (table.phi[e] / (2 * np.pi) * g.n_phi) % g.n_phi
            j0 = min(int(np.floor(ph)), g.n_phi - 1)
            fp = ph - j0
            j1 = (j0 + 1) % g.n_phi
            stencil = [(i0 * g.n_phi + j0, (1 - fr) * (1 - fp)), ((i0 + 1) * g.n_phi + j0, fr * (1 - fp)),
                       (i0 * g.n_phi + j1, (1 - fr) * fp), ((i0 + 1) * g.n_phi + j1, fr * fp)]
            for f in range(T):
                ts = t.t0 + t.cadence * f - table.delay[e]
                hv = np.maximum(0.0, 1.0 - np.abs(ts - tk) / t.hat_step)
                for node, bw in stencil:
                    M[row * T + f, node * K:(node + 1) * K] += scl * table.weight[e] * bw * hv
    return M


# ---------------------------------------------------------------------------
# Order mixing (Sec. 3.1 Eq. 4): d_L = (L (x) I) d_R, C_L = (L (x) I) C_R (L^T (x) I)
# ---------------------------------------------------------------------------
MIX_UNRESOLVED = 1  # L sums the orders of each pixel (the unresolved image)
MIX_TOTAL_FLUX = 2  # L sums every row (the total-flux readout)


def mixer(table: Table, mode: int, orders=(0, 1, 2)):
    """W = C_L^{-1/2} L, the whitened collapse of Eq. 4 on the rows of `orders`
    (scipy.sparse CSR, output rows x selected rows, selected rows in the
    table's row order).  The data rows are already whitened (C_R = I), so
    C_L = L L^T; its noise is the propagated one, not a new level (Sec. 3.1,
    Sec. 4.2).  Unresolved image: one output row per pixel of the selected
    rows, in ascending pixel order, L = 1 on that pixel's rows.  Total flux:
    one output row, L = 1 on every selected row.  Each selected row feeds one
    output row, so C_L is diagonal (checked) and C_L^{-1/2} is taken entry by
    entry."""
    from scipy import sparse
    sel = np.nonzero(np.isin(table.row_order, tuple(orders)))[0]
    R = sel.size
    if mode == MIX_UNRESOLVED:
        upix, grp = np.unique(table.row_pixel[sel], return_inverse=True)
        L = sparse.csr_matrix((np.ones(R), (grp, np.arange(R))), shape=(upix.size, R))
    elif mode == MIX_TOTAL_FLUX:
        L = sparse.csr_matrix((np.ones(R), (np.zeros(R, np.int64), np.arange(R))), shape=(1, R))
    else:
        raise ValueError(f"mix mode {mode}")
    C = (L @ L.T).tocoo()
    assert np.all(C.row == C.col), "C_L is diagonal: each row feeds one output row"
    cdiag = np.zeros(L.shape[0])
    cdiag[C.row] = C.data
    return sparse.diags(1.0 / np.sqrt(cdiag)) @ L


def mix_rows(table: Table, y: np.ndarray, mode: int, orders=(0, 1, 2)) -> np.ndarray:
    """d_L = W d_R for data y [selected rows][frames][batch] (Eq. 4)."""
    W = mixer(table, mode, orders)
    y2 = y.reshape(y.shape[0], -1)
    return np.asarray(W @ y2).reshape((W.shape[0],) + y.shape[1:])


def mix_rows_T(table: Table, yl: np.ndarray, mode: int, orders=(0, 1, 2)) -> np.ndarray:
    """W^T applied to mixed data yl [output rows][frames][batch] (the adjoint
    of the Eq. 4 collapse)."""
    W = mixer(table, mode, orders)
    y2 = yl.reshape(yl.shape[0], -1)
    return np.asarray(W.T @ y2).reshape((W.shape[1],) + yl.shape[1:])


# ---------------------------------------------------------------------------
# Probes, reach and old-age innovation (Eq. 10-13, 29-30, 35)
# ---------------------------------------------------------------------------
AGES = np.arange(0.0, 253.0, 4.0)  # 0 ... 252 M on a 4 M grid (Sec. 6.2)
PROBE_H = 3.0


def probe_info(w, table: Table, scl: float, ages=AGES, h: float = PROBE_H) -> np.ndarray:
    """I(a) = || C^{-1/2} A q_a ||^2 with q_a evaluated directly at each ray's
    source point (Eq. 10-12, 29)."""
    ages = _c64(ages)
    info = np.empty(ages.shape[0])
    lib().orc_probe_info(ctypes.byref(_grid(w)), table.n_rows,
                         np.ascontiguousarray(table.row_ptr, np.int64).ctypes.data_as(
                             ctypes.POINTER(ctypes.c_int64)),
                         _dp(_c64(table.r)), _dp(_c64(table.delay)), _dp(_c64(table.weight)),
                         scl, h, ages.shape[0], _dp(ages), _dp(info))
    return info


def mix_probe_info(w, table: Table, scl: float, mode: int, orders=(0, 1, 2), ages=AGES,
                   h: float = PROBE_H) -> np.ndarray:
    """I_L(a) = || W C^{-1/2} A q_a ||^2 for a mixed arm (Eq. 4 with Eq. 10-12,
    29): per age, the whitened probe response of every selected (row, frame)
    (the row's rays' w_e q_a at their source points, q_a = 1_[r_in, r_out](r)
    / N_h exp(-(t + a)^2 / (2 h^2)), t = t_o(f) - Delta_e), collapsed by the
    mixer W of `mode`, then its squared norm.  numpy, one age at a time."""
    W = mixer(table, mode, orders)
    sel = np.nonzero(np.isin(table.row_order, tuple(orders)))[0]
    T = w.time.n_frames
    to = w.time.frame_times()
    Nh = probe_norm_const(w, h)
    g = w.grid
    # the selected rows' rays, in row order, and the start of each row among them
    counts = table.row_ptr[sel + 1] - table.row_ptr[sel]
    rays = np.concatenate([np.arange(table.row_ptr[i], table.row_ptr[i + 1]) for i in sel])
    starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
    ind = ((table.r[rays] >= g.r_in) & (table.r[rays] <= g.r_out)).astype(np.float64)
    wt = table.weight[rays] * ind / Nh
    t = to[None, :] - table.delay[rays][:, None]  # [rays, T]
    out = np.empty(len(ages))
    for i, a in enumerate(np.asarray(ages, np.float64)):
        contrib = wt[:, None] * np.exp(-(t + a) ** 2 / (2.0 * h * h))
        Y = np.add.reduceat(contrib, starts, axis=0)  # [selected rows, T]
        out[i] = scl * scl * float(np.sum(np.asarray(W @ Y) ** 2))
    return out


N_LOCAL = 28  # 4 radial x 7 azimuthal localized directions (Eq. 14)


def local_direction_norms(w, h: float = PROBE_H) -> np.ndarray:
    """N_{h,l} of Eq. 14: each direction psi_l(r, phi) = R_i(r) Phi_m(phi)
    (l = 7 i + m; R_i the cubic Bernstein polynomials in the log-radius
    coordinate, Phi in {1, cos phi, sin phi, ..., cos 3 phi, sin 3 phi})
    normalised to unit L2 norm under the equatorial area measure r dr dphi
    times the Gaussian's h sqrt(pi) (the scalar probe's Eq. 11 convention):
    N^2 = int R_i^2 r dr * int Phi_m^2 dphi * h sqrt(pi), by quadrature."""
    from scipy import integrate
    g = w.grid
    L = math.log(g.r_out / g.r_in)
    rad = []
    for i in range(4):
        def f(r, i=i):
            s = math.log(r / g.r_in) / L
            return (math.comb(3, i) * s ** i * (1 - s) ** (3 - i)) ** 2 * r
        rad.append(integrate.quad(f, g.r_in, g.r_out, epsabs=0, epsrel=1e-13, limit=200)[0])
    az = [2 * math.pi] + [math.pi] * 6
    return np.array([math.sqrt(rad[i] * az[m] * h * math.sqrt(math.pi))
                     for i in range(4) for m in range(7)])


def local_direction_values(w, r: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """psi_l at source points (r, phi), unnormalised, [points, 28]: the 28
    spatial directions of the localized probes (Sec. 3.3 Eq. 14)."""
    g = w.grid
    s = np.log(np.asarray(r) / g.r_in) / math.log(g.r_out / g.r_in)
    R = np.stack([math.comb(3, i) * s ** i * (1 - s) ** (3 - i) for i in range(4)], axis=1)
    ph = np.asarray(phi)
    P = [np.ones_like(ph)]
    for m in (1, 2, 3):
        P += [np.cos(m * ph), np.sin(m * ph)]
    P = np.stack(P, axis=1)
    return (R[:, :, None] * P[:, None, :]).reshape(-1, 28)


def local_probe_responses(w, table: Table, a: float, orders=(0, 1, 2), h: float = PROBE_H):
    """Whitened responses (before scale) of the 28 localized probes q_{a,l} of
    Eq. 14 on the rows of `orders`: Y[l, row, f] = sum_{e in row} w_e
    1_[r_in, r_out](r_e) psi_l(r_e, phi_e) / N_{h,l} exp(-(t + a)^2/(2h^2)),
    t = t_o(f) - Delta_e.  numpy."""
    sel = np.nonzero(np.isin(table.row_order, tuple(orders)))[0]
    counts = table.row_ptr[sel + 1] - table.row_ptr[sel]
    rays = np.concatenate([np.arange(table.row_ptr[i], table.row_ptr[i + 1]) for i in sel])
    starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
    g = w.grid
    ind = ((table.r[rays] >= g.r_in) & (table.r[rays] <= g.r_out)).astype(np.float64)
    psi = local_direction_values(w, table.r[rays], table.phi[rays]) / local_direction_norms(w, h)
    coef = (table.weight[rays] * ind)[:, None] * psi  # [rays, 28]
    t = w.time.frame_times()[None, :] - table.delay[rays][:, None]
    gauss = np.exp(-(t + a) ** 2 / (2.0 * h * h))  # [rays, T]
    contrib = coef.T[:, :, None] * gauss[None, :, :]  # [28, rays, T]
    return np.add.reduceat(contrib, starts, axis=1)  # [28, rows, T]


def local_probe_info(w, table: Table, scl: float, orders=(0, 1, 2), ages=AGES,
                     h: float = PROBE_H) -> np.ndarray:
    """I_l(a) = scl^2 || Y_l(a) ||^2 per age and direction, [ages, 28] (the
    diagonal of the age-local Fisher matrix M(a) = P(a)^T P(a), Sec. 3.3)."""
    return np.stack([scl * scl * np.sum(local_probe_responses(w, table, a, orders, h) ** 2,
                                        axis=(1, 2)) for a in np.asarray(ages, np.float64)])


def local_reach(info_local: np.ndarray, rho: float = 1.0, ages=AGES):
    """Localized directional reach: the deepest age at which at least one
    normalised localized direction passes, I_l(a) >= rho^2 (Sec. 3.3, the
    table of reported quantities); None if none passes."""
    ok = np.any(np.asarray(info_local) >= rho * rho, axis=1)
    return float(np.asarray(ages)[np.nonzero(ok)[0][-1]]) if ok.any() else None


def probe_norm_const(w, h: float = PROBE_H) -> float:
    """N_h of Eq. 11."""
    g = w.grid
    return math.sqrt(math.pi * (g.r_out ** 2 - g.r_in ** 2) * h * math.sqrt(math.pi))


def footprints(w, table: Table, orders):
    """Continuous footprints W_n = [t_o,min - Delta_n^max, t_o,max - Delta_n^min]
    (Eq. 13) for the given orders that have rays."""
    t = w.time
    to = t.frame_times()
    out = []
    for n in orders:
        d = table.delay[table.order == n]
        if d.size:
            out.append((to.min() - d.max(), to.max() - d.min()))
    return out


def _covered(intervals, lo, hi) -> bool:
    """Is [lo, hi] inside the union of the closed intervals?"""
    cur = lo
    for a, b in sorted(intervals):
        if a > cur:
            break
        cur = max(cur, b)
        if cur >= hi:
            return True
    return cur >= hi


@dataclasses.dataclass
class Reach:
    passing: np.ndarray  # bool per age
    anchor: float | None  # youngest fully supported age (None: none)
    L_anchor: float
    T_reach: float | None  # oldest passing age (Eq. 30)


def reach(w, table: Table, info: np.ndarray, orders, rho: float = 1.0, ages=AGES,
          h: float = PROBE_H) -> Reach:
    """pass(a) <=> I(a) >= rho^2 (Eq. 30, scale^2 already holds SNR_0^2).
    Anchor: the smallest grid age whose support [-a - 3h, -a + 3h] lies inside
    the arm's footprint union (Sec. 3.3, 3h convention).  L_anchor = a_last -
    anchor for the contiguous passing run starting at the anchor (reading of
    the anchor-connected span, Sec. 4.4); 0 if the anchor fails or is absent."""
    passing = np.asarray(info) >= rho * rho
    fp = footprints(w, table, orders)
    anchor_i = None
    for i, a in enumerate(ages):
        if _covered(fp, -a - 3 * h, -a + 3 * h):
            anchor_i = i
            break
    L = 0.0
    if anchor_i is not None and passing[anchor_i]:
        j = anchor_i
        while j + 1 < len(ages) and passing[j + 1]:
            j += 1
        L = float(ages[j] - ages[anchor_i])
    tre = float(ages[np.nonzero(passing)[0][-1]]) if passing.any() else None
    return Reach(passing, None if anchor_i is None else float(ages[anchor_i]), L, tre)


def a0999(w, table: Table, q: float = 0.999) -> float:
    """Direct order's throughput-weighted age quantile A_{0,q} (Sec. 4.5):
    ages Delta_e - t_o(f) of all direct (ray, frame) samples weighted by tau_e;
    reading: the smallest sample age whose cumulative weight reaches q of the
    total (no interpolation)."""
    d = table.select((0,))
    to = w.time.frame_times()
    ages = (d.delay[:, None] - to[None, :]).ravel()
    wt = np.repeat(d.throughput, to.size)
    o = np.argsort(ages, kind="stable")
    cw = np.cumsum(wt[o])
    k = int(np.searchsorted(cw, q * cw[-1], side="left"))
    return float(ages[o][min(k, ages.size - 1)])


def j_old(info: np.ndarray, A0: float, ages=AGES, da: float = 4.0) -> float:
    """J_old = int_{a > A_0,0.999} log(1 + I(a)) da (Eq. 35); reading: rectangle
    rule on the 4 M age grid with strict '>'."""
    ages = np.asarray(ages)
    m = ages > A0
    return float(da * np.sum(np.log1p(np.asarray(info)[m])))


# ---------------------------------------------------------------------------
# Representation classes (Eq. 8; Sec. 7 compact classes)
# ---------------------------------------------------------------------------
def _radial_bernstein(w):
    """The 4 clamped cubic B-splines in log r with no interior knot (cubic
    Bernstein polynomials) at the radial nodes (Eq. 8)."""
    g = w.grid
    s = (np.log(g.radii()) - np.log(g.r_in)) / (np.log(g.r_out) - np.log(g.r_in))
    return np.stack([math.comb(3, j) * s ** j * (1 - s) ** (3 - j) for j in range(4)], axis=1)


def _azimuthal(w):
    """1, cos m phi, sin m phi for m = 1..3 at the azimuthal nodes (Eq. 8)."""
    ph = w.grid.azimuths()
    cols = [np.ones_like(ph)]
    for m in (1, 2, 3):
        cols += [np.cos(m * ph), np.sin(m * ph)]
    return np.stack(cols, axis=1)  # [n_phi, 7]


# the nested ladder of Sec. 7-8 (Eq. 43): (radial, real azimuthal, temporal)
# dimensions and the temporal family (DCT-II modes or degree-one B-splines)
CLASS_SHAPES = {"S224": (4, 7, 8, "dct"), "L224": (4, 7, 8, "hat"),
                "S448T": (4, 7, 16, "dct"), "S528S": (6, 11, 8, "dct"),
                "S1056ST": (6, 11, 16, "dct"), "L448": (4, 7, 16, "hat"),
                "L1056": (6, 11, 16, "hat")}


def radial_bsplines(s: np.ndarray, n: int) -> np.ndarray:
    """n clamped cubic B-splines on uniform knots in the normalised log radius
    s in [0, 1] (n = 4: no interior knot, the cubic Bernstein basis), [len(s), n];
    by scipy's B-spline evaluation (the radial factor of the ladder, Sec. 8
    Eq. 42-43)."""
    from scipy.interpolate import BSpline
    inner = np.linspace(0.0, 1.0, n - 2)[1:-1]
    t = np.concatenate([[0.0] * 4, inner, [1.0] * 4])
    out = np.empty((np.size(s), n))
    for i in range(n):
        c = np.zeros(n)
        c[i] = 1.0
        out[:, i] = BSpline(t, c, 3, extrapolate=False)(np.clip(s, 0.0, 1.0))
    return np.nan_to_num(out)


def synth_class_ladder(w, kind: str) -> np.ndarray:
    """Q of a class of the ladder as nodal values, rows s * K + k, columns
    (i * NA + l) * NT + m: radial cubic B-splines x {1, cos m phi, sin m phi}
    x NT temporal functions on the hat window [t_{K-1}, t_0] (DCT-II modes for
    S classes, degree-one B-splines on uniform knots for L classes; Sec. 7,
    Eq. 43).  Parents are literal prefixes in the azimuthal and temporal
    indices; the radial refinement moves knots (containment, not prefix)."""
    NR, NA, NT, fam = CLASS_SHAPES[kind]
    g, t = w.grid, w.time
    sr = (np.log(g.radii()) - np.log(g.r_in)) / (np.log(g.r_out) - np.log(g.r_in))
    R = radial_bsplines(sr, NR)
    ph = g.azimuths()
    P = [np.ones_like(ph)]
    for m in range(1, (NA - 1) // 2 + 1):
        P += [np.cos(m * ph), np.sin(m * ph)]
    P = np.stack(P, axis=1)
    tk = t.hat_times()
    ta, tb = tk.min(), tk.max()
    if fam == "dct":
        Tm = np.stack([np.cos(np.pi * m * (tk - ta) / (tb - ta)) for m in range(NT)], axis=1)
    else:
        step = (tb - ta) / (NT - 1)
        Tm = np.stack([np.maximum(0.0, 1.0 - np.abs(tk - (ta + step * m)) / step) for m in range(NT)],
                      axis=1)
    spatial = (R[:, None, :, None] * P[None, :, None, :]).reshape(g.n_nodes, NR, NA)
    Q = spatial[:, None, :, :, None] * Tm[None, :, None, None, :]
    return Q.reshape(g.n_nodes * t.n_hats, NR * NA * NT)


def synth_class(w, kind: str = "S224") -> np.ndarray:
    """Q_d as nodal values, rows s * K + k, columns (i_rad * 7 + l_az) * 8 + m.
    S224: 4 clamped cubic B-splines in log r (no interior knots: the cubic
    Bernstein basis) x {1, cos m phi, sin m phi}_{m<=3} x 8 DCT-II modes
    cos(pi m (t - t_a)/(t_b - t_a)) on the hat window [t_a, t_b] (Eq. 8).
    L224: the temporal factor replaced by 8 degree-one B-splines uniform on
    the same window (Sec. 7).  reading: columns unnormalised."""
    g, t = w.grid, w.time
    R = _radial_bernstein(w)  # [n_r, 4]
    P = _azimuthal(w)  # [n_phi, 7]
    tk = t.hat_times()
    ta, tb = tk.min(), tk.max()
    if kind == "S224":
        Tm = np.stack([np.cos(np.pi * m * (tk - ta) / (tb - ta)) for m in range(8)], axis=1)
    elif kind == "L224":
        step = (tb - ta) / 7.0
        knots = ta + step * np.arange(8)
        Tm = np.stack([np.maximum(0.0, 1.0 - np.abs(tk - kn) / step) for kn in knots], axis=1)
    else:
        raise ValueError(kind)
    spatial = (R[:, None, :, None] * P[None, :, None, :]).reshape(g.n_nodes, 4, 7)  # [S, 4, 7]
    Q = spatial[:, None, :, :, None] * Tm[None, :, None, None, :]  # [S, K, 4, 7, 8]
    return Q.reshape(g.n_nodes * t.n_hats, 224)


# ---------------------------------------------------------------------------
# Gram, spectrum and operational rank (Eq. 21, 31)
# ---------------------------------------------------------------------------
def restricted_response(w, table: Table, Q: np.ndarray, scl: float) -> np.ndarray:
    """P = scl * A Q as an (rows*frames) x d matrix (the restricted operator
    of Eq. 7)."""
    d = Q.shape[1]
    x = Q.reshape(w.grid.n_nodes, w.time.n_hats, d)
    return apply_A(w, table, x, scl).reshape(-1, d)


def gram(P: np.ndarray) -> np.ndarray:
    """G = P^T P (Eq. 21, whitened, sigma_Omega folded into scl)."""
    return P.T @ P


def range_finder(G: np.ndarray, omega: np.ndarray, block: int, rho: float = 1.0):
    """Adaptive randomized range finder for the spectrum of the symmetric
    PSD G (the restricted normal operator of Eq. 21) from the Gaussian draws
    omega [d, block * n_blocks] (Sec. 7-8: the spectra of the large classes).
    Per block: Y = G Omega_i, made orthogonal to the basis V so far (two
    passes), then orthonormal columns by QR with column pivoting, keeping the
    columns whose pivot exceeds 1e-12 of Y's largest column norm before the
    projection; the Ritz values are the eigenvalues of V^T G V.  Stops after
    a block that adds no Ritz value >= rho^2, when V has d columns, or after
    the last block.  Returns (Ritz values descending, basis size, blocks)."""
    import scipy.linalg
    d = G.shape[0]
    n_blocks = omega.shape[1] // block
    V = np.zeros((d, 0))
    ritz = np.zeros(0)
    prev = -1
    used = 0
    for i in range(n_blocks):
        if V.shape[1] >= d:
            break
        Y = G @ omega[:, i * block:(i + 1) * block]
        used += 1
        ymax = float(np.max(np.linalg.norm(Y, axis=0)))
        for _ in range(2):
            if V.shape[1]:
                Y = Y - V @ (V.T @ Y)
        Qy, R, _ = scipy.linalg.qr(Y, mode="economic", pivoting=True)
        piv = np.abs(np.diag(R))
        r = 0
        while r < piv.size and piv[r] > 1e-12 * ymax:
            r += 1
        nk = min(r, d - V.shape[1])
        if nk == 0:
            break
        V = np.hstack([V, Qy[:, :nk]])
        T = V.T @ G @ V
        ritz = np.sort(np.linalg.eigvalsh(0.5 * (T + T.T)))[::-1]
        count = int(np.count_nonzero(ritz >= rho * rho))
        if count == prev:
            break
        prev = count
    return ritz, V.shape[1], used


@dataclasses.dataclass
class Spectrum:
    sigma: np.ndarray  # descending
    rank: int
    margin: float


def operational_rank(G: np.ndarray, rho: float = 1.0) -> Spectrum:
    """sigma_i = sqrt(max(lambda_i(G), 0)); rank = #{sigma_i >= rho} (Eq. 31,
    SNR_0 already in the whitening scale); margin = min_i |sigma_i - rho| / rho."""
    lam = np.linalg.eigvalsh(G)[::-1]
    sig = np.sqrt(np.maximum(lam, 0.0))
    return Spectrum(sig, int(np.count_nonzero(sig >= rho)),
                    float(np.min(np.abs(sig - rho)) / rho) if sig.size else math.inf)


# ---------------------------------------------------------------------------
# Estimators (Sec. 9: TSVD and ridge)
# ---------------------------------------------------------------------------
def ridge_cg(w, table: Table, scl: float, data: np.ndarray, lam: float, tol: float = 1e-12,
             max_iter: int = 5000):
    """Solve (A^T A + lam I) x = A^T d by conjugate gradients in FP64, with
    A = scl * A_table (whitened): the ridge/Tikhonov estimator of Sec. 9.  data: [rows, T, B]; returns (x, iters)."""
    b = apply_AT(w, table, data, scl)

    def op(v):
        return apply_AT(w, table, apply_A(w, table, v, scl), scl) + lam * v

    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rs = np.sum(r * r, axis=(0, 1))
    bn = np.sqrt(np.sum(b * b, axis=(0, 1)))
    it = 0
    while it < max_iter and np.any(np.sqrt(rs) > tol * bn):
        Ap = op(p)
        alpha = rs / np.sum(p * Ap, axis=(0, 1))
        x += alpha * p
        r -= alpha * Ap
        rs_new = np.sum(r * r, axis=(0, 1))
        p = r + (rs_new / rs) * p
        rs = rs_new
        it += 1
    return x, it


def tsvd_in_class(w, table: Table, scl: float, Q: np.ndarray, data: np.ndarray, rank: int | None,
                  rho: float = 1.0):
    """TSVD in the class Q (the truncated-SVD estimator of Sec. 9):
    x = Q V_r L_r^{-1} V_r^T Q^T A^T d with (V, L) the eigenpairs of
    G = Q^T A^T A Q; reading: r = operational rank (Eq. 31)."""
    P = restricted_response(w, table, Q, scl)
    G = gram(P)
    lam, V = np.linalg.eigh(G)
    lam, V = lam[::-1], V[:, ::-1]
    sig = np.sqrt(np.maximum(lam, 0.0))
    r = int(np.count_nonzero(sig >= rho)) if rank is None else rank
    atd = apply_AT(w, table, data, scl)  # [S, K, B]
    c = Q.T @ atd.reshape(-1, atd.shape[-1])  # [d, B]
    coef = V[:, :r] @ ((V[:, :r].T @ c) / lam[:r, None])
    return (Q @ coef).reshape(w.grid.n_nodes, w.time.n_hats, -1), r
