"""Thin ctypes binding of librtt.so (declarations in include/rtt.h).

Argument marshalling only: every step of the operator runs in the library's
CUDA kernels.  torch supplies device memory and streams.  If the library is
missing or cannot be loaded, every entry point raises (there is no CPU
fallback).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librtt.so")
_LIB = None
ABI_VERSION = 2  # RTT_ABI_VERSION of include/rtt.h

i8p = ctypes.POINTER(ctypes.c_int8)
i32p = ctypes.POINTER(ctypes.c_int32)
i64p = ctypes.POINTER(ctypes.c_int64)
dp = ctypes.POINTER(ctypes.c_double)
vp = ctypes.c_void_p


class RttError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: status {status}: {msg}")
        self.status = status


class Geometry(ctypes.Structure):
    _fields_ = [("spin", ctypes.c_double), ("incl_deg", ctypes.c_double)]


class SourceGrid(ctypes.Structure):
    _fields_ = [("n_r", ctypes.c_int32), ("n_phi", ctypes.c_int32), ("r_in", ctypes.c_double),
                ("r_out", ctypes.c_double)]


class TimeGrid(ctypes.Structure):
    _fields_ = [("n_frames", ctypes.c_int32), ("t0", ctypes.c_double), ("cadence", ctypes.c_double),
                ("n_hats", ctypes.c_int32), ("hat_step", ctypes.c_double),
                ("t_end", ctypes.c_double)]


class RayTable(ctypes.Structure):
    _fields_ = [("n_rays", ctypes.c_int64), ("order", i8p), ("pixel", i32p), ("r", dp),
                ("phi", dp), ("delay", dp), ("weight", dp), ("throughput", dp)]


class RayBuffer(ctypes.Structure):
    _fields_ = [("capacity", ctypes.c_int64), ("order", i8p), ("pixel", i32p), ("r", dp),
                ("phi", dp), ("delay", dp), ("weight", dp), ("throughput", dp)]


class Options(ctypes.Structure):
    _fields_ = [("snr0", ctypes.c_double), ("rho", ctypes.c_double)]


class OpInfo(ctypes.Structure):
    _fields_ = [("n_rays", ctypes.c_int64), ("n_rows", ctypes.c_int64),
                ("rows_per_order", ctypes.c_int64 * 3), ("n_nodes", ctypes.c_int64),
                ("n_hats", ctypes.c_int32), ("n_frames", ctypes.c_int32),
                ("s_ref", ctypes.c_double), ("scale", ctypes.c_double),
                ("delay_min", ctypes.c_double * 3), ("delay_max", ctypes.c_double * 3),
                ("total_rows", ctypes.c_int64), ("total_rows_per_order", ctypes.c_int64 * 3),
                ("shard_row_begin", ctypes.c_int64),
                ("shard_index", ctypes.c_int32), ("shard_count", ctypes.c_int32),
                ("weight_precision", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Shard(ctypes.Structure):
    _fields_ = [("index", ctypes.c_int32), ("count", ctypes.c_int32)]


class ReachResult(ctypes.Structure):
    _fields_ = [("anchor_index", ctypes.c_int32), ("anchor_age", ctypes.c_double),
                ("L_anchor", ctypes.c_double), ("T_reach", ctypes.c_double),
                ("A0q", ctypes.c_double), ("J_old", ctypes.c_double)]


class AuditRecord(ctypes.Structure):
    _fields_ = [("arm_mask", ctypes.c_int32), ("rank", ctypes.c_int32), ("margin", ctypes.c_double),
                ("sigma_max", ctypes.c_double), ("sigma_min_pos", ctypes.c_double),
                ("s_ref", ctypes.c_double), ("jacobi_sweeps", ctypes.c_int32),
                ("reach", ReachResult), ("seconds", ctypes.c_double),
                ("seconds_probe", ctypes.c_double), ("seconds_gram", ctypes.c_double),
                ("seconds_eig", ctypes.c_double)]


class Screen(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("alpha", dp), ("beta", dp), ("pixel", i32p),
                ("n_sub", i32p), ("d_omega_pixel", ctypes.c_double)]


class TuneResult(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int32), ("fwd_kernel", ctypes.c_int32),
                ("fwd_bc", ctypes.c_int32), ("fwd_frames_per_lane", ctypes.c_int32),
                ("fwd_staging", ctypes.c_int32), ("adj_kernel", ctypes.c_int32),
                ("fwd_ms", ctypes.c_float), ("adj_ms", ctypes.c_float),
                ("fwd_ms_rule", ctypes.c_float), ("adj_ms_rule", ctypes.c_float),
                ("candidates", ctypes.c_int32), ("fwd_order", ctypes.c_int32),
                ("fwd_cols", ctypes.c_int32), ("adj_cols", ctypes.c_int32)]


class Variant(ctypes.Structure):
    _fields_ = [("fwd_kernel", ctypes.c_int32), ("fwd_bc", ctypes.c_int32),
                ("fwd_half", ctypes.c_int32), ("adj_kernel", ctypes.c_int32),
                ("fwd_staging", ctypes.c_int32), ("fwd_order", ctypes.c_int32),
                ("fwd_cols", ctypes.c_int32), ("adj_cols", ctypes.c_int32)]


# name -> (restype, argtypes)
_SIGS = {
    "rtt_error_string": (ctypes.c_char_p, [ctypes.c_int]),
    "rtt_last_error": (ctypes.c_char_p, []),
    "rtt_abi_version": (ctypes.c_int, []),
    "rtt_trace_rays": (ctypes.c_int, [ctypes.POINTER(Geometry), ctypes.POINTER(SourceGrid),
                                      ctypes.POINTER(Screen), ctypes.POINTER(RayBuffer), i64p,
                                      vp]),
    "rtt_build_operator": (ctypes.c_int, [ctypes.POINTER(Geometry), ctypes.POINTER(SourceGrid),
                                          ctypes.POINTER(TimeGrid), ctypes.POINTER(RayTable),
                                          ctypes.POINTER(Options), vp, ctypes.POINTER(vp)]),
    "rtt_build_operator_shard": (ctypes.c_int, [ctypes.POINTER(Geometry), ctypes.POINTER(SourceGrid),
                                                ctypes.POINTER(TimeGrid), ctypes.POINTER(RayTable),
                                                ctypes.POINTER(Options), ctypes.POINTER(Shard), vp,
                                                ctypes.POINTER(vp)]),
    "rtt_set_weight_precision": (ctypes.c_int, [vp, ctypes.c_int, vp]),
    "rtt_shard_rows": (ctypes.c_int, [ctypes.c_int64, ctypes.POINTER(Shard),
                                      ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "rtt_op_query": (ctypes.c_int, [vp, ctypes.POINTER(OpInfo)]),
    "rtt_arm_rows": (ctypes.c_int, [vp, ctypes.c_int, i64p]),
    "rtt_op_status": (ctypes.c_int, [vp, i32p, ctypes.c_int, vp]),
    "rtt_apply_A": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, ctypes.c_int, vp]),
    "rtt_apply_AT": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, ctypes.c_int, vp]),
    "rtt_apply_A_f64": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, ctypes.c_int, vp]),
    "rtt_apply_A_AT": (ctypes.c_int, [vp, vp, vp, vp, vp, ctypes.c_int, ctypes.c_int, vp]),
    "rtt_apply_AT_f64": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, ctypes.c_int, vp]),
    "rtt_probe_info": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_double, dp, vp]),
    "rtt_probe_info_noalloc": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, vp,
                                              ctypes.c_double, vp, vp]),
    "rtt_direct_age_quantile": (ctypes.c_int, [vp, ctypes.c_double, dp, vp]),
    "rtt_reach": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_double, ctypes.POINTER(ReachResult),
                                 ctypes.POINTER(ctypes.c_uint8)]),
    "rtt_gram": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_int, vp, vp]),
    "rtt_eig_sym": (ctypes.c_int, [ctypes.c_int, vp, dp, vp, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_int), vp]),
    "rtt_eig_sym_batched": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, vp, dp, vp, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_int), vp]),
    "rtt_eigvals_sym_batched": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, vp, dp, vp]),
    "rtt_solve_ridge": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_int, dp, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_double, ctypes.c_int, vp,
                                       ctypes.POINTER(ctypes.c_int), dp, vp]),
    "rtt_solve_tsvd": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_int, vp, dp, ctypes.c_int, vp,
                                      ctypes.c_int, vp, vp]),
    "rtt_gram_normal": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_int, vp, vp]),
    "rtt_gram_normal_mix": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int, vp, vp]),
    "rtt_probe_info_mix": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp,
                                          ctypes.c_double, dp, vp]),
    "rtt_class_dim": (ctypes.c_int, [ctypes.c_int]),
    "rtt_probe_info_local": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_double, dp,
                                            vp]),
    "rtt_mix_rows_count": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_int64)]),
    "rtt_mix_rows": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, vp, vp, ctypes.c_int, vp]),
    "rtt_mix_rows_T": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, vp, vp, ctypes.c_int, vp]),
    "rtt_mix_rows_f64": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, vp, vp, ctypes.c_int, vp]),
    "rtt_mix_rows_T_f64": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, vp, vp, ctypes.c_int, vp]),
    "rtt_gram_class": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, vp, vp]),
    "rtt_synth_class": (ctypes.c_int, [vp, ctypes.c_int, vp, vp]),
    "rtt_rank_audit": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp),
                                      ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                      ctypes.c_int, dp, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int, ctypes.POINTER(AuditRecord), dp, vp]),
    "rtt_range_finder": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        dp, ctypes.c_double, dp, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), vp]),
    "rtt_audit_plan_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                             ctypes.c_int, ctypes.c_int, dp, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_int, vp, ctypes.POINTER(vp)]),
    "rtt_audit_plan_run": (ctypes.c_int, [vp, vp]),
    "rtt_audit_plan_results": (ctypes.c_int, [vp, ctypes.POINTER(AuditRecord), dp, vp]),
    "rtt_audit_plan_destroy": (ctypes.c_int, [vp]),
    "rtt_autotune": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, vp,
                                    ctypes.POINTER(TuneResult)]),
    "rtt_set_variant": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(Variant)]),
    "rtt_get_variant": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(Variant)]),
    "rtt_arm_table": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(RayTable), dp, dp, dp, dp]),
    "rtt_operational_rank": (ctypes.c_int, [ctypes.c_int, dp, ctypes.c_double,
                                            ctypes.POINTER(ctypes.c_int), dp, dp]),
    "rtt_gemm_tn_f64": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int64,
                                       vp, ctypes.c_int64, vp, ctypes.c_int64, vp]),
    "rtt_destroy": (None, [vp]),
}


def lib():
    """Load librtt.so (raises if it is missing: there is no fallback)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2609_05528_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        # the structs below mirror rtt.h of this ABI version; a library of
        # another version would write past them
        if L.rtt_abi_version() != ABI_VERSION:
            raise RuntimeError(f"{LIB_PATH} has ABI version {L.rtt_abi_version()}, the binding "
                               f"expects {ABI_VERSION}: rebuild it")
        _LIB = L
    return _LIB


def exported_symbols():
    return list(_SIGS)


def check(status: int, where: str):
    if status != 0:
        L = lib()
        raise RttError(status, where, L.rtt_last_error().decode())


def _ptr(a: np.ndarray, typ):
    return a.ctypes.data_as(typ)


_FLOATS = ("float32", "float64")


def _on_gpu(t) -> bool:
    return bool(t.is_cuda)


def _want(t, name: str, shape, dtypes=_FLOATS, like=None):
    """Check a tensor argument before its pointer reaches the library, which
    reads and writes exactly the sizes its header states: a torch tensor of
    one of `dtypes` (names), of `shape` (None matches any extent), contiguous,
    on the GPU, and on the same device and of the same dtype as `like` when
    given.  Raises ValueError; returns t."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name}: expected a torch tensor, got {type(t).__name__}")
    dt = str(t.dtype).replace("torch.", "")
    if dt not in dtypes:
        raise ValueError(f"{name}: dtype {dt}, expected {' or '.join(dtypes)}")
    if like is not None and t.dtype != like.dtype:
        raise ValueError(f"{name}: dtype {dt} differs from the input's {like.dtype}")
    if t.dim() != len(shape) or any(w is not None and int(n) != int(w)
                                    for n, w in zip(t.shape, shape)):
        want = ", ".join("*" if w is None else str(int(w)) for w in shape)
        raise ValueError(f"{name}: shape {list(t.shape)}, expected [{want}]")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if not _on_gpu(t):
        raise ValueError(f"{name}: must be a CUDA tensor")
    if like is not None and t.device != like.device:
        raise ValueError(f"{name}: on {t.device}, the input is on {like.device}")
    return t


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def rtt_trace_rays(spin, incl_deg, grid, samples, stream=None):
    """Trace screen samples on the GPU; returns the raw FP64 table as numpy arrays
    (dict with order, pixel, r, phi, delay, weight, throughput)."""
    L = lib()
    n = len(samples)
    al = np.ascontiguousarray(samples.alpha, np.float64)
    be = np.ascontiguousarray(samples.beta, np.float64)
    px = np.ascontiguousarray(samples.pixel, np.int32)
    ns = np.ascontiguousarray(samples.n_sub, np.int32)
    scr = Screen(n, _ptr(al, dp), _ptr(be, dp), _ptr(px, i32p), _ptr(ns, i32p),
                 float(samples.d_omega_pixel))
    cap = 3 * n
    out = {"order": np.empty(cap, np.int8), "pixel": np.empty(cap, np.int32)}
    for k in ("r", "phi", "delay", "weight", "throughput"):
        out[k] = np.empty(cap, np.float64)
    buf = RayBuffer(cap, _ptr(out["order"], i8p), _ptr(out["pixel"], i32p), _ptr(out["r"], dp),
                    _ptr(out["phi"], dp), _ptr(out["delay"], dp), _ptr(out["weight"], dp),
                    _ptr(out["throughput"], dp))
    n_out = ctypes.c_int64(0)
    g = Geometry(float(spin), float(incl_deg))
    sg = SourceGrid(grid.n_r, grid.n_phi, grid.r_in, grid.r_out)
    check(L.rtt_trace_rays(ctypes.byref(g), ctypes.byref(sg), ctypes.byref(scr), ctypes.byref(buf),
                           ctypes.byref(n_out), _stream(stream)), "rtt_trace_rays")
    m = n_out.value
    return {k: v[:m].copy() for k, v in out.items()}


class Operator:
    """Owns an rtt_op handle (rtt_build_operator / rtt_destroy)."""

    def __init__(self, workload, table, snr0: float = 100.0, rho: float = 1.0, stream=None,
                 shard=None):
        """shard = (index, count): rtt_build_operator_shard, the block of rows
        `index` of `count` with the whole table's whitening (the whole table is
        passed on every rank)."""
        L = lib()
        self.workload = workload
        g, t = workload.grid, workload.time
        arr = {
            "order": np.ascontiguousarray(table["order"], np.int8),
            "pixel": np.ascontiguousarray(table["pixel"], np.int32),
        }
        for k in ("r", "phi", "delay", "weight", "throughput"):
            arr[k] = np.ascontiguousarray(table[k], np.float64)
        self._keep = arr
        rt = RayTable(arr["r"].shape[0], _ptr(arr["order"], i8p), _ptr(arr["pixel"], i32p),
                      _ptr(arr["r"], dp), _ptr(arr["phi"], dp), _ptr(arr["delay"], dp),
                      _ptr(arr["weight"], dp), _ptr(arr["throughput"], dp))
        geo = Geometry(workload.geometry.spin, workload.geometry.incl_deg)
        sg = SourceGrid(g.n_r, g.n_phi, g.r_in, g.r_out)
        tg = TimeGrid(t.n_frames, t.t0, t.cadence, t.n_hats, t.hat_step, t.t_end)
        opt = Options(snr0, rho)
        h = ctypes.c_void_p()
        sh = Shard(int(shard[0]), int(shard[1])) if shard is not None else None
        check(L.rtt_build_operator_shard(ctypes.byref(geo), ctypes.byref(sg), ctypes.byref(tg),
                                         ctypes.byref(rt), ctypes.byref(opt),
                                         ctypes.byref(sh) if sh is not None else None,
                                         _stream(stream), ctypes.byref(h)),
              "rtt_build_operator_shard")
        self.handle = h
        self._keep = None
        info = OpInfo()
        check(L.rtt_op_query(self.handle, ctypes.byref(info)), "rtt_op_query")
        self.info = info
        self.n_nodes = int(info.n_nodes)
        self.n_hats = int(info.n_hats)
        self.n_frames = int(info.n_frames)
        self.scale = float(info.scale)
        self.s_ref = float(info.s_ref)
        self.shard_index, self.shard_count = int(info.shard_index), int(info.shard_count)
        self.shard_row_begin, self.total_rows = int(info.shard_row_begin), int(info.total_rows)
        self.total_rows_per_order = tuple(int(v) for v in info.total_rows_per_order)

    def set_weight_precision(self, precision: int, stream=None):
        """rtt_set_weight_precision: WEIGHTS_FP32 or WEIGHTS_BF16 corner
        weights for the FP32 applies."""
        check(lib().rtt_set_weight_precision(self.handle, int(precision), _stream(stream)),
              "rtt_set_weight_precision")
        info = OpInfo()
        check(lib().rtt_op_query(self.handle, ctypes.byref(info)), "rtt_op_query")
        self.info = info

    def arm_rows(self, arm_mask: int = 7) -> int:
        n = ctypes.c_int64(0)
        check(lib().rtt_arm_rows(self.handle, arm_mask, ctypes.byref(n)), "rtt_arm_rows")
        return int(n.value)

    def autotune(self, batch: int, arm_mask: int = 7, stream=None) -> dict:
        """rtt_autotune: time the FP32 kernel variants for `batch` columns and
        keep the fastest for later applies of that batch size."""
        r = TuneResult()
        check(lib().rtt_autotune(self.handle, int(batch), int(arm_mask), _stream(stream),
                                 ctypes.byref(r)), "rtt_autotune")
        return {k: getattr(r, k) for k, _ in TuneResult._fields_}

    def set_variant(self, batch: int, fwd_kernel=None, fwd_bc=None, fwd_half=0, adj_kernel=None,
                    fwd_staging=0, fwd_order=0, fwd_cols=0, adj_cols=0):
        """rtt_set_variant; all None resets `batch` to the default rule."""
        if fwd_kernel is None and fwd_bc is None and adj_kernel is None:
            check(lib().rtt_set_variant(self.handle, int(batch), None), "rtt_set_variant")
            return
        v = Variant(int(fwd_kernel), int(fwd_bc), int(fwd_half), int(adj_kernel), int(fwd_staging),
                    int(fwd_order), int(fwd_cols), int(adj_cols))
        check(lib().rtt_set_variant(self.handle, int(batch), ctypes.byref(v)), "rtt_set_variant")

    def get_variant(self, batch: int) -> dict:
        v = Variant()
        check(lib().rtt_get_variant(self.handle, int(batch), ctypes.byref(v)), "rtt_get_variant")
        return {k: getattr(v, k) for k, _ in Variant._fields_}

    def status(self, clear: bool = False, stream=None) -> int:
        """rtt_op_status: device status word (0 = no bounded wait timed out)."""
        v = ctypes.c_int32(0)
        check(lib().rtt_op_status(self.handle, ctypes.byref(v), int(clear), _stream(stream)),
              "rtt_op_status")
        return int(v.value)

    def close(self):
        if getattr(self, "handle", None):
            lib().rtt_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- applies (torch tensors on the current CUDA device) --
    def _launch(self, name, src, dst, batch, arm, stream):
        fn = getattr(lib(), name)
        check(fn(self.handle, ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()),
                 int(batch), int(arm), _stream(stream)), name)

    def apply_A(self, x, y=None, arm_mask: int = 7, stream=None):
        """y = scale * A x; x: [n_nodes, n_hats, B] (float32 or float64, CUDA)."""
        import torch
        _want(x, "x", (self.n_nodes, self.n_hats, None))
        B = x.shape[2]
        R = self.arm_rows(arm_mask)
        if y is None:
            y = torch.empty((R, self.n_frames, B), dtype=x.dtype, device=x.device)
        else:
            _want(y, "y", (R, self.n_frames, B), like=x)
        name = "rtt_apply_A" if x.dtype == torch.float32 else "rtt_apply_A_f64"
        self._launch(name, x, y, B, arm_mask, stream)
        return y

    def apply_A_AT(self, x, d=None, y=None, g=None, arm_mask: int = 7, stream=None):
        """rtt_apply_A_AT: (y, g) = (scale A x, scale A^T (y - d)), FP32, one call."""
        import torch
        _want(x, "x", (self.n_nodes, self.n_hats, None), ("float32",))
        B = x.shape[2]
        R = self.arm_rows(arm_mask)
        if y is None:
            y = torch.empty((R, self.n_frames, B), dtype=x.dtype, device=x.device)
        else:
            _want(y, "y", (R, self.n_frames, B), like=x)
        if g is None:
            g = torch.empty_like(x)
        else:
            _want(g, "g", tuple(x.shape), like=x)
        if d is not None:
            _want(d, "d", (R, self.n_frames, B), like=x)
        dp_ = ctypes.c_void_p(d.data_ptr()) if d is not None else None
        check(lib().rtt_apply_A_AT(self.handle, ctypes.c_void_p(x.data_ptr()), dp_,
                                   ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(g.data_ptr()),
                                   int(B), int(arm_mask), _stream(stream)), "rtt_apply_A_AT")
        return y, g

    def apply_AT(self, y, x=None, arm_mask: int = 7, stream=None):
        """x = scale * A^T y; y: [arm_rows, n_frames, B]."""
        import torch
        _want(y, "y", (self.arm_rows(arm_mask), self.n_frames, None))
        B = y.shape[2]
        if x is None:
            x = torch.empty((self.n_nodes, self.n_hats, B), dtype=y.dtype, device=y.device)
        else:
            _want(x, "x", (self.n_nodes, self.n_hats, B), like=y)
        name = "rtt_apply_AT" if y.dtype == torch.float32 else "rtt_apply_AT_f64"
        self._launch(name, y, x, B, arm_mask, stream)
        return x

    def mix_rows_count(self, mode: int, arm_mask: int = 7) -> int:
        """rtt_mix_rows_count: rows of the mixed arm (Eq. 4)."""
        n = ctypes.c_int64()
        check(lib().rtt_mix_rows_count(self.handle, arm_mask, mode, ctypes.byref(n)),
              "rtt_mix_rows_count")
        return int(n.value)

    def mix_rows(self, y, mode: int, arm_mask: int = 7, out=None, stream=None):
        """rtt_mix_rows(_f64): the whitened collapse of the arm's data y
        [arm_rows, n_frames, B] into [mixed rows, n_frames, B] (Eq. 4)."""
        import torch
        _want(y, "y", (self.arm_rows(arm_mask), self.n_frames, None))
        B = y.shape[2]
        n_out = self.mix_rows_count(mode, arm_mask)
        if out is None:
            out = torch.empty((n_out, self.n_frames, B), dtype=y.dtype, device=y.device)
        else:
            _want(out, "out", (n_out, self.n_frames, B), like=y)
        name = "rtt_mix_rows" if y.dtype == torch.float32 else "rtt_mix_rows_f64"
        check(getattr(lib(), name)(self.handle, arm_mask, mode, ctypes.c_void_p(y.data_ptr()),
                                   ctypes.c_void_p(out.data_ptr()), B, _stream(stream)), name)
        return out

    def mix_rows_T(self, yl, mode: int, arm_mask: int = 7, out=None, stream=None):
        """rtt_mix_rows_T(_f64): the adjoint of the collapse, [mixed rows,
        n_frames, B] -> [arm_rows, n_frames, B]."""
        import torch
        _want(yl, "yl", (self.mix_rows_count(mode, arm_mask), self.n_frames, None))
        B = yl.shape[2]
        R = self.arm_rows(arm_mask)
        if out is None:
            out = torch.empty((R, self.n_frames, B), dtype=yl.dtype, device=yl.device)
        else:
            _want(out, "out", (R, self.n_frames, B), like=yl)
        name = "rtt_mix_rows_T" if yl.dtype == torch.float32 else "rtt_mix_rows_T_f64"
        check(getattr(lib(), name)(self.handle, arm_mask, mode, ctypes.c_void_p(yl.data_ptr()),
                                   ctypes.c_void_p(out.data_ptr()), B, _stream(stream)), name)
        return out


AGES = np.arange(0.0, 253.0, 4.0)


def probe_info(op: "Operator", arm_mask: int = 7, ages=AGES, h: float = 3.0, stream=None):
    ages = np.ascontiguousarray(ages, np.float64)
    info = np.empty(ages.shape[0])
    check(lib().rtt_probe_info(op.handle, arm_mask, ages.shape[0], _ptr(ages, dp), h,
                               _ptr(info, dp), _stream(stream)), "rtt_probe_info")
    return info


def direct_age_quantile(op: "Operator", q: float = 0.999, stream=None) -> float:
    out = ctypes.c_double(0.0)
    check(lib().rtt_direct_age_quantile(op.handle, q, ctypes.byref(out), _stream(stream)),
          "rtt_direct_age_quantile")
    return out.value


def reach(op: "Operator", info, arm_mask: int = 7, ages=AGES, h: float = 3.0, a0q: float = 0.0,
          age_step: float = 4.0):
    ages = np.ascontiguousarray(ages, np.float64)
    info = np.ascontiguousarray(info, np.float64)
    res = ReachResult()
    passed = np.zeros(ages.shape[0], np.uint8)
    check(lib().rtt_reach(op.handle, arm_mask, ages.shape[0], _ptr(ages, dp), _ptr(info, dp), h,
                          a0q, age_step, ctypes.byref(res),
                          passed.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))), "rtt_reach")
    return res, passed.astype(bool)


WEIGHTS_FP32 = 0  # rtt.h RTT_WEIGHTS_FP32
WEIGHTS_BF16 = 1  # rtt.h RTT_WEIGHTS_BF16
MIX_UNRESOLVED = 1  # rtt.h RTT_MIX_UNRESOLVED
MIX_TOTAL_FLUX = 2  # rtt.h RTT_MIX_TOTAL_FLUX
GRAM_DATA = 0
GRAM_NORMAL = 1
GRAM_CLASS_S224 = 2
GRAM_CLASS_L224 = 3
CLASS_S224 = 0
CLASS_L224 = 1
CLASS_S448T = 2
CLASS_S528S = 3
CLASS_S1056ST = 4
CLASS_L448 = 5
CLASS_L1056 = 6


def class_dim(kind: int) -> int:
    """rtt_class_dim: the dimension of class `kind` (0 if unknown)."""
    return int(lib().rtt_class_dim(int(kind)))


def synth_class(op: "Operator", kind: int = CLASS_S224, stream=None):
    """Class matrix Q (CUDA float64 [n_nodes, n_hats, d]) synthesised on the GPU."""
    import torch
    d = class_dim(kind)
    if d == 0:
        raise RttError(-1, "synth_class", f"unknown class kind {kind}")
    Q = torch.empty((op.n_nodes, op.n_hats, d), dtype=torch.float64, device="cuda")
    check(lib().rtt_synth_class(op.handle, kind, ctypes.c_void_p(Q.data_ptr()), _stream(stream)),
          "rtt_synth_class")
    return Q


def gram(op: "Operator", Q, arm_mask: int = 7, mode: int = GRAM_DATA, stream=None):
    """G = P^T P, P = scale A_arm Q; Q: CUDA float64 [n_nodes, n_hats, d].
    mode GRAM_DATA: over data samples; GRAM_NORMAL: Q^T A^T A Q."""
    import torch
    _want(Q, "Q", (op.n_nodes, op.n_hats, None), ("float64",))
    d = Q.shape[2]
    G = torch.empty((d, d), dtype=torch.float64, device=Q.device)
    name = "rtt_gram" if mode == GRAM_DATA else "rtt_gram_normal"
    check(getattr(lib(), name)(op.handle, arm_mask, ctypes.c_void_p(Q.data_ptr()), d,
                               ctypes.c_void_p(G.data_ptr()), _stream(stream)), name)
    return G


def gram_class(op: "Operator", kind: int = CLASS_S224, arm_mask: int = 7, stream=None):
    """rtt_gram_class: the restricted Gram of a separable class (224 x 224 FP64)."""
    import torch
    G = torch.empty((224, 224), dtype=torch.float64, device="cuda")
    check(lib().rtt_gram_class(op.handle, arm_mask, int(kind), ctypes.c_void_p(G.data_ptr()),
                               _stream(stream)), "rtt_gram_class")
    return G


def eig_sym(G, max_sweeps: int = 60, stream=None):
    """Eigenvalues (descending) and eigenvectors of a symmetric CUDA FP64 matrix."""
    import torch
    n = G.shape[0] if G.dim() == 2 else -1
    A = _want(G.clone().contiguous(), "G", (n, n), ("float64",))
    V = torch.empty_like(A)
    ev = np.empty(n)
    sw = ctypes.c_int(0)
    check(lib().rtt_eig_sym(n, ctypes.c_void_p(A.data_ptr()), _ptr(ev, dp),
                            ctypes.c_void_p(V.data_ptr()), max_sweeps, ctypes.byref(sw),
                            _stream(stream)), "rtt_eig_sym")
    order = np.argsort(-ev, kind="stable")
    return ev[order], V[:, torch.from_numpy(order).to(V.device)], sw.value


def eigvals_sym_batched(G, stream=None):
    """Eigenvalues (ascending per matrix) of CUDA FP64 symmetric matrices
    [batch, n, n] by tridiagonal reduction and bisection (input is copied)."""
    b, n = (G.shape[0], G.shape[1]) if G.dim() == 3 else (-1, -1)
    A = _want(G.clone().contiguous(), "G", (b, n, n), ("float64",))
    ev = np.empty(b * n)
    check(lib().rtt_eigvals_sym_batched(n, b, ctypes.c_void_p(A.data_ptr()), _ptr(ev, dp),
                                        _stream(stream)), "rtt_eigvals_sym_batched")
    return ev.reshape(b, n)


def gemm_tn(A, B, stream=None):
    """rtt_gemm_tn_f64: C = A^T B (CUDA float64 2D tensors, k x m and k x n) in
    FP64 accuracy on the tensor cores."""
    import torch
    k, m = (A.shape[0], A.shape[1]) if A.dim() == 2 else (-1, -1)
    _want(A, "A", (k, m), ("float64",))
    _want(B, "B", (k, None), ("float64",), like=A)
    n = B.shape[1]
    C = torch.empty((m, n), dtype=torch.float64, device=A.device)
    check(lib().rtt_gemm_tn_f64(k, m, n, ctypes.c_void_p(A.data_ptr()), m,
                                ctypes.c_void_p(B.data_ptr()), n, ctypes.c_void_p(C.data_ptr()), n,
                                _stream(stream)), "rtt_gemm_tn_f64")
    return C


def shard_rows(n_rows: int, index: int, count: int):
    """rtt_shard_rows: rows [begin, end) of row shard `index` of `count`."""
    b, e = ctypes.c_int64(0), ctypes.c_int64(0)
    sh = Shard(int(index), int(count))
    check(lib().rtt_shard_rows(int(n_rows), ctypes.byref(sh), ctypes.byref(b), ctypes.byref(e)),
          "rtt_shard_rows")
    return int(b.value), int(e.value)


def range_finder(op: "Operator", Q, omega, arm_mask: int = 7, block: int = 256, rho: float = 1.0,
                 stream=None):
    """rtt_range_finder: (sigma descending, rank, blocks used) of the
    restricted normal operator Q^T A^T A Q from the Gaussian draws omega
    (host float64 [d, block * max_blocks])."""
    _want(Q, "Q", (op.n_nodes, op.n_hats, None), ("float64",))
    d = Q.shape[2]
    om = np.ascontiguousarray(omega, np.float64)
    if om.ndim != 2 or om.shape[0] != d or om.shape[1] % block:
        raise ValueError(f"omega: want [{d}, a multiple of {block}], got {om.shape}")
    sig = np.empty(d)
    n, rank, blocks = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    check(lib().rtt_range_finder(op.handle, arm_mask, ctypes.c_void_p(Q.data_ptr()), d, block,
                                 om.shape[1] // block, _ptr(om, dp), rho, _ptr(sig, dp),
                                 ctypes.byref(n), ctypes.byref(rank), ctypes.byref(blocks),
                                 _stream(stream)), "rtt_range_finder")
    return sig[:n.value].copy(), rank.value, blocks.value


def rank_from_eigenvalues(evals, rho: float = 1.0):
    """rtt_operational_rank: (sigma sorted descending, rank, margin) of Eq. 31."""
    ev = np.ascontiguousarray(evals, np.float64).reshape(-1)
    sig = np.empty(ev.shape[0])
    rank = ctypes.c_int(0)
    margin = ctypes.c_double(0.0)
    check(lib().rtt_operational_rank(ev.shape[0], _ptr(ev, dp), rho, ctypes.byref(rank),
                                     ctypes.byref(margin), _ptr(sig, dp)), "rtt_operational_rank")
    return sig, rank.value, margin.value


def operational_rank(op: "Operator", Q, arm_mask: int = 7, rho: float = 1.0,
                     mode: int = GRAM_DATA):
    """Singular values (descending) of the whitened restricted operator and
    its operational rank (Eq. 31), both from the library: the Gram, its
    eigenvalues and the count."""
    G = gram(op, Q, arm_mask, mode)
    ev, V, _ = eig_sym(G)
    sig, rank, _ = rank_from_eigenvalues(ev, rho)
    return sig, rank


ARM_PAIRING_DESTROYED = 1  # rtt.h RTT_ARM_PAIRING_DESTROYED
ARM_DELAY_ONLY = 2
ARM_SPATIAL_ONLY = 3


def arm_table(table: dict, kind: int, keys=None) -> dict:
    """rtt_arm_table: the ray table of a Sec. 6.4 mechanism arm (dict of host
    arrays, as Operator takes); `keys` (one float per ray) is the random draw
    of the pairing-destroyed arm."""
    n = int(np.asarray(table["r"]).shape[0])
    order = np.ascontiguousarray(table["order"], np.int8)
    cols = {k: np.ascontiguousarray(table[k], np.float64) for k in ("r", "phi", "delay")}
    if order.shape[0] != n or any(v.shape[0] != n for v in cols.values()):
        raise ValueError("table columns differ in length")
    kd = None
    if keys is not None:
        kd = np.ascontiguousarray(keys, np.float64).reshape(-1)
        if kd.shape[0] != n:
            raise ValueError(f"keys: {kd.shape[0]} values for {n} rays")
    t = RayTable(n, order.ctypes.data_as(i8p), None, _ptr(cols["r"], dp), _ptr(cols["phi"], dp),
                 _ptr(cols["delay"], dp), None, None)
    out = {k: np.empty(n) for k in ("r", "phi", "delay")}
    check(lib().rtt_arm_table(int(kind), ctypes.byref(t), _ptr(kd, dp) if kd is not None else None,
                              _ptr(out["r"], dp), _ptr(out["phi"], dp), _ptr(out["delay"], dp)),
          "rtt_arm_table")
    res = dict(table)
    res.update(out)
    return res


def solve_ridge(op: "Operator", data, lambdas, arm_mask: int = 7, max_iter: int = 500,
                tol: float = 1e-6, refresh_every: int = 10, raise_on_stall: bool = True,
                stream=None):
    """Batched CG ridge solve; data: CUDA float32 [rows, frames, n_rhs].
    Returns (x [n_nodes, n_hats, n_rhs * n_lambda], iterations, relres)."""
    import torch
    _want(data, "data", (op.arm_rows(arm_mask), op.n_frames, None), ("float32",))
    lam = np.ascontiguousarray(lambdas, np.float64).reshape(-1)
    n_rhs = data.shape[2]
    ncol = n_rhs * lam.shape[0]
    x = torch.empty((op.n_nodes, op.n_hats, ncol), dtype=torch.float32, device=data.device)
    it = ctypes.c_int(0)
    rel = np.empty(ncol)
    st = lib().rtt_solve_ridge(op.handle, arm_mask, ctypes.c_void_p(data.data_ptr()), n_rhs,
                               _ptr(lam, dp), lam.shape[0], max_iter, tol, refresh_every,
                               ctypes.c_void_p(x.data_ptr()), ctypes.byref(it), _ptr(rel, dp),
                               _stream(stream))
    if st != -5 or raise_on_stall:
        check(st, "rtt_solve_ridge")
    return x, it.value, rel


def solve_tsvd(op: "Operator", Q, V, evals, rank: int, data, arm_mask: int = 7, stream=None):
    """TSVD in class Q (CUDA float64 [n_nodes, n_hats, d]) with eigenpairs (V, evals)
    sorted descending; data: CUDA float64 [rows, frames, n_rhs]."""
    import torch
    _want(Q, "Q", (op.n_nodes, op.n_hats, None), ("float64",))
    d = Q.shape[2]
    Vc = _want(V.contiguous(), "V", (d, d), ("float64",), like=Q)
    _want(data, "data", (op.arm_rows(arm_mask), op.n_frames, None), ("float64",), like=Q)
    n_rhs = data.shape[2]
    ev = np.ascontiguousarray(evals, np.float64).reshape(-1)
    if ev.shape[0] != d:
        raise ValueError(f"evals: {ev.shape[0]} values, expected d = {d}")
    xh = torch.empty((op.n_nodes, op.n_hats, n_rhs), dtype=torch.float64, device=data.device)
    check(lib().rtt_solve_tsvd(op.handle, arm_mask, ctypes.c_void_p(Q.data_ptr()), d,
                               ctypes.c_void_p(Vc.data_ptr()), _ptr(ev, dp), rank,
                               ctypes.c_void_p(data.data_ptr()), n_rhs,
                               ctypes.c_void_p(xh.data_ptr()), _stream(stream)), "rtt_solve_tsvd")
    return xh


def probe_info_mix(op: "Operator", mode: int, arm_mask: int = 7, ages=AGES, h: float = 3.0,
                   stream=None):
    """rtt_probe_info_mix: I_L(a) of the mixed arm `mode` (Eq. 4 with Eq. 10-12)."""
    ages = np.ascontiguousarray(ages, np.float64)
    info = np.empty(ages.shape[0])
    check(lib().rtt_probe_info_mix(op.handle, arm_mask, mode, ages.shape[0], _ptr(ages, dp), h,
                                   _ptr(info, dp), _stream(stream)), "rtt_probe_info_mix")
    return info


def probe_info_local(op: "Operator", arm_mask: int = 7, ages=AGES, h: float = 3.0, stream=None):
    """rtt_probe_info_local: I_l(a) of the 28 localized directions (Eq. 14),
    [n_ages, 28]."""
    ages = np.ascontiguousarray(ages, np.float64)
    info = np.empty((ages.shape[0], 28))
    check(lib().rtt_probe_info_local(op.handle, arm_mask, ages.shape[0], _ptr(ages, dp), h,
                                     _ptr(info, dp), _stream(stream)), "rtt_probe_info_local")
    return info


def gram_normal_mix(op: "Operator", Q, mode: int, arm_mask: int = 7, stream=None):
    """rtt_gram_normal_mix: G = Q^T A^T W^T W A Q for the mixed arm `mode`
    (Eq. 4, Eq. 7); Q: CUDA float64 [n_nodes, n_hats, d]."""
    import torch
    _want(Q, "Q", (op.n_nodes, op.n_hats, None), ("float64",))
    d = Q.shape[2]
    G = torch.empty((d, d), dtype=torch.float64, device=Q.device)
    check(lib().rtt_gram_normal_mix(op.handle, arm_mask, mode, ctypes.c_void_p(Q.data_ptr()), d,
                                    ctypes.c_void_p(G.data_ptr()), _stream(stream)),
          "rtt_gram_normal_mix")
    return G


def rank_audit(ops, Qs, arm_masks=(1, 7), ages=AGES, h: float = 3.0, quantile: float = 0.999,
               mode: int = GRAM_NORMAL, stream=None):
    """rtt_rank_audit over several operators; Qs: CUDA float64 [n_nodes, n_hats, d] each
    (entries may be None in the GRAM_CLASS_* modes, d = 224 there).
    Returns (records [n_ops][n_arms], sigma [n_ops, n_arms, d])."""
    n = len(ops)
    if Qs is None:
        Qs = [None] * n
    if len(Qs) != n:
        raise ValueError(f"Qs: {len(Qs)} entries for {n} operators")
    d = next((q.shape[2] for q in Qs if q is not None and q.dim() == 3), 224)
    for o, q in zip(ops, Qs):
        if q is not None:
            _want(q, "Q", (o.n_nodes, o.n_hats, d), ("float64",))
    arr_ops = (vp * n)(*[o.handle for o in ops])
    arr_q = (vp * n)(*[ctypes.c_void_p(q.data_ptr() if q is not None else None) for q in Qs])
    arms = (ctypes.c_int * len(arm_masks))(*arm_masks)
    ages = np.ascontiguousarray(ages, np.float64)
    recs = (AuditRecord * (n * len(arm_masks)))()
    sig = np.empty((n, len(arm_masks), d))
    check(lib().rtt_rank_audit(arr_ops, n, arr_q, d, arms, len(arm_masks), ages.shape[0],
                               _ptr(ages, dp), h, quantile, mode, recs, _ptr(sig, dp),
                               _stream(stream)),
          "rtt_rank_audit")
    out = [[recs[g * len(arm_masks) + a] for a in range(len(arm_masks))] for g in range(n)]
    return out, sig


class AuditPlan:
    """rtt_audit_plan_*: the class-Gram audit of several geometries as one
    batched plan (create builds every table; run enqueues the device work
    only, so it can be replayed or captured in a CUDA graph; results
    synchronises and returns (records [n_ops][n_arms], sigma [n_ops, n_arms,
    224]))."""

    def __init__(self, ops, arm_masks=(1, 7), ages=AGES, h: float = 3.0, quantile: float = 0.999,
                 kind: int = CLASS_S224, stream=None):
        self._ops = list(ops)  # keeps the operators alive as long as the plan
        self.n_ops, self.arms = len(self._ops), tuple(int(a) for a in arm_masks)
        arr_ops = (vp * self.n_ops)(*[o.handle for o in self._ops])
        arms = (ctypes.c_int * len(self.arms))(*self.arms)
        ages = np.ascontiguousarray(ages, np.float64)
        h_out = vp()
        check(lib().rtt_audit_plan_create(arr_ops, self.n_ops, arms, len(self.arms), ages.shape[0],
                                          _ptr(ages, dp), h, quantile, int(kind), _stream(stream),
                                          ctypes.byref(h_out)), "rtt_audit_plan_create")
        self.handle = h_out

    def run(self, stream=None):
        check(lib().rtt_audit_plan_run(self.handle, _stream(stream)), "rtt_audit_plan_run")

    def results(self, stream=None):
        n, na = self.n_ops, len(self.arms)
        recs = (AuditRecord * (n * na))()
        sig = np.empty((n, na, 224))
        check(lib().rtt_audit_plan_results(self.handle, recs, _ptr(sig, dp), _stream(stream)),
              "rtt_audit_plan_results")
        return [[recs[g * na + a] for a in range(na)] for g in range(n)], sig

    def close(self):
        if getattr(self, "handle", None):
            lib().rtt_audit_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _autograd():
    import torch

    class ApplyA(torch.autograd.Function):
        """y = scale * A x with the hand-written adjoint as its backward:
        grad_x = scale * A^T grad_y (both in librtt kernels)."""

        @staticmethod
        def forward(ctx, x, op: Operator, arm_mask: int):
            ctx.op = op
            ctx.arm = arm_mask
            return op.apply_A(x.contiguous(), arm_mask=arm_mask)

        @staticmethod
        def backward(ctx, gy):
            return ctx.op.apply_AT(gy.contiguous(), arm_mask=ctx.arm), None, None

    return ApplyA


_APPLY = None


def apply_A_autograd(x, op: Operator, arm_mask: int = 7):
    global _APPLY
    if _APPLY is None:
        _APPLY = _autograd()
    return _APPLY.apply(x, op, arm_mask)
