"""The C-ABI library loads, exports every entry point declared in
include/rtt.h, and rejects invalid arguments before touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2609_05528_b300 import build, rtt
from paper_2609_05528_b300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return rtt.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rtt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rtt_[A-Za-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert "rtt_apply_A" in names and "rtt_build_operator" in names
    for n in names:
        assert hasattr(L, n), n
    # the binding wraps exactly the declared entry points
    assert set(rtt.exported_symbols()) == set(names)


def test_status_strings(L):
    assert L.rtt_abi_version() == rtt.ABI_VERSION == 2
    assert L.rtt_error_string(0) == b"ok"
    assert L.rtt_error_string(-1) == b"invalid argument"


def _table(n=4):
    return {"order": np.zeros(n, np.int8), "pixel": np.arange(n, dtype=np.int32),
            "r": np.full(n, 5.0), "phi": np.linspace(0, 1, n), "delay": np.zeros(n),
            "weight": np.ones(n), "throughput": np.ones(n)}


@pytest.mark.parametrize("bad", ["r_out_of_range", "order", "nonfinite", "no_direct",
                                 "cadence", "grid", "negative_pixel", "negative_order", "empty",
                                 "huge_delay", "hat_offset", "no_hats", "no_frames",
                                 "radial_range", "spin", "snr0"])
def test_build_rejects_invalid_tables_on_host(L, bad):
    w = I.schw32()
    tab = _table()
    kw = {}
    if bad == "negative_pixel":
        tab["pixel"][3] = -1
    elif bad == "negative_order":
        tab["order"][0] = -1
    elif bad == "empty":
        tab = {k: v[:0] for k, v in tab.items()}
    elif bad == "huge_delay":
        tab["delay"][1] = 2e6
    elif bad == "hat_offset":  # |u0| above 2^20 hat steps of 4 M
        w = I.Workload("h", w.geometry, w.grid, I.TimeGrid(24, 2.0, 12, t_end=4.0 * 2 ** 21))
    elif bad == "no_hats":
        w = I.Workload("k", w.geometry, w.grid, I.TimeGrid(24, 2.0, 0, t_end=0.0))
    elif bad == "no_frames":
        w = I.Workload("f", w.geometry, w.grid, I.TimeGrid(0, 2.0, 12, t_end=0.0))
    elif bad == "radial_range":
        w = I.Workload("r", w.geometry, I.SourceGrid(4, 16, r_in=5.0, r_out=5.0), w.time)
    elif bad == "spin":
        w = I.Workload("s", I.Geometry(1.0, 50.0, 32), w.grid, w.time)
    elif bad == "snr0":
        kw = {"snr0": 0.0}
    if bad == "r_out_of_range":
        tab["r"][1] = 11.5
    elif bad == "order":
        tab["order"][2] = 3
    elif bad == "nonfinite":
        tab["delay"][0] = np.nan
    elif bad == "no_direct":
        tab["order"][:] = 1
    elif bad == "cadence":
        w = I.Workload("c", w.geometry, w.grid, I.TimeGrid(24, 0.3, 12, t_end=0.0))
    elif bad == "grid":
        w = I.Workload("g", w.geometry, I.SourceGrid(1, 16), w.time)
    with pytest.raises(rtt.RttError) as ei:
        rtt.Operator(w, tab, stream=0, **kw)
    assert ei.value.status == -1


def test_trace_rejects_bad_geometry(L):
    w = I.schw32()
    s = I.screen_samples(w)
    with pytest.raises(rtt.RttError):
        rtt.rtt_trace_rays(0.5, 95.0, w.grid, s, stream=0)
    with pytest.raises(rtt.RttError):
        rtt.rtt_trace_rays(1.2, 50.0, w.grid, s, stream=0)


def test_mix_rejects_invalid_arguments_on_host(L):
    """Order mixing checks its mode and pointers before any device work."""
    n = ctypes.c_int64()
    assert L.rtt_mix_rows_count(None, 7, 1, ctypes.byref(n)) == -1
    assert L.rtt_mix_rows(None, 7, 1, None, None, 1, None) == -1
    assert L.rtt_mix_rows_T_f64(None, 7, 2, None, None, 1, None) == -1
    assert L.rtt_gram_normal_mix(None, 7, 3, None, 4, None, None) == -1
    assert L.rtt_gram_normal_mix(None, 7, 1, None, 4, None, None) == -1


def test_mixed_probe_rejects_invalid_arguments_on_host(L):
    ages = np.zeros(4)
    info = np.zeros(4)
    dp = ctypes.POINTER(ctypes.c_double)
    a = ages.ctypes.data_as(dp)
    i = info.ctypes.data_as(dp)
    assert L.rtt_probe_info_mix(None, 7, 1, 4, a, 3.0, i, None) == -1
    assert L.rtt_probe_info_mix(None, 7, 5, 4, a, 3.0, i, None) == -1


def test_localized_probe_rejects_invalid_arguments_on_host(L):
    ages = np.zeros(4)
    info = np.zeros(4 * 28)
    dp = ctypes.POINTER(ctypes.c_double)
    assert L.rtt_probe_info_local(None, 7, 4, ages.ctypes.data_as(dp), 3.0,
                                  info.ctypes.data_as(dp), None) == -1


def test_class_dimensions(L):
    """The ladder of Sec. 7-8: (4,7,8), (4,7,8), (4,7,16), (6,11,8), (6,11,16),
    (4,7,16), (6,11,16) -> 224, 224, 448, 528, 1056, 448, 1056."""
    assert [L.rtt_class_dim(k) for k in range(7)] == [224, 224, 448, 528, 1056, 448, 1056]
    assert L.rtt_class_dim(7) == 0 and L.rtt_class_dim(-1) == 0


def test_every_entry_point_rejects_null_arguments(L):
    """Each status-returning entry point, called with null pointers and zero
    sizes, returns RTT_EINVAL and sets the error message before it touches a
    GPU (no crash, no CUDA call on the CPU host)."""
    plain = {"rtt_error_string", "rtt_last_error", "rtt_abi_version", "rtt_class_dim",
             "rtt_destroy", "rtt_audit_plan_destroy"}
    for name, (_, argtypes) in rtt._SIGS.items():
        if name in plain:
            continue
        vals = [0 if a in (ctypes.c_int, ctypes.c_int32, ctypes.c_int64)
                else 0.0 if a is ctypes.c_double else None for a in argtypes]
        assert getattr(L, name)(*vals) == -1, name
        assert L.rtt_last_error(), name


def test_every_entry_point_is_documented():
    """Each declaration block of include/rtt.h carries a comment that cites
    the passage it implements (or says the paper has no counterpart) and
    states its error behaviour."""
    src = open(os.path.join(ROOT, "include", "rtt.h")).read()
    n = 0
    for m in re.finditer(r"^(?:rtt_status|int|void|const char\*)\s+(rtt_\w+)\s*\(", src, re.M):
        end = src.rfind("*/", 0, m.start())
        if end < 0 or src[end + 2:m.start()].strip():
            continue  # shares the comment of the declaration before it
        doc, name = src[src.rfind("/*", 0, end) + 2:end], m.group(1)
        n += 1
        if name == "rtt_probe_info_noalloc":
            # an allocation-free variant: no passage of its own to cite
            assert "no counterpart" in doc and not re.search(r"Sec\.|Eq\.", doc), name
        else:
            assert re.search(r"Sec\.|Eq\.|Theorem|counterpart", doc), name
        assert re.search(r"\bErrors?\b|RTT_E|never fails", doc, re.I), name
    assert n >= 25
