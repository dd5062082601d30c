"""rtt_probe_info_noalloc: the probe-information pass for callers that cannot
allocate device memory at run time (for example an application whose pool
allocator already holds all free device memory, or a runtime that forbids
allocation after start-up).  Its scratch is a static device array inside the
library; inputs and outputs stay caller-owned device buffers.

Checked through the C ABI against the allocating entry point rtt_probe_info,
within the tolerance the probe parity tests use, on two calls in a row (the
shared static array keeps the previous call's contents, which must not leak
into the next result).  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_2609_05528_b300 import build, rtt
from paper_2609_05528_b300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_noalloc_probe_matches_allocating_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    L = rtt.lib()
    w = I.small_kerr(spin=0.5, incl_deg=50.0, nx=48, n_r=12, n_phi=24, n_frames=96, n_hats=24)
    tab = O.build_table(w, I.screen_samples(w))
    op = rtt.Operator(w, {"order": tab.order, "pixel": tab.pixel, "r": tab.r, "phi": tab.phi,
                          "delay": tab.delay, "weight": tab.weight,
                          "throughput": tab.throughput})
    stream = torch.cuda.current_stream()
    for mask, ages in ((7, rtt.AGES), (1, rtt.AGES[:17] + 1.0)):
        ref = rtt.probe_info(op, mask, ages)
        ages_d = torch.from_numpy(np.ascontiguousarray(ages)).cuda()
        for call in range(2):
            out = torch.full((ages.shape[0],), np.nan, dtype=torch.float64, device="cuda")
            st = L.rtt_probe_info_noalloc(op.handle, mask, ages.shape[0],
                                          ctypes.c_void_p(ages_d.data_ptr()), 3.0,
                                          ctypes.c_void_p(out.data_ptr()),
                                          ctypes.c_void_p(stream.cuda_stream))
            rtt.check(st, "rtt_probe_info_noalloc")
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            big = ref > 1e-30 * ref.max()
            assert np.allclose(got[big], ref[big], rtol=2e-5), (mask, call)
            assert np.all(np.abs(got[~big]) <= 1e-6 * ref.max())
    # sizes beyond the static scratch are rejected with a clear error
    too_many = torch.zeros(257, dtype=torch.float64, device="cuda")
    st = L.rtt_probe_info_noalloc(op.handle, 7, 257, ctypes.c_void_p(too_many.data_ptr()), 3.0,
                                  ctypes.c_void_p(too_many.data_ptr()),
                                  ctypes.c_void_p(stream.cuda_stream))
    assert st == -1
    assert b"static scratch limit" in L.rtt_last_error()
