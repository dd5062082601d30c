"""The delay-only and spatial-only mechanism arms (Sec. 6.4) on the GPU: the
operators built from their tables (ring source points or ring delays moved to
their direct quantile partners') against the oracle on the same tables."""
import numpy as np
import pytest

import oracle as O
from paper_2609_05528_b300 import build, rtt
from paper_2609_05528_b300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


@pytest.fixture(scope="module")
def schw():
    w = I.schw32()
    return w, O.build_table(w, I.screen_samples(w))


def _optable(tab):
    return {"order": tab.order, "pixel": tab.pixel, "r": tab.r, "phi": tab.phi,
            "delay": tab.delay, "weight": tab.weight, "throughput": tab.throughput}


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("arm", ["delay_only", "spatial_only"])
def test_delay_only_and_spatial_only_operators(schw, arm):
    w, tab = schw
    kind = rtt.ARM_DELAY_ONLY if arm == "delay_only" else rtt.ARM_SPATIAL_ONLY
    t = rtt.arm_table(_optable(tab), kind)           # the library's construction
    tt = getattr(O, arm)(tab)                          # the oracle's own
    op = rtt.Operator(w, t)
    x = I.uniform_batch(w, range(3))
    scl = O.scale(tt)
    assert abs(op.scale / scl - 1.0) < 1e-12
    y = op.apply_A(torch.from_numpy(x).cuda()).cpu().numpy()
    assert _rel(y, O.apply_A(w, tt, x, scl)) <= 1e-12
    info = rtt.probe_info(op, 7)
    assert _rel(info, O.probe_info(w, tt, scl)) <= 1e-5
    op.close()
