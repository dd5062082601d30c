"""The mechanism arms of Sec. 6.4 as built by the library (rtt_arm_table,
host code) against the oracle's own constructions (oracle.pairing_destroyed,
oracle.delay_only, oracle.spatial_only), table for table: the two are written
independently, so a wrong quantile-partner or permutation rule on either side
fails here.  No GPU is needed."""
import numpy as np
import pytest

import oracle as O
from paper_2609_05528_b300 import build, rtt
from paper_2609_05528_b300 import inputs as I


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    rtt.lib()


def _dict(tab):
    return {"order": tab.order, "pixel": tab.pixel, "r": tab.r, "phi": tab.phi,
            "delay": tab.delay, "weight": tab.weight, "throughput": tab.throughput}


@pytest.fixture(scope="module", params=["schw32", "small_kerr"])
def case(request):
    w = I.schw32() if request.param == "schw32" else I.small_kerr(
        spin=0.94, incl_deg=75.0, nx=64, n_r=8, n_phi=16, n_frames=64, n_hats=16, ss=2)
    return w, O.build_table(w, I.screen_samples(w))


def test_library_arm_tables_equal_the_oracle(case):
    w, tab = case
    keys = I.uniforms(1000, tab.n_rays)
    pairs = ((rtt.ARM_PAIRING_DESTROYED, O.pairing_destroyed(tab, keys)),
             (rtt.ARM_DELAY_ONLY, O.delay_only(tab)),
             (rtt.ARM_SPATIAL_ONLY, O.spatial_only(tab)))
    for kind, ref in pairs:
        got = rtt.arm_table(_dict(tab), kind, keys if kind == rtt.ARM_PAIRING_DESTROYED else None)
        for k in ("r", "phi", "delay"):
            np.testing.assert_array_equal(got[k], getattr(ref, k), err_msg=f"{kind} {k}")
        for k in ("order", "pixel", "weight", "throughput"):
            assert got[k] is _dict(tab)[k] or np.array_equal(got[k], getattr(tab, k))


def test_library_arm_table_hand_case():
    """The hand case of the oracle's quantile-partner pin, through the
    library: ring rays 4, 5, 6 take direct partners 2, 3, 0."""
    order = np.array([0, 0, 0, 0, 1, 1, 2], np.int8)
    t = {"order": order, "r": 3.0 + np.arange(7.0), "phi": 0.1 * np.arange(7.0),
         "delay": np.array([3.0, 1.0, 4.0, 2.0, 9.0, 7.0, 20.0])}
    do = rtt.arm_table(t, rtt.ARM_DELAY_ONLY)
    assert do["r"].tolist() == [3.0, 4.0, 5.0, 6.0, 5.0, 6.0, 3.0]
    so = rtt.arm_table(t, rtt.ARM_SPATIAL_ONLY)
    assert so["delay"].tolist() == [3.0, 1.0, 4.0, 2.0, 4.0, 2.0, 3.0]
    pd = rtt.arm_table(t, rtt.ARM_PAIRING_DESTROYED, [0.5, 0.1, 0.3, 0.2, 0.9, 0.8, 0.0])
    # order 0 by key: rays 1, 3, 2, 0 -> ray 0 takes 1's delay, 1 takes 3's, ...
    assert pd["delay"].tolist() == [1.0, 2.0, 4.0, 3.0, 7.0, 9.0, 20.0]


def test_library_arm_table_rejects_bad_input():
    t = {"order": np.array([1, 1], np.int8), "r": np.ones(2), "phi": np.zeros(2),
         "delay": np.zeros(2)}
    with pytest.raises(rtt.RttError):
        rtt.arm_table(t, rtt.ARM_DELAY_ONLY)  # no direct ray
    with pytest.raises(rtt.RttError):
        rtt.arm_table(t, rtt.ARM_PAIRING_DESTROYED)  # keys missing
    with pytest.raises(rtt.RttError):
        rtt.arm_table(t, 9)
