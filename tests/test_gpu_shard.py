"""Row shards of the operator (rtt_build_operator_shard) on one GPU, against
the whole operator and the oracle.  The shards are built and applied one
after another (no rank waits on another); the rank-order combination is the
one ShardedOperator performs over torch.distributed:

  * the shards' A x, concatenated in shard order, are the whole operator's
    A x bit for bit (FP32 and FP64): each row is computed from its own rays
    and the whole table's whitening scale (Sec. 3.1, Eq. 17-18);
  * the shards' A^T y of their rows, summed in shard order, are the whole
    A^T y within rounding (FP64: 1e-13 relative; FP32: the apply tolerance
    against the oracle);
  * row-additive reductions (probe information, Gram) sum over shards;
  * entry points that need every row refuse a shard (RTT_ESTATE).
"""
import numpy as np
import pytest

import oracle as O
from paper_2609_05528_b300 import build, rtt
from paper_2609_05528_b300 import inputs as I
from paper_2609_05528_b300.shard import arm_row_range

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    rtt.lib()


def _optable(tab):
    return {"order": tab.order, "pixel": tab.pixel, "r": tab.r, "phi": tab.phi,
            "delay": tab.delay, "weight": tab.weight, "throughput": tab.throughput}


@pytest.fixture(scope="module")
def case():
    w = I.small_kerr(spin=0.5, incl_deg=50.0, nx=48, n_r=12, n_phi=24, n_frames=300,
                     n_hats=80, ss=2)
    tab = O.build_table(w, I.screen_samples(w))
    whole = rtt.Operator(w, _optable(tab))
    return w, tab, whole


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("n", [2, 3, 5])
@pytest.mark.parametrize("mask", [7, 1, 6])
def test_shards_tile_the_whole_operator(case, n, mask):
    w, tab, whole = case
    shards = [rtt.Operator(w, _optable(tab), shard=(i, n)) for i in range(n)]
    assert sum(s.info.n_rows for s in shards) == whole.info.n_rows
    assert sum(s.info.n_rays for s in shards) == whole.info.n_rays
    for i, s in enumerate(shards):
        assert (s.shard_index, s.shard_count) == (i, n)
        assert s.scale == whole.scale and s.total_rows == whole.info.n_rows
        assert (s.shard_row_begin, s.shard_row_begin + s.info.n_rows) == \
            rtt.shard_rows(whole.info.n_rows, i, n)
    B = 8
    for dt in (torch.float32, torch.float64):
        x = torch.from_numpy(I.uniform_batch(w, range(B))).to(dt).cuda()
        y = whole.apply_A(x, arm_mask=mask)
        parts = [s.apply_A(x, arm_mask=mask) for s in shards]
        assert torch.equal(torch.cat(parts, 0), y)
        d = torch.from_numpy(I.noise((y.shape[0], w.time.n_frames, B), 9 + n)).to(dt).cuda()
        g = whole.apply_AT(d, arm_mask=mask)
        acc = None
        for s in shards:
            a, b = arm_row_range(s.total_rows_per_order, s.shard_row_begin,
                                 s.shard_row_begin + s.info.n_rows, mask)
            part = s.apply_AT(d[a:b].contiguous(), arm_mask=mask)
            acc = part.clone() if acc is None else acc + part
        tol = 1e-13 if dt == torch.float64 else 1e-5
        assert _rel(acc, g) <= tol
    assert all(s.status() == 0 for s in shards)


def test_shard_fp32_against_oracle(case):
    w, tab, whole = case
    n, B = 2, 4
    shards = [rtt.Operator(w, _optable(tab), shard=(i, n)) for i in range(n)]
    scl = O.scale(tab)
    y = np.ascontiguousarray(O.apply_A(w, tab, I.uniform_batch(w, range(B)), scl))
    ref = O.apply_AT(w, tab, y, scl)
    acc = None
    for s in shards:
        a, b = s.shard_row_begin, s.shard_row_begin + s.info.n_rows
        part = s.apply_AT(torch.from_numpy(y[a:b].astype(np.float32)).cuda())
        acc = part.clone() if acc is None else acc + part
    got = acc.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5


def test_row_additive_reductions(case):
    w, tab, whole = case
    n = 3
    shards = [rtt.Operator(w, _optable(tab), shard=(i, n)) for i in range(n)]
    ages = np.linspace(0.0, 40.0, 9)
    info = rtt.probe_info(whole, arm_mask=7, ages=ages)
    parts = sum(rtt.probe_info(s, arm_mask=7, ages=ages) for s in shards)
    # FP32 exponentials with FP64 sums; values near rho^2 are re-evaluated in
    # FP64, which a shard decides on its own partial value
    np.testing.assert_allclose(parts, info, rtol=1e-6, atol=0)
    Q = rtt.synth_class(whole, rtt.CLASS_S224)
    G = rtt.gram(whole, Q, arm_mask=7)
    Gs = sum(rtt.gram(s, Q, arm_mask=7) for s in shards)
    assert _rel(Gs, G) <= 1e-12


def test_whole_only_entry_points_refuse_a_shard(case):
    w, tab, whole = case
    s = rtt.Operator(w, _optable(tab), shard=(1, 2))
    with pytest.raises(rtt.RttError, match="whole operator"):
        rtt.direct_age_quantile(s, 0.999)
    with pytest.raises(rtt.RttError, match="whole operator"):
        s.mix_rows_count(rtt.MIX_UNRESOLVED, arm_mask=7)
    with pytest.raises(rtt.RttError):
        rtt.Operator(w, _optable(tab), shard=(2, 2))
    with pytest.raises(rtt.RttError):
        rtt.Operator(w, _optable(tab), shard=(0, tab.n_rows + 1))
