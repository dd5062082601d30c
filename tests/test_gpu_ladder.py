"""The class ladder of Sec. 7-8 on the GPU: every class synthesised against
the oracle; Theorem 4.1's exactly-zero direct columns bit for bit; the
restricted Gram of the larger classes against the oracle; rank along the
nesting."""
import numpy as np
import pytest

import oracle as O
from paper_2609_05528_b300 import build, rtt
from paper_2609_05528_b300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

KINDS = {"S224": 0, "L224": 1, "S448T": 2, "S528S": 3, "S1056ST": 4, "L448": 5, "L1056": 6}


def _optable(tab):
    return {"order": tab.order, "pixel": tab.pixel, "r": tab.r, "phi": tab.phi,
            "delay": tab.delay, "weight": tab.weight, "throughput": tab.throughput}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


@pytest.fixture(scope="module")
def schw():
    w = I.schw32()
    tab = O.build_table(w, I.screen_samples(w))
    op = rtt.Operator(w, _optable(tab))
    yield w, tab, op
    op.close()


@pytest.mark.parametrize("kind", list(KINDS))
def test_synthesis(schw, kind):
    w, _, op = schw
    Q = rtt.synth_class(op, KINDS[kind]).cpu().numpy().reshape(-1, rtt.class_dim(KINDS[kind]))
    ref = O.synth_class_ladder(w, kind)
    assert np.max(np.abs(Q - ref)) <= 1e-13


@pytest.mark.parametrize("kind", ["L224", "L448", "L1056", "S448T"])
def test_exact_zero_direct_columns(schw, kind):
    """The direct Gram's zero diagonal entries are exactly the oracle's zero
    columns of the direct response (Theorem 4.1 and joint support)."""
    w, tab, op = schw
    Q = rtt.synth_class(op, KINDS[kind])
    G = rtt.gram(op, Q, 1, mode=rtt.GRAM_NORMAL).cpu().numpy()
    P = O.restricted_response(w, tab.select((0,)), O.synth_class_ladder(w, kind), 1.0)
    want = np.all(P == 0.0, axis=0)
    got = np.diag(G) == 0.0
    assert np.array_equal(got, want)
    if kind.startswith("L"):
        assert got.sum() > 0


@pytest.mark.parametrize("kind", ["S448T", "S528S", "L1056"])
def test_gram_against_oracle(schw, kind):
    w, tab, op = schw
    Q = rtt.synth_class(op, KINDS[kind])
    G = rtt.gram(op, Q, 7, mode=rtt.GRAM_NORMAL).cpu().numpy()
    P = O.restricted_response(w, tab, O.synth_class_ladder(w, kind), O.scale(tab))
    Gref = P.T @ P
    assert np.max(np.abs(G - Gref)) <= 1e-10 * np.max(np.abs(Gref))


def test_rank_along_the_nesting(schw):
    """S224 within S448T within S1056ST and S224 within S528S within S1056ST:
    the operational rank (sigma >= 1) never decreases along the nesting."""
    w, tab, op = schw
    rank = {}
    for kind in ("S224", "S448T", "S528S", "S1056ST"):
        G = rtt.gram(op, rtt.synth_class(op, KINDS[kind]), 7, mode=rtt.GRAM_NORMAL)
        ev = rtt.eigvals_sym_batched(G[None])[0]
        rank[kind] = int(np.count_nonzero(np.sqrt(np.maximum(ev, 0)) >= 1.0))
    assert rank["S224"] <= rank["S448T"] <= rank["S1056ST"]
    assert rank["S224"] <= rank["S528S"] <= rank["S1056ST"]
