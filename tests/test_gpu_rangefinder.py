"""rtt_range_finder (adaptive randomized range finder, block 256, FP64
projected eigensolve; Sec. 7-8) against the oracle's range finder on the
oracle's dense restricted Gram, with the same Gaussian draws:

  * the blocks used and the Ritz values above the rounding level agree (the
    Ritz values depend only on the span each block adds);
  * the rank read from them equals the oracle's;
  * with blocks until the basis spans the class, the rank equals the
    operational rank of the full Gram.
"""
import numpy as np
import pytest

import oracle as O
from paper_2609_05528_b300 import build, rtt
from paper_2609_05528_b300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

KINDS = {"S224": 0, "L448": 5, "S528S": 3}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


@pytest.fixture(scope="module")
def case():
    w = I.schw32()
    tab = O.build_table(w, I.screen_samples(w))
    op = rtt.Operator(w, {"order": tab.order, "pixel": tab.pixel, "r": tab.r, "phi": tab.phi,
                          "delay": tab.delay, "weight": tab.weight,
                          "throughput": tab.throughput})
    yield w, tab, op
    op.close()


@pytest.mark.parametrize("kind", list(KINDS))
@pytest.mark.parametrize("mask", [1, 7])
def test_range_finder_matches_the_oracle(case, kind, mask):
    w, tab, op = case
    d = rtt.class_dim(KINDS[kind])
    Q = rtt.synth_class(op, KINDS[kind])
    Qo = O.synth_class_ladder(w, kind)
    sub = tab.select(tuple(n for n in range(3) if mask & (1 << n)))
    G = O.gram(O.restricted_response(w, sub, Qo, O.scale(tab)))
    n_blocks = (d + 255) // 256 + 1
    omega = I.normals(900 + d + mask, d * 256 * n_blocks).reshape(d, 256 * n_blocks)
    ritz, k_ref, used_ref = O.range_finder(G, omega, 256, rho=1.0)
    sig, rank, used = rtt.range_finder(op, Q, omega, mask, 256, rho=1.0)
    lam_max = float(np.max(np.linalg.eigvalsh(G)))
    assert used == used_ref, (used, used_ref, sig.shape[0], k_ref)
    # the basis sizes may differ by directions at the rounding level (kept on
    # one side, dropped on the other); the Ritz values above it agree.  H
    # enters twice through contractions truncated at 49 bits (2^-44 of
    # sum |a| |b|, with cancellation in Q^T z): about 1e-9 of lambda_max
    top = ritz[ritz >= 1e-6 * lam_max]
    assert sig.shape[0] >= top.shape[0]
    np.testing.assert_allclose(sig[:top.shape[0]] ** 2, top, rtol=0, atol=1e-8 * lam_max)
    sig_ref = np.sqrt(np.maximum(ritz, 0.0))
    if np.min(np.abs(sig_ref - 1.0)) > 1e-6:
        assert rank == int(np.count_nonzero(sig_ref >= 1.0))
    if k_ref == d:  # the basis spans the class: the operational rank of the Gram
        lam = np.linalg.eigvalsh(G)
        s = np.sqrt(np.maximum(lam, 0.0))
        if np.min(np.abs(s - 1.0)) > 1e-6:
            assert rank == int(np.count_nonzero(s >= 1.0))
