"""BF16 corner weights (rtt_set_weight_precision) on the GPU against the
oracle's BF16-weight operator:

  * FP32 applies with BF16 weights match the FP64 oracle with the same
    BF16-rounded weights to the FP32 tolerance (1e-5 relative L2);
  * every kernel variant gives the same bits (the FP32 table holds the same
    rounded values that the fast kernels read from the BF16 copy);
  * the FP64 applies keep the FP64 weights; switching back to FP32 weights
    restores the original bits.
"""
import numpy as np
import pytest

import oracle as O
from paper_2609_05528_b300 import build, rtt
from paper_2609_05528_b300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    rtt.lib()


def _optable(tab):
    return {"order": tab.order, "pixel": tab.pixel, "r": tab.r, "phi": tab.phi,
            "delay": tab.delay, "weight": tab.weight, "throughput": tab.throughput}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def case():
    w = I.small_kerr(spin=0.5, incl_deg=50.0, nx=48, n_r=12, n_phi=24, n_frames=300,
                     n_hats=80, ss=2)
    tab = O.build_table(w, I.screen_samples(w))
    return w, tab, O.scale(tab)


@pytest.mark.parametrize("B", [1, 4, 8, 16])
def test_bf16_weights_against_oracle_and_variants(case, B):
    w, tab, scl = case
    op = rtt.Operator(w, _optable(tab))
    x = I.uniform_batch(w, range(B))
    xt = torch.from_numpy(x.astype(np.float32)).cuda()
    y32 = op.apply_A(xt)
    op.set_weight_precision(rtt.WEIGHTS_BF16)
    assert op.info.weight_precision == rtt.WEIGHTS_BF16
    y = op.apply_A(xt)
    ref = O.apply_A(w, tab, x, scl, bf16=True)
    assert _rel(y.cpu().numpy().astype(np.float64), ref) <= TOL32
    # the BF16 operator is a different operator from the FP32-weight one
    assert _rel(y.cpu().numpy().astype(np.float64), O.apply_A(w, tab, x, scl)) > 1e-5
    d = I.noise((tab.n_rows, w.time.n_frames, B), 7 + B)
    g = op.apply_AT(torch.from_numpy(d.astype(np.float32)).cuda())
    assert _rel(g.cpu().numpy().astype(np.float64), O.apply_AT(w, tab, d, scl, bf16=True)) <= TOL32
    # every forward and adjoint kernel variant: the same bits
    dt = torch.from_numpy(d.astype(np.float32)).cuda()
    bc = 1
    while bc < min(B, 16):
        bc *= 2
    for fk in (1, 2, 3, 4, 5, 6, 7, 8, 9):
        op.set_variant(B, fk, bc, 0, 1)
        assert torch.equal(op.apply_A(xt), y), fk
    for ak in (1, 2, 3, 4):
        op.set_variant(B, 1, bc, 0, ak)
        assert torch.equal(op.apply_AT(dt), g), ak
    op.set_variant(B)
    assert op.status() == 0
    # FP64 applies keep the FP64 weights
    y64 = op.apply_A(torch.from_numpy(x).cuda()).cpu().numpy()
    assert _rel(y64, O.apply_A(w, tab, x, scl)) <= 1e-12
    # back to FP32 weights: the original bits
    op.set_weight_precision(rtt.WEIGHTS_FP32)
    assert torch.equal(op.apply_A(xt), y32)
    op.close()
