"""Parity at the workloads' full sizes.

* kerr256 (Kerr a=0.5, i=50 deg, 256x256 with 2x2 sub-rays in the photon-ring
  annulus, 64x128 nodes, 64 hats at 4M, 256 frames), in the launch
  configuration the benchmark times (FP32, batch 8, all three orders): every
  output of A and A^T against the oracle on the oracle's ray table, and the
  operator built from the GPU tracer's table against the oracle's rows.
* stress1024 (a in {0.94, 0}, i=75 deg, 1024x1024, 256x512 nodes, 256 hats,
  1024 frames): A on every coefficient of a dense batch, checked on sampled
  rows the oracle evaluates one sub-table at a time; A^T checked on every node
  for data supported on sampled rows (rows with zero data add nothing, so the
  oracle's sub-table adjoint is the exact full output); the dot identity
  <Ax, y> = <x, A^T y> on dense data in FP32 and FP64.
"""
import numpy as np
import pytest

import oracle as O
from paper_2609_05528_b300 import build, rtt
from paper_2609_05528_b300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _optable(tab):
    return {"order": tab.order, "pixel": tab.pixel, "r": tab.r, "phi": tab.phi,
            "delay": tab.delay, "weight": tab.weight, "throughput": tab.throughput}


def _rows(tab, rows):
    """Sub-table of the given rows (ascending), rays and row ids kept in order."""
    rows = np.asarray(rows, np.int64)
    counts = tab.row_ptr[rows + 1] - tab.row_ptr[rows]
    idx = np.concatenate([np.arange(tab.row_ptr[i], tab.row_ptr[i + 1]) for i in rows])
    rp = np.zeros(rows.size + 1, np.int64)
    rp[1:] = np.cumsum(counts)
    return O.Table(tab.order[idx], tab.pixel[idx], tab.r[idx], tab.phi[idx], tab.delay[idx],
                   tab.weight[idx], tab.throughput[idx], rp, tab.row_order[rows],
                   tab.row_pixel[rows], tab.sample[idx])


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


@pytest.fixture(scope="module")
def k256():
    w = I.kerr256()
    s = I.screen_samples(w)
    return w, s, O.build_table(w, s)


def test_kerr256_every_output(k256):
    w, _, tab = k256
    op = rtt.Operator(w, _optable(tab))
    scl = O.scale(tab)
    assert abs(op.scale / scl - 1.0) < 1e-12
    x = I.history_batch(w, range(100, 108))
    ref = O.apply_A(w, tab, x, scl)
    y = op.apply_A(torch.from_numpy(x.astype(np.float32)).cuda()).cpu().numpy().astype(np.float64)
    assert _rel(y, ref) < 1e-5
    assert np.max(np.abs(y - ref)) <= 1e-5 * np.max(np.abs(ref))
    yd = I.noise(ref.shape, 7)
    gref = O.apply_AT(w, tab, yd, scl)
    g = op.apply_AT(torch.from_numpy(yd.astype(np.float32)).cuda()).cpu().numpy().astype(np.float64)
    assert _rel(g, gref) < 1e-5
    assert np.max(np.abs(g - gref)) <= 1e-5 * np.max(np.abs(gref))
    # the benchmark's launch configuration: variants autotuned for batch 8,
    # the same bits as the default rule
    yt = torch.from_numpy(yd.astype(np.float32)).cuda()
    xt = torch.from_numpy(x.astype(np.float32)).cuda()
    y_rule, g_rule = op.apply_A(xt), op.apply_AT(yt)
    op.autotune(8)
    assert torch.equal(op.apply_A(xt), y_rule) and torch.equal(op.apply_AT(yt), g_rule)
    assert op.status(clear=True) == 0
    # direct-only arm on the same buffers
    d = tab.select((0,))
    y1 = op.apply_A(torch.from_numpy(x.astype(np.float32)).cuda(), arm_mask=1).cpu().numpy()
    assert _rel(y1.astype(np.float64), O.apply_A(w, d, x, scl)) < 1e-5
    op.close()


def test_kerr256_gpu_traced_operator(k256):
    """The benchmark's operator (GPU tracer table) against the oracle's rows:
    the same (order, pixel) rows up to rays at the source-grid edges, and the
    same outputs on the rows whose sub-ray count agrees."""
    w, s, tab = k256
    got = rtt.rtt_trace_rays(w.geometry.spin, w.geometry.incl_deg, w.grid, s)
    op = rtt.Operator(w, got)
    npx = w.geometry.nx * w.geometry.nx
    gkey = got["order"].astype(np.int64) * npx + got["pixel"]
    gk, gcount = np.unique(gkey, return_counts=True)  # device rows are sorted by (order, pixel)
    okey = tab.row_order.astype(np.int64) * npx + tab.row_pixel
    ocount = tab.row_ptr[1:] - tab.row_ptr[:-1]
    edge = (np.abs(tab.r - w.grid.r_in) < 1e-6) | (np.abs(tab.r - w.grid.r_out) < 1e-6)
    assert abs(gk.size - okey.size) <= int(edge.sum()) + 2
    common, gi, oi = np.intersect1d(gk, okey, return_indices=True)
    same = gcount[gi] == ocount[oi]
    assert same.sum() >= okey.size - int(edge.sum()) - 2
    x = I.history_batch(w, range(100, 108))
    sub = _rows(tab, oi[same])
    ref = O.apply_A(w, sub, x, O.scale(tab))
    y = op.apply_A(torch.from_numpy(x.astype(np.float32)).cuda()).cpu().numpy().astype(np.float64)
    assert abs(op.scale / O.scale(tab) - 1.0) < 1e-6
    assert _rel(y[gi[same]], ref) < 1e-5
    op.close()


@pytest.mark.parametrize("spin", [0.94, 0.0])
def test_stress1024(spin):
    w = I.stress1024(spin)
    tab = O.build_table(w, I.screen_samples(w))
    op = rtt.Operator(w, _optable(tab))
    scl = O.scale(tab)
    B = 2
    R, F = tab.n_rows, w.time.n_frames
    rng = np.random.default_rng(5)
    rows = np.unique(np.concatenate([[0, R - 1], rng.integers(0, R, 400),
                                     np.nonzero(tab.row_order > 0)[0][::97]]))
    # A: dense batch on the device, sampled rows through the oracle
    x = I.uniform_batch(w, range(1, 1 + B))
    xd = torch.from_numpy(x.astype(np.float32)).cuda()
    y = op.apply_A(xd)
    got = y[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
    ref = O.apply_A(w, _rows(tab, rows), x, scl)
    assert _rel(got, ref) < 1e-5
    # A^T: data on the sampled rows only, every node compared
    yd = np.zeros((R, F, B), np.float32)
    yd[rows] = I.noise((rows.size, F, B), 13).astype(np.float32)
    g = op.apply_AT(torch.from_numpy(yd).cuda()).cpu().numpy().astype(np.float64)
    gref = O.apply_AT(w, _rows(tab, rows), yd[rows].astype(np.float64), scl)
    assert _rel(g, gref) < 1e-5
    # dot identity on dense data, FP32 and FP64
    yn = torch.randn((R, F, B), generator=torch.Generator().manual_seed(3)).cuda()
    lhs = float((y.double() * yn.double()).sum())
    rhs = float((xd.double() * op.apply_AT(yn).double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
    del y
    y64 = op.apply_A(xd.double())
    yn64 = yn.double()
    lhs = float((y64 * yn64).sum())
    rhs = float((xd.double() * op.apply_AT(yn64)).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    op.close()
