"""Adversarial ray tables (hand-made, on the 32x32 workload's grids): radii
exactly at r_in and r_out, azimuths at 0, 2 pi, negative and several turns,
delays that put source times exactly on hat centres, on half-hat points, on
the oldest hat, past it and younger than the youngest, and rows of one and of
four sub-rays.  The oracle half runs on CPU; the GPU half compares both
applies, FP64 and FP32, with the oracle and checks their exact zero patterns:
in FP64 the GPU's zeros are the oracle's zeros for A and A^T alike; in FP32 a
hat whose exact weight is below 2^-24 (the 24-bit fixed-point hat fraction
floors it to zero) may give an exact zero where the oracle's output is not
zero, but never the reverse, and only where that output is below 2^-24 of
the output scale max A^T |y| (A has no negative entry)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2609_05528_b300 import inputs as I

TWO_PI = 2.0 * math.pi

# (order, pixel, r, phi, delay, sub-rays of the pixel); rows sorted by (order, pixel)
RAYS = [
    (0, 0, 3.0, 0.0, 0.0, 1),                     # r_in, phi 0, source time on hat 0
    (0, 1, 11.0, TWO_PI, 4.0, 1),                 # r_out, phi = 2 pi, on hat 1
    (0, 2, 5.0, -0.5 * math.pi, 2.0, 1),          # negative phi, half-hat points
    (0, 3, 4.0, TWO_PI - 1e-12, 8.0 + 1e-9, 4),   # just below 2 pi, just off a hat centre
    (0, 3, 6.5, math.pi, 8.0, 4),
    (0, 3, 10.999999999, 1e-300, 12.0, 4),        # tiny phi, r just inside r_out
    (0, 3, 3.000000001, 3 * TWO_PI + 0.5, 20.0, 4),  # three turns
    (0, 4, 7.0, 1.0, 44.0, 1),                    # frame 0 on the oldest hat
    (0, 5, 8.0, 2.0, 50.0, 1),                    # older than every hat at early frames
    (1, 0, 3.0, 3.0, 25.0, 1),
    (1, 7, 11.0, -6.0, 31.5, 1),
    (2, 1, 9.0, 6.283185307179586, 40.0, 1),
]


def edge_table():
    a = np.array([r[:5] for r in RAYS], dtype=np.float64)
    nsub = np.array([r[5] for r in RAYS], dtype=np.float64)
    order = a[:, 0].astype(np.int8)
    pixel = a[:, 1].astype(np.int32)
    key = order.astype(np.int64) * 1024 + pixel
    starts = np.nonzero(np.concatenate([[True], key[1:] != key[:-1]]))[0]
    rp = np.concatenate([starts, [key.size]]).astype(np.int64)
    w = 1.0 / nsub
    return O.Table(order, pixel, a[:, 2].copy(), a[:, 3].copy(), a[:, 4].copy(), w, w.copy(),
                   rp, order[starts], pixel[starts], np.arange(key.size, dtype=np.int64))


def test_edge_table_oracle_structure():
    """The table is what it claims: sorted rows, and the oracle's outputs
    hold exact zeros (frames whose source time misses every hat) as well as
    non-zeros on every row."""
    w = I.schw32()
    tab = edge_table()
    assert tab.n_rows == 9 and tab.n_rays == len(RAYS)
    x = I.uniform_batch(w, range(2))
    y = O.apply_A(w, tab, x, 1.0)
    assert np.any(y == 0.0) and np.all(np.any(y != 0.0, axis=(1, 2)))
    # the ray at the oldest hat sees it with weight one at frame 0
    r4 = int(np.nonzero((tab.row_order == 0) & (tab.row_pixel == 4))[0][0])
    assert np.all(y[r4, 0] != 0.0)
    # dot test of the oracle pair on this table
    yd = I.noise(y.shape, 3)
    lhs = float(np.sum(y * yd))
    rhs = float(np.sum(x * O.apply_AT(w, tab, yd, 1.0)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.gpu
def test_edge_table_gpu_against_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_05528_b300 import build, rtt
    build.build()
    w = I.schw32()
    tab = edge_table()
    op = rtt.Operator(w, {"order": tab.order, "pixel": tab.pixel, "r": tab.r, "phi": tab.phi,
                          "delay": tab.delay, "weight": tab.weight,
                          "throughput": tab.throughput})
    scl = O.scale(tab)
    assert abs(op.scale / scl - 1.0) < 1e-12
    x = I.uniform_batch(w, range(4))
    ref = O.apply_A(w, tab, x, scl)
    yd = I.noise(ref.shape, 5)
    gref = O.apply_AT(w, tab, yd, scl)
    gabs = O.apply_AT(w, tab, np.abs(yd), scl)  # A^T |y|: A is entrywise nonnegative
    # the row at delay 8 + 1e-9 has hat fractions in (0, 2^-24): the case the
    # 24-bit coordinate floors to zero
    assert np.any((gabs > 0) & (gabs < 2.0 ** -24 * gabs.max()))
    for dt, tol in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
        y = op.apply_A(torch.from_numpy(x).to(dt).cuda()).cpu().double().numpy()
        g = op.apply_AT(torch.from_numpy(yd).to(dt).cuda()).cpu().double().numpy()
        assert np.max(np.abs(y - ref)) <= tol * np.max(np.abs(ref)), dt
        assert np.max(np.abs(g - gref)) <= tol * np.max(np.abs(gref)), dt
        assert np.array_equal(y == 0.0, ref == 0.0), dt  # exact hat supports
        if dt == torch.float64:
            assert np.array_equal(g == 0.0, gref == 0.0)
            # the FP64 pair are exact transposes on this table
            xd = torch.from_numpy(x).cuda()
            yy = torch.from_numpy(yd).cuda()
            lhs = float(torch.sum(op.apply_A(xd) * yy))
            rhs = float(torch.sum(xd * op.apply_AT(yy)))
            assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
        else:
            assert np.all(g[gref == 0.0] == 0.0)
            only32 = (g == 0.0) & (gref != 0.0)
            # such an output sums only hat weights below 2^-24, so it lies below
            # 2^-24 of the output scale: FP32 cannot hold it next to the rest
            assert np.all(np.abs(gref[only32]) <= 2.0 ** -24 * gabs.max())
    assert op.status(clear=True) == 0
    op.close()
