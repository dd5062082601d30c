"""GPU parity of the forward operator A and its adjoint A^T against the FP64
oracle, through the C ABI (librtt.so).  The oracle's raw ray table is fed to
both sides, so the comparison isolates the kernels.

Tolerance (FP32 path): relative L2 error <= 1e-5 over the output and an
elementwise bound |gpu - ref| <= 1e-4 * max|ref| (ten times the L2 bound: a
few outputs sum many rays); FP64 path: 1e-12 and 1e-11 * max|ref|.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2609_05528_b300 import build, rtt
from paper_2609_05528_b300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL32 = 1e-5
TOL64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    rtt.lib()


def _optable(tab: O.Table) -> dict:
    return {"order": tab.order, "pixel": tab.pixel, "r": tab.r, "phi": tab.phi,
            "delay": tab.delay, "weight": tab.weight, "throughput": tab.throughput}


def _cmp(got: np.ndarray, ref: np.ndarray, tol: float):
    assert got.shape == ref.shape
    err = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300)
    assert err <= tol, f"relative L2 error {err:.3e} > {tol}"
    amax = np.max(np.abs(ref)) if ref.size else 0.0
    assert np.max(np.abs(got - ref), initial=0.0) <= tol * max(amax, 1e-300) * 10


class Case:
    def __init__(self, w, seeds_x=(1, 2, 3)):
        self.w = w
        self.tab = O.build_table(w, I.screen_samples(w))
        self.op = rtt.Operator(w, _optable(self.tab))
        self.scale = O.scale(self.tab)


@pytest.fixture(scope="module")
def small():
    # several warps / chunks on every axis plus ragged tails
    return Case(I.small_kerr(spin=0.5, incl_deg=50.0, nx=48, n_r=12, n_phi=24, n_frames=300,
                             n_hats=80, ss=2))


@pytest.fixture(scope="module")
def schw():
    return Case(I.schw32())


def _arm_orders(mask):
    return tuple(n for n in range(3) if mask & (1 << n))


def test_scale_and_rows_match_oracle(small):
    c = small
    assert c.op.s_ref == pytest.approx(O.s_ref(c.tab), rel=1e-13)
    assert c.op.info.n_rows == c.tab.n_rows
    for n in range(3):
        assert c.op.info.rows_per_order[n] == c.tab.rows_of_order(n)


@pytest.mark.parametrize("B", [1, 3, 8, 33])
@pytest.mark.parametrize("mask", [1, 7, 6, 5])
def test_forward_parity(small, B, mask):
    c = small
    x = I.history_batch(c.w, range(10, 10 + B)) + 0.1 * I.uniform_batch(c.w, range(50, 50 + B))
    sub = c.tab.select(_arm_orders(mask))
    ref = O.apply_A(c.w, sub, x, c.scale)
    xt = torch.from_numpy(x.astype(np.float32)).cuda()
    y = c.op.apply_A(xt, arm_mask=mask)
    torch.cuda.synchronize()
    _cmp(y.cpu().numpy().astype(np.float64), ref, TOL32)
    y64 = c.op.apply_A(torch.from_numpy(x).cuda(), arm_mask=mask)
    _cmp(y64.cpu().numpy(), ref, TOL64)


@pytest.mark.parametrize("B", [1, 8, 33])
@pytest.mark.parametrize("mask", [1, 7, 6])
def test_adjoint_parity(small, B, mask):
    c = small
    sub = c.tab.select(_arm_orders(mask))
    y = I.noise((sub.n_rows, c.w.time.n_frames, B), 77 + B)
    ref = O.apply_AT(c.w, sub, y, c.scale)
    x = c.op.apply_AT(torch.from_numpy(y.astype(np.float32)).cuda(), arm_mask=mask)
    _cmp(x.cpu().numpy().astype(np.float64), ref, TOL32)
    x64 = c.op.apply_AT(torch.from_numpy(y).cuda(), arm_mask=mask)
    _cmp(x64.cpu().numpy(), ref, TOL64)


@pytest.mark.parametrize("cadence", [0.5, 2.0, 3.0, 4.0])
@pytest.mark.parametrize("B", [2, 4, 8])
def test_cadence_variants(cadence, B):
    """Frame steps of 1/8, 1/2, 3/4 and 1 hat step: the periodic-weight adjoint
    (integer frames per hat step 8 and 2), the general kernel (3/4) and one
    frame per hat step, against the oracle."""
    n_frames = int(round(120 / cadence))
    w = I.Workload(f"cad{cadence:g}", I.Geometry(0.5, 50.0, 32), I.SourceGrid(10, 20),
                   I.TimeGrid(n_frames, cadence, 40, t_end=cadence * (n_frames - 1)),
                   supersample=2)
    c = Case(w)
    x = I.uniform_batch(w, range(B))
    _cmp(c.op.apply_A(torch.from_numpy(x.astype(np.float32)).cuda()).cpu().numpy().astype(np.float64),
         O.apply_A(w, c.tab, x, c.scale), TOL32)
    y = I.noise((c.tab.n_rows, n_frames, B), 17)
    ref = O.apply_AT(w, c.tab, y, c.scale)
    got = c.op.apply_AT(torch.from_numpy(y.astype(np.float32)).cuda())
    _cmp(got.cpu().numpy().astype(np.float64), ref, TOL32)
    _cmp(c.op.apply_AT(torch.from_numpy(y).cuda()).cpu().numpy(), ref, TOL64)


def test_dot_product_fp64(small):
    c = small
    x = torch.from_numpy(I.uniform_batch(c.w, [3, 4])).cuda()
    y = torch.from_numpy(I.noise((c.tab.n_rows, c.w.time.n_frames, 2), 5)).cuda()
    lhs = torch.sum(c.op.apply_A(x) * y).item()
    rhs = torch.sum(x * c.op.apply_AT(y)).item()
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_deterministic_bitwise(small):
    c = small
    x = torch.from_numpy(I.uniform_batch(c.w, range(8)).astype(np.float32)).cuda()
    y1 = c.op.apply_A(x)
    y2 = c.op.apply_A(x)
    assert torch.equal(y1, y2)
    g1 = c.op.apply_AT(y1)
    g2 = c.op.apply_AT(y2)
    assert torch.equal(g1, g2)


def test_batch_columns_independent_bitwise(small):
    """Each batch column of A x and A^T y is the same bits whatever the batch
    size (B = 8 takes the 16-byte vector kernels, B = 1 and B = 3 the scalar
    ones): every kernel variant sums in the same order."""
    c = small
    x = torch.from_numpy(I.uniform_batch(c.w, range(8)).astype(np.float32)).cuda()
    y = c.op.apply_A(x)
    g = c.op.apply_AT(y)
    for j in (0, 5):
        yj = c.op.apply_A(x[:, :, j:j + 1].contiguous())
        assert torch.equal(yj[:, :, 0], y[:, :, j])
        gj = c.op.apply_AT(y[:, :, j:j + 1].contiguous())
        assert torch.equal(gj[:, :, 0], g[:, :, j])
    y3 = c.op.apply_A(x[:, :, 2:5].contiguous())
    assert torch.equal(y3, y[:, :, 2:5])
    g3 = c.op.apply_AT(y[:, :, 2:5].contiguous())
    assert torch.equal(g3, g[:, :, 2:5])


@pytest.mark.parametrize("B", [3, 8])
def test_autotune_keeps_bits(B):
    """rtt_autotune times the kernel variants and installs the fastest; the
    outputs after tuning are the same bits as before."""
    w = I.small_kerr(spin=0.5, incl_deg=50.0, nx=40, n_r=10, n_phi=20, n_frames=200,
                     n_hats=60, ss=2)
    c = Case(w)
    x = torch.from_numpy(I.uniform_batch(w, range(B)).astype(np.float32)).cuda()
    y0 = c.op.apply_A(x)
    g0 = c.op.apply_AT(y0)
    r = c.op.autotune(B)
    assert r["batch"] == B and r["candidates"] >= 4
    assert r["fwd_kernel"] in range(1, 10) and r["adj_kernel"] in (1, 2, 3, 4)
    if B % 4:
        assert r["adj_kernel"] <= 2  # the TMA adjoint needs 16-byte frame records
    assert 0 < r["fwd_ms"] <= r["fwd_ms_rule"] and 0 < r["adj_ms"] <= r["adj_ms_rule"]
    y1 = c.op.apply_A(x)
    g1 = c.op.apply_AT(y0)
    assert torch.equal(y0, y1) and torch.equal(g0, g1)
    _cmp(y1.cpu().numpy().astype(np.float64),
         O.apply_A(w, c.tab, x.cpu().numpy().astype(np.float64), c.scale), TOL32)


@pytest.mark.parametrize("which", ["small", "schw"])
@pytest.mark.parametrize("B", [1, 2, 3, 4, 8, 16])
def test_every_variant_same_bits(which, small, schw, B):
    """Every kernel variant (rtt_set_variant) of the FP32 forward and adjoint
    gives the same bits as the default rule, which matches the oracle; the
    TMA-staged adjoint's bounded waits never time out (status word 0)."""
    c = small if which == "small" else schw
    x = torch.from_numpy(I.uniform_batch(c.w, range(B)).astype(np.float32)).cuda()
    c.op.set_variant(B)  # default rule
    y0 = c.op.apply_A(x)
    g0 = c.op.apply_AT(y0)
    _cmp(y0.cpu().numpy().astype(np.float64),
         O.apply_A(c.w, c.tab, x.cpu().numpy().astype(np.float64), c.scale), TOL32)
    _cmp(g0.cpu().numpy().astype(np.float64),
         O.apply_AT(c.w, c.tab, y0.cpu().numpy().astype(np.float64), c.scale), TOL32)
    bc_max = 1
    while bc_max < min(B, 32):
        bc_max *= 2
    n = 0
    for fk in (1, 2, 3, 4, 5, 6, 7, 8, 9):
        for bc in sorted({bc_max, max(1, bc_max // 2), max(1, bc_max // 4)}):
            for half in (0, 1):
                for su in ((1, 2, 3) if (fk == 1 and half == 0 and bc in (4, 8)) else (2,)):
                    for order in (0, 1):  # task rows in (order, pixel) or source-cell order
                        c.op.set_variant(B, fk, bc, half, 1, fwd_staging=su, fwd_order=order)
                        assert torch.equal(c.op.apply_A(x), y0), (fk, bc, half, su, order)
                        n += 1
    for ak in (1, 2, 3, 4):
        c.op.set_variant(B, 1, bc_max, 0, ak)
        assert torch.equal(c.op.apply_AT(y0), g0), ak
        n += 1
    # direct arm only: rays of the other orders are skipped by every adjoint kernel
    c.op.set_variant(B)
    y1 = c.op.apply_A(x, arm_mask=1)
    g1 = c.op.apply_AT(y1, arm_mask=1)
    for ak in (1, 2, 3, 4):
        c.op.set_variant(B, 1, bc_max, 0, ak)
        assert torch.equal(c.op.apply_AT(y1, arm_mask=1), g1), ak
    for fk in (1, 3, 4, 5, 7, 9):
        for order in (0, 1):
            c.op.set_variant(B, fk, bc_max, 0, 1, fwd_order=order)
            assert torch.equal(c.op.apply_A(x, arm_mask=1), y1), (fk, order)
    # column passes: the periodic forward and the adjoint over a few columns at a time
    if B % 8 == 0 and B > 8:
        c.op.set_variant(B, 5, 8, 0, 2, fwd_cols=8)
        assert torch.equal(c.op.apply_A(x), y0)
        for ak in (1, 2):
            for pc in (4, 8):
                c.op.set_variant(B, 5, 8, 0, ak, adj_cols=pc)
                assert torch.equal(c.op.apply_AT(y0), g0), (ak, pc)
    # rings only (an arm that starts after the direct block)
    c.op.set_variant(B)
    y6 = c.op.apply_A(x, arm_mask=6)
    for order in (0, 1):
        c.op.set_variant(B, 1, bc_max, 0, 1, fwd_order=order)
        assert torch.equal(c.op.apply_A(x, arm_mask=6), y6), order
    c.op.set_variant(B)
    assert c.op.status(clear=True) == 0
    assert n >= 12


@pytest.mark.parametrize("which", ["small", "schw"])
@pytest.mark.parametrize("B", [4, 8, 16, 32, 64])
def test_quad_lane_forward_same_bits(which, small, schw, B):
    """The quad-lane forward (kernels 7 and 8: B/4 lanes share a frame, each
    holding 4 of its columns) at every chunk width from 4 to 64 columns and
    both frame counts per lane gives the bits of the staged kernel, which
    matches the oracle: ragged frame chunks (300 frames), hat windows past
    either end of the hats, cadences of 1/4 (small) and 1/2 (schw) hat step,
    every arm."""
    c = small if which == "small" else schw
    x = torch.from_numpy(I.uniform_batch(c.w, range(B)).astype(np.float32)).cuda()
    qbc = 64
    while B % qbc:
        qbc //= 2
    for mask in (7, 1, 6):
        c.op.set_variant(B, 1, min(B, 32), 0, 1)
        y0 = c.op.apply_A(x, arm_mask=mask)
        if B in (8, 64):
            sub = c.tab.select(_arm_orders(mask))
            _cmp(y0.cpu().numpy().astype(np.float64),
                 O.apply_A(c.w, sub, x.cpu().numpy().astype(np.float64), c.scale), TOL32)
        for fk in (7, 8, 9):
            for bc in (qbc, qbc // 2, qbc // 4):
                if bc < 4:
                    continue
                for half in (0, 1):
                    for order in (0, 1):
                        c.op.set_variant(B, fk, bc, half, 1, fwd_order=order)
                        assert torch.equal(c.op.apply_A(x, arm_mask=mask), y0), (mask, fk, bc, half, order)
    c.op.set_variant(B)
    assert c.op.get_variant(B)["fwd_kernel"] == 7 and c.op.get_variant(B)["fwd_bc"] == min(qbc, 32)
    assert c.op.status(clear=True) == 0


@pytest.fixture(scope="module")
def eighth():
    """small_kerr with a frame step of 1/8 hat step (the periodic kernels' P = 8)."""
    import dataclasses
    w = I.small_kerr(spin=0.5, incl_deg=50.0, nx=40, n_r=10, n_phi=20, n_frames=300, n_hats=40, ss=2)
    w = dataclasses.replace(w, time=I.TimeGrid(300, 0.5, 40, t_end=149.5))
    return Case(w)


@pytest.mark.parametrize("B", [1, 2, 4, 8, 16, 32])
def test_periodic_kernels_at_eighth_hat_step(eighth, B):
    """P = 8 frames per hat step: every periodic forward (5-8) and adjoint
    (2-4) kernel, including the TMA adjoint of 4 columns, which needs P = 8,
    and the 32-column-pass adjoint, gives the staged and general kernels'
    bits, which match the oracle."""
    c = eighth
    assert c.w.time.hat_step / c.w.time.cadence == 8.0
    x = torch.from_numpy(I.uniform_batch(c.w, range(B)).astype(np.float32)).cuda()
    c.op.set_variant(B, 1, min(B, 32), 0, 1)
    y0 = c.op.apply_A(x)
    g0 = c.op.apply_AT(y0)
    if B == 8:
        _cmp(y0.cpu().numpy().astype(np.float64),
             O.apply_A(c.w, c.tab, x.cpu().numpy().astype(np.float64), c.scale), TOL32)
        _cmp(g0.cpu().numpy().astype(np.float64),
             O.apply_AT(c.w, c.tab, y0.cpu().numpy().astype(np.float64), c.scale), TOL32)
    for fk in (5, 6, 7, 8, 9):
        for half in (0, 1):
            c.op.set_variant(B, fk, min(B, 16 if fk < 7 else 32), half, 1)
            assert torch.equal(c.op.apply_A(x), y0), (fk, half)
    for ak in (2, 3, 4):
        c.op.set_variant(B, 1, min(B, 32), 0, ak)
        assert torch.equal(c.op.apply_AT(y0), g0), ak
    c.op.set_variant(B)
    assert c.op.status(clear=True) == 0


@pytest.mark.parametrize("which", ["small", "schw"])
@pytest.mark.parametrize("B", [32, 64])
def test_adjoint_32_column_passes_same_bits(which, small, schw, B):
    """The adjoint at batches of whole 32-column passes: the TMA kernel of
    32-column passes (adjoint kernels 3 and 4; two lanes per hat) gives the
    bits of the general and periodic kernels, which match the oracle, on
    every arm, with 1/4 (small) and 1/2 (schw) hat-step cadences and the
    records of narrower passes."""
    c = small if which == "small" else schw
    for mask in (7, 1, 6):
        d = torch.from_numpy(I.noise((c.op.arm_rows(mask), c.w.time.n_frames, B), 31 + B).astype(np.float32)).cuda()
        c.op.set_variant(B, 1, 32, 0, 1)
        g0 = c.op.apply_AT(d, arm_mask=mask)
        if B == 32:
            sub = c.tab.select(_arm_orders(mask))
            _cmp(g0.cpu().numpy().astype(np.float64),
                 O.apply_AT(c.w, sub, d.cpu().numpy().astype(np.float64), c.scale), TOL32)
        for ak in (2, 3, 4):
            c.op.set_variant(B, 1, 32, 0, ak)
            assert torch.equal(c.op.apply_AT(d, arm_mask=mask), g0), (mask, ak)
        c.op.set_variant(B, 1, 32, 0, 4, adj_cols=16)
        assert torch.equal(c.op.apply_AT(d, arm_mask=mask), g0), (mask, "16-column passes")
    c.op.set_variant(B)
    assert c.op.get_variant(B)["adj_kernel"] == 4
    assert c.op.status(clear=True) == 0


@pytest.mark.parametrize("which", ["small", "schw"])
@pytest.mark.parametrize("B", [3, 4, 8])
@pytest.mark.parametrize("mask", [7, 1])
@pytest.mark.parametrize("with_d", [False, True])
def test_apply_A_AT(which, small, schw, B, mask, with_d):
    """rtt_apply_A_AT gives the bits of rtt_apply_A followed by rtt_apply_AT
    on y - d, with every adjoint kernel, and matches the oracle."""
    c = small if which == "small" else schw
    x = torch.from_numpy(I.uniform_batch(c.w, range(B)).astype(np.float32)).cuda()
    y_ref = c.op.apply_A(x, arm_mask=mask)
    d = None
    r = y_ref
    if with_d:
        d = torch.from_numpy(I.noise(tuple(y_ref.shape), 23).astype(np.float32)).cuda()
        r = (y_ref - d).contiguous()
    g_ref = c.op.apply_AT(r, arm_mask=mask)
    bc = 1
    while bc < B:
        bc *= 2
    for ak in (1, 2, 3, 4):
        c.op.set_variant(B, 1, bc, 0, ak)
        y, g = c.op.apply_A_AT(x, d, arm_mask=mask)
        assert torch.equal(y, y_ref), ak
        assert torch.equal(g, g_ref), ak
    c.op.set_variant(B)
    sub = c.tab.select(_arm_orders(mask))
    _cmp(g.cpu().numpy().astype(np.float64),
         O.apply_AT(c.w, sub, r.cpu().numpy().astype(np.float64), c.scale), TOL32)
    assert c.op.status(clear=True) == 0


def test_direct_zero_columns_bit_exact(schw):
    """Theorem 4.1: columns the oracle finds exactly zero in the direct block
    are exactly zero on the GPU (FP32 and FP64 paths), and vice versa."""
    c = schw
    n = c.w.n_dof
    D0 = O.dense_A(c.w, c.tab.select((0,)), c.scale)
    ref_zero = np.all(D0 == 0.0, axis=0)
    assert ref_zero.sum() > 0
    E = torch.eye(n, dtype=torch.float64).reshape(c.w.grid.n_nodes, c.w.time.n_hats, n).cuda()
    for dt in (torch.float32, torch.float64):
        M = c.op.apply_A(E.to(dt).contiguous(), arm_mask=1).reshape(-1, n).cpu().numpy()
        gpu_zero = np.all(M == 0.0, axis=0)
        assert np.array_equal(gpu_zero, ref_zero)
        _cmp(M.astype(np.float64), D0, TOL32 if dt == torch.float32 else TOL64)


def test_empty_arm_and_errors(schw):
    c = schw
    assert c.op.arm_rows(4) == 0  # no n=2 rows at 32x32
    x = torch.ones((c.w.grid.n_nodes, c.w.time.n_hats, 2), device="cuda")
    y = c.op.apply_A(x, arm_mask=4)
    assert y.shape[0] == 0
    g = c.op.apply_AT(y, arm_mask=4)
    assert torch.count_nonzero(g).item() == 0
    with pytest.raises(rtt.RttError):
        c.op._launch("rtt_apply_A", x, x, 0, 7, None)
    with pytest.raises(rtt.RttError):
        c.op._launch("rtt_apply_A", x, x, 2, 0, None)


def test_autograd_backward_is_adjoint_and_matches_fd(small):
    """forward A / backward A^T as a torch.autograd.Function; the gradient of
    L(x) = 1/2 ||A x - d||^2 matches the oracle's A^T (A x - d) and central
    finite differences in FP64 (step 1e-3)."""
    c = small
    B = 2
    xt = I.history_batch(c.w, [21, 22])
    d = O.apply_A(c.w, c.tab, xt, c.scale) + I.noise((c.tab.n_rows, c.w.time.n_frames, B), 23)
    x0 = I.history_batch(c.w, [31, 32])
    x = torch.from_numpy(x0.astype(np.float32)).cuda().requires_grad_(True)
    yd = torch.from_numpy(d.astype(np.float32)).cuda()
    loss = 0.5 * torch.sum((rtt.apply_A_autograd(x, c.op) - yd) ** 2)
    loss.backward()
    g = x.grad.cpu().numpy().astype(np.float64)
    ref = O.apply_AT(c.w, c.tab, O.apply_A(c.w, c.tab, x0, c.scale) - d, c.scale)
    err = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    assert err < 1e-4  # FP32 residual of a large data vector
    h = 1e-3
    for k in range(4):
        v = I.noise(x0.shape, 100 + k)
        Lp = 0.5 * np.sum((O.apply_A(c.w, c.tab, x0 + h * v, c.scale) - d) ** 2)
        Lm = 0.5 * np.sum((O.apply_A(c.w, c.tab, x0 - h * v, c.scale) - d) ** 2)
        fd = (Lp - Lm) / (2 * h)
        assert np.sum(g * v) == pytest.approx(fd, rel=1e-4)


def test_gpu_tracer_matches_oracle():
    """rtt_trace_rays (RK4 on the GPU) vs the oracle's DP5 integrator: the same
    valid (order, pixel) entries, and per entry r, phi, delay and weight."""
    w = I.small_kerr(spin=0.94, incl_deg=75.0, nx=64, ss=2)
    s = I.screen_samples(w)
    ref = O.build_table(w, s)
    got = rtt.rtt_trace_rays(w.geometry.spin, w.geometry.incl_deg, w.grid, s)
    # rays whose radius sits within 1e-6 M of r_in / r_out may flip validity
    edge = (np.abs(ref.r - w.grid.r_in) < 1e-6) | (np.abs(ref.r - w.grid.r_out) < 1e-6)
    assert abs(len(got["r"]) - ref.n_rays) <= int(edge.sum()) + 2
    groups = {}
    for i, key in enumerate(zip(ref.order.tolist(), ref.pixel.tolist())):
        groups.setdefault(key, []).append(i)
    n_match = 0
    dr = dphi = ddel = dw = 0.0
    for j, key in enumerate(zip(got["order"].tolist(), got["pixel"].tolist())):
        cand = groups.get(key)
        if not cand:
            continue
        # nearest oracle sub-ray of the same (order, pixel)
        dist = [abs(ref.r[i] - got["r"][j]) + abs(np.angle(np.exp(1j * (ref.phi[i] - got["phi"][j]))))
                for i in cand]
        i = cand[int(np.argmin(dist))]
        if min(dist) > 1e-4:
            continue  # a sub-ray valid on one side only (radius at a grid edge)
        n_match += 1
        dr = max(dr, abs(ref.r[i] - got["r"][j]))
        dphi = max(dphi, abs(np.angle(np.exp(1j * (ref.phi[i] - got["phi"][j])))))
        ddel = max(ddel, abs(ref.delay[i] - got["delay"][j]))
        dw = max(dw, abs(ref.weight[i] / got["weight"][j] - 1.0))
    assert n_match >= ref.n_rays - int(edge.sum()) - 2
    # the table oracle traces at rtol 1e-13 (its phi is good to ~1e-9 there);
    # the tight bounds are in the two tests below
    assert dr < 1e-9 and dphi < 2e-9 and ddel < 1e-8 and dw < 1e-9, (dr, dphi, ddel, dw)


def _trace_errors(w, ref):
    """Largest |r| and |phi| differences per order between rtt_trace_rays and
    a reference trace of the same screen samples (each GPU entry matched to
    the nearest sample of its pixel with that order)."""
    s = I.screen_samples(w)
    got = rtt.rtt_trace_rays(w.geometry.spin, w.geometry.incl_deg, w.grid, s)
    out = {}
    for o in range(3):
        dr = dphi = 0.0
        n = 0
        for j in np.nonzero(got["order"] == o)[0]:
            cand = np.nonzero((s.pixel == got["pixel"][j]) & ref.found[:, o])[0]
            if cand.size == 0:
                continue
            d = np.abs(ref.r[cand, o] - got["r"][j]) + \
                np.abs(np.angle(np.exp(1j * (ref.phi[cand, o] - got["phi"][j]))))
            if d.min() > 1e-6:
                continue
            k = cand[int(np.argmin(d))]
            n += 1
            dr = max(dr, abs(ref.r[k, o] - got["r"][j]))
            dphi = max(dphi, abs(np.angle(np.exp(1j * (ref.phi[k, o] - got["phi"][j])))))
        out[o] = (n, dr, dphi)
    return out


def test_gpu_tracer_against_exact_schwarzschild():
    """At a = 0 the oracle's orbit integral is exact (elliptic integrals): the
    GPU's Mino-time integration reaches r and phi to 1e-10 for every order."""
    w = I.schw32()
    s = I.screen_samples(w)
    ref = O.trace(0.0, w.geometry.incl, s.alpha, s.beta, method="schw", r_esc=w.grid.r_out)
    for o, (n, dr, dphi) in _trace_errors(w, ref).items():
        assert dr <= 1e-10 and dphi <= 1e-10, (o, n, dr, dphi)
    assert _trace_errors(w, ref)[0][0] > 500


@pytest.mark.parametrize("a,incl", [(0.94, 75.0), (0.5, 50.0)])
def test_gpu_tracer_against_oracle_kerr(a, incl):
    """Kerr rays against the oracle's DP5 Carter integration at rtol 1e-15:
    r to 1e-10; phi to 5e-10, the oracle's own reproducibility in phi (its
    runs at rtol 1e-15 and 2e-16 differ by up to 2.5e-10)."""
    w = I.small_kerr(spin=a, incl_deg=incl, nx=64, ss=2)
    s = I.screen_samples(w)
    ref = O.trace(a, w.geometry.incl, s.alpha, s.beta, method="kerr", r_esc=w.grid.r_out,
                  rtol=1e-15)
    res = _trace_errors(w, ref)
    for o, (n, dr, dphi) in res.items():
        assert dr <= 1e-10 and dphi <= 5e-10, (o, n, dr, dphi)
    assert res[0][0] > 1000 and res[1][0] > 100 and res[2][0] > 10


@pytest.mark.parametrize("kind", ["S224", "L224"])
def test_forward_class_batch_224(schw, kind):
    """P = scale A Q for a 224-column class as one batch (7 batch chunks)."""
    c = schw
    Q = O.synth_class(c.w, kind)
    x = Q.reshape(c.w.grid.n_nodes, c.w.time.n_hats, -1)
    for mask, orders in ((1, (0,)), (7, (0, 1, 2))):
        ref = O.restricted_response(c.w, c.tab.select(orders), Q, c.scale)
        got = c.op.apply_A(torch.from_numpy(x.copy()).cuda(), arm_mask=mask).cpu().numpy()
        got = got.reshape(ref.shape)
        bad = np.argwhere(np.abs(got - ref) > 1e-12 * np.abs(ref).max())
        assert bad.shape[0] == 0, (bad[:5].tolist(), got[tuple(bad[0])], ref[tuple(bad[0])])
        g32 = c.op.apply_A(torch.from_numpy(x.astype(np.float32)).cuda(), arm_mask=mask)
        _cmp(g32.cpu().numpy().astype(np.float64).reshape(ref.shape), ref, TOL32)
