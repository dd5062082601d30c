"""Order mixing on the GPU (Sec. 3.1 Eq. 4) against the oracle: the unresolved
image and the total-flux readout of the whitened data, their adjoints, FP32
and FP64, every arm; the mixed arm's restricted Gram; repeatability."""
import numpy as np
import pytest

import oracle as O
from paper_2609_05528_b300 import build, rtt
from paper_2609_05528_b300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ARMS = {7: (0, 1, 2), 3: (0, 1), 1: (0,), 6: (1, 2)}
MODES = [O.MIX_UNRESOLVED, O.MIX_TOTAL_FLUX]


def _optable(tab):
    return {"order": tab.order, "pixel": tab.pixel, "r": tab.r, "phi": tab.phi,
            "delay": tab.delay, "weight": tab.weight, "throughput": tab.throughput}


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


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


@pytest.fixture(scope="module")
def k256():
    w = I.kerr256()
    tab = O.build_table(w, I.screen_samples(w))
    op = rtt.Operator(w, _optable(tab))
    yield w, tab, op
    op.close()


def test_constants_match_oracle():
    assert rtt.MIX_UNRESOLVED == O.MIX_UNRESOLVED and rtt.MIX_TOTAL_FLUX == O.MIX_TOTAL_FLUX


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("mask", sorted(ARMS))
@pytest.mark.parametrize("B", [1, 3, 8])
def test_small_against_oracle(schw, mode, mask, B):
    """Every arm, odd and vector batch widths, both directions, FP32 and FP64."""
    w, tab, op = schw
    orders = ARMS[mask]
    x = I.uniform_batch(w, range(B))  # non-negative sources: data without cancellation
    y = op.apply_A(torch.from_numpy(x).cuda(), arm_mask=mask)  # FP64 data of the arm
    yl = op.mix_rows(y, mode, arm_mask=mask)
    ref = O.mix_rows(tab, y.cpu().numpy(), mode, orders)
    assert yl.shape == ref.shape == (op.mix_rows_count(mode, mask), w.time.n_frames, B)
    assert _rel(yl.cpu().numpy(), ref) <= 1e-14
    y32 = y.float().contiguous()
    yl32 = op.mix_rows(y32, mode, arm_mask=mask).cpu().numpy().astype(np.float64)
    ref32 = O.mix_rows(tab, y32.cpu().numpy().astype(np.float64), mode, orders)
    # FP32 sums: <= 3 terms per pixel; total flux over fixed blocks of rows
    assert _rel(yl32, ref32) <= (1e-6 if mode == O.MIX_UNRESOLVED else 2e-5)
    # adjoint on independent data
    z = I.noise(ref.shape, 5 + B)
    back = op.mix_rows_T(torch.from_numpy(z).cuda(), mode, arm_mask=mask).cpu().numpy()
    refb = O.mix_rows_T(tab, z, mode, orders)
    assert back.shape == (op.arm_rows(mask), w.time.n_frames, B)
    assert _rel(back, refb) <= 1e-15
    back32 = op.mix_rows_T(torch.from_numpy(z.astype(np.float32)).cuda(), mode, arm_mask=mask)
    assert _rel(back32.cpu().numpy().astype(np.float64), refb) <= 1e-6


@pytest.mark.parametrize("mode", MODES)
def test_kerr256_every_output(k256, mode):
    """The benchmark's sizes (FP32, batch 8, resolved arm): every mixed output
    and every row of the adjoint against the oracle on the same data."""
    w, tab, op = k256
    x = torch.from_numpy(I.history_batch(w, range(100, 108)).astype(np.float32)).cuda()
    y = op.apply_A(x)
    yl = op.mix_rows(y, mode).cpu().numpy().astype(np.float64)
    ref = O.mix_rows(tab, y.cpu().numpy().astype(np.float64), mode)
    assert _rel(yl, ref) <= (1e-6 if mode == O.MIX_UNRESOLVED else 2e-5)
    z = I.noise(ref.shape, 31).astype(np.float32)
    back = op.mix_rows_T(torch.from_numpy(z).cuda(), mode).cpu().numpy().astype(np.float64)
    assert _rel(back, O.mix_rows_T(tab, z.astype(np.float64), mode)) <= 1e-6
    # repeatable to the bit
    y2 = op.mix_rows(y, mode).cpu().numpy().astype(np.float64)
    assert np.array_equal(y2, yl)


@pytest.mark.parametrize("mode", MODES)
def test_mixed_gram(schw, mode):
    """rtt_gram_normal_mix = P^T W^T W P with P the oracle's scaled response on
    S224, and no eigenvalue above the resolved arm's (W^T W is a projector)."""
    w, tab, op = schw
    Qn = O.synth_class(w, "S224")
    scl = O.scale(tab)
    P = O.restricted_response(w, tab, Qn, scl)
    T, d = w.time.n_frames, P.shape[1]
    Pl = O.mix_rows(tab, P.reshape(tab.n_rows, T, d), mode).reshape(-1, d)
    Gref = Pl.T @ Pl
    Q = torch.from_numpy(np.ascontiguousarray(Qn.reshape(w.grid.n_nodes, w.time.n_hats, d))).cuda()
    G = rtt.gram_normal_mix(op, Q, mode).cpu().numpy()
    assert _rel(G, Gref) <= 1e-10
    Gr = rtt.gram(op, Q, mode=rtt.GRAM_NORMAL).cpu().numpy()
    lr, ll = np.linalg.eigvalsh(Gr), np.linalg.eigvalsh(G)
    assert np.all(ll <= lr + 1e-9 * lr.max())


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("mask", [7, 3, 1])
def test_mixed_probe_info_small(schw, mode, mask):
    """rtt_probe_info_mix against the oracle's mixed probe information on all
    64 ages, and (direct arm, unresolved) the plain probe information."""
    w, tab, op = schw
    got = rtt.probe_info_mix(op, mode, mask)
    ref = O.mix_probe_info(w, tab, O.scale(tab), mode, ARMS[mask])
    assert _rel(got, ref) <= 1e-10
    if mask == 1 and mode == O.MIX_UNRESOLVED:  # one row per pixel: no collapse
        assert _rel(got, O.probe_info(w, tab.select((0,)), O.scale(tab))) <= 1e-10


@pytest.mark.parametrize("mode", MODES)
def test_mixed_probe_info_kerr256(k256, mode):
    """The benchmark's sizes on eight ages spanning the history (the oracle
    evaluates every (ray, frame) term per age), and the mixed arm's reach and
    J_old from rtt_reach."""
    w, tab, op = k256
    ages = np.array([0.0, 20.0, 40.0, 60.0, 92.0, 128.0, 200.0, 252.0])
    got = rtt.probe_info_mix(op, mode, 7, ages)
    ref = O.mix_probe_info(w, tab, O.scale(tab), mode, (0, 1, 2), ages)
    assert _rel(got, ref) <= 1e-10
    full = rtt.probe_info_mix(op, mode, 7)
    res = rtt.probe_info(op, 7)
    # rtt_probe_info evaluates in FP32 (its old tail underflows): bound with a floor
    assert np.all(full <= res * (1 + 1e-5) + 1e-6 * res.max())
    r, passed = rtt.reach(op, full, 7, a0q=5.0)
    assert r.J_old >= 0 and passed.shape == full.shape


def test_pairing_destroyed_operator(schw):
    """The operator built from the pairing-destroyed table (delays permuted
    within each order) against the oracle on the same permuted table, and its
    probe information against the oracle's.  The library builds the table
    (rtt_arm_table), the oracle its own copy (oracle.pairing_destroyed)."""
    w, tab, _ = schw
    keys = I.uniforms(7, tab.n_rays)
    tp = O.pairing_destroyed(tab, keys)
    op = rtt.Operator(w, rtt.arm_table(_optable(tab), rtt.ARM_PAIRING_DESTROYED, keys))
    x = I.uniform_batch(w, range(3))
    scl = O.scale(tp)
    assert abs(op.scale / scl - 1.0) < 1e-12
    y = op.apply_A(torch.from_numpy(x).cuda()).cpu().numpy()
    assert _rel(y, O.apply_A(w, tp, x, scl)) <= 1e-12
    info = rtt.probe_info(op, 7)
    ref = O.probe_info(w, tp, scl)
    assert _rel(info, ref) <= 1e-5
    op.close()


def _subtable(tab, rows):
    rows = np.asarray(rows, np.int64)
    counts = tab.row_ptr[rows + 1] - tab.row_ptr[rows]
    idx = np.concatenate([np.arange(tab.row_ptr[i], tab.row_ptr[i + 1]) for i in rows])
    rp = np.zeros(rows.size + 1, np.int64)
    rp[1:] = np.cumsum(counts)
    return O.Table(tab.order[idx], tab.pixel[idx], tab.r[idx], tab.phi[idx], tab.delay[idx],
                   tab.weight[idx], tab.throughput[idx], rp, tab.row_order[rows],
                   tab.row_pixel[rows], tab.sample[idx])


@pytest.mark.parametrize("mask", [7, 1])
def test_localized_probe_small(schw, mask):
    """rtt_probe_info_local against the oracle's direct evaluation of the 28
    directions (schw32: one ray per row; a supersampled Kerr case: rows of
    up to four rays), all 64 ages, and the localized directional reach."""
    w, tab, op = schw
    got = rtt.probe_info_local(op, mask)
    ref = O.local_probe_info(w, tab, O.scale(tab), ARMS[mask])
    assert got.shape == (64, 28)
    assert _rel(got, ref) <= 1e-10
    ok = np.any(got >= 1.0, axis=1)
    assert (O.AGES[np.nonzero(ok)[0][-1]] if ok.any() else None) == O.local_reach(ref)
    wk = I.small_kerr(spin=0.5, incl_deg=50.0, nx=40, n_r=10, n_phi=20, n_frames=120, n_hats=30, ss=2)
    tk = O.build_table(wk, I.screen_samples(wk))
    assert np.max(tk.row_ptr[1:] - tk.row_ptr[:-1]) > 1
    ok_ = rtt.Operator(wk, _optable(tk))
    gk = rtt.probe_info_local(ok_, mask, O.AGES[:32])
    rk = O.local_probe_info(wk, tk, O.scale(tk), ARMS[mask], O.AGES[:32])
    assert _rel(gk, rk) <= 1e-10
    ok_.close()


def test_localized_probe_kerr256_rows(k256):
    """kerr256 rays (2x2 sub-rays, rows of up to four rays): the operator of a
    sample of 1500 rows against the oracle on the same rows, 16 ages."""
    w, tab, _ = k256
    rng = np.random.default_rng(9)
    rows = np.unique(np.concatenate([rng.integers(0, tab.n_rows, 1500),
                                     np.nonzero(tab.row_ptr[1:] - tab.row_ptr[:-1] == 4)[0][:200]]))
    sub = _subtable(tab, rows)
    op = rtt.Operator(w, _optable(sub))
    ages = O.AGES[::4]
    got = rtt.probe_info_local(op, 7, ages)
    ref = O.local_probe_info(w, sub, O.scale(sub), (0, 1, 2), ages)
    assert _rel(got, ref) <= 1e-10
    op.close()
