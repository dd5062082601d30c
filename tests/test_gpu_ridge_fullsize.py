"""Ridge recovery at the full recovery size (Sec. 9: Kerr a = 0.94, i = 50 deg,
kerr256 sizes) against the FP64 oracle.  The ridge solution of
(A^T A + lambda I) x = A^T d is unique; the oracle checks the GPU's solution
by its own FP64 applies at full size: the normal-equation residual
||A^T d - (A^T A + lambda I) x|| / ||A^T d|| must be at the solver's
tolerance (an FP64 CG run of the oracle to that tolerance at this size
would take hours on the host).  Four histories of the held-out set, the
validation-selected lambda = 10 and a larger one."""
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
    rtt.lib()


def test_ridge_at_full_size_solves_the_normal_equations():
    w = I.recovery()
    tab = O.build_table(w, I.screen_samples(w))
    scl = O.scale(tab)
    op = rtt.Operator(w, {"order": tab.order, "pixel": tab.pixel, "r": tab.r, "phi": tab.phi,
                          "delay": tab.delay, "weight": tab.weight,
                          "throughput": tab.throughput})
    xt = I.recovery_batch(w, range(1000, 1004))
    d = O.apply_A(w, tab, xt, scl) + I.noise((tab.n_rows, w.time.n_frames, 4), 11)
    lams = [10.0, 1000.0]
    tol = 1e-6
    x, iters, rel = rtt.solve_ridge(op, torch.from_numpy(d.astype(np.float32)).cuda(), lams,
                                    max_iter=2000, tol=tol, refresh_every=25)
    assert np.all(rel <= tol), (iters, rel)
    xg = x.cpu().numpy().astype(np.float64)
    atd = O.apply_AT(w, tab, d, scl)
    for j in range(4):
        for l, lam in enumerate(lams):
            xs = xg[:, :, j * len(lams) + l]
            res = atd[:, :, j] - (O.apply_AT(w, tab, O.apply_A(w, tab, xs, scl), scl) + lam * xs)
            rr = np.linalg.norm(res) / np.linalg.norm(atd[:, :, j])
            # the FP32 x itself carries rounding: 2 tol allows for it
            assert rr <= 2 * tol, (j, lam, rr, iters)
    op.close()
