"""rtt_gemm_tn_f64, the tensor-core FP64 contraction C = A^T B (digit
splitting onto BF16 tcgen05.mma with exact FP32 windows and integer
accumulation), against the definition:

  * inputs with at most 20 significant bits per entry (any column scales):
    every product and every partial sum is exact in FP64, so numpy's A^T B is
    exact, and so must the tensor-core result be (the 7 x 7-bit digits hold
    every entry exactly);
  * random FP64 inputs with column scales spread over 2^+-200: within
    2^-44 of sum_k |A_ki| |B_kj| (the 49-bit digit truncation), and the
    result is bitwise repeatable;
  * ragged sizes (k, m, n not multiples of the tiles), zero columns."""
import numpy as np
import pytest

from paper_2609_05528_b300 import build, rtt

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    rtt.lib()


def _cols(rng, k, m, lo, hi):
    return 2.0 ** rng.integers(lo, hi, size=m)


@pytest.mark.parametrize("k,m,n", [(300, 5, 7), (4096, 224, 96), (1000, 130, 65)])
def test_exact_on_short_inputs(k, m, n):
    rng = np.random.default_rng(k + m + n)
    A = rng.integers(-(1 << 20), 1 << 20, size=(k, m)).astype(np.float64) * _cols(rng, k, m, -60, 60)
    B = rng.integers(-(1 << 20), 1 << 20, size=(k, n)).astype(np.float64) * _cols(rng, k, n, -60, 60)
    A[:, 1] = 0.0  # a zero column
    ref = A.T @ B  # exact: 40-bit products, sums below 2^53 relative to the column scales
    got = rtt.gemm_tn(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()).cpu().numpy()
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("k,m,n", [(20000, 224, 224), (777, 33, 17)])
def test_fp64_accuracy_and_repeatability(k, m, n):
    rng = np.random.default_rng(7 + k)
    A = rng.standard_normal((k, m)) * _cols(rng, k, m, -200, 200)
    B = rng.standard_normal((k, n)) * _cols(rng, k, n, -200, 200)
    At, Bt = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    got = rtt.gemm_tn(At, Bt)
    again = rtt.gemm_tn(At, Bt)
    assert torch.equal(got, again)
    ref = A.T @ B
    bound = np.abs(A).T @ np.abs(B)
    err = np.abs(got.cpu().numpy() - ref)
    assert np.all(err <= 2.0 ** -44 * bound + 1e-300), float(np.max(err / bound))
