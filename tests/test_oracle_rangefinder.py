"""Pins of the oracle's randomized range finder (the spectrum of the
restricted normal operator from Gaussian blocks, Sec. 7-8):

  * with blocks until the basis spans the space, the Ritz values are the
    eigenvalues (numpy eigvalsh) to FP64 accuracy (operators whose eigenvalues
    span less than the 1e-12 pivot tolerance of a block, relative);
  * on an operator of rank r <= block, one block finds its r non-zero
    eigenvalues (the range of G Omega is the range of G), each to about
    eps * lambda_max;
  * on any basis the Ritz values interlace: the i-th largest never exceeds
    the i-th largest eigenvalue (Cauchy), and the rank read from them never
    exceeds the operational rank.
"""
import numpy as np

import oracle as O


def _spd(d, rank, seed, scale=1e6):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((d, rank)) * np.logspace(0, np.log10(scale), rank)
    return X @ X.T


def test_full_span_gives_the_eigenvalues():
    G = _spd(60, 60, 1, scale=1e4)
    om = np.random.default_rng(2).standard_normal((60, 16 * 5))
    ritz, k, used = O.range_finder(G, om, 16, rho=1e-9)
    lam = np.sort(np.linalg.eigvalsh(G))[::-1]
    assert k == 60
    np.testing.assert_allclose(ritz, lam, rtol=0, atol=1e-12 * lam[0])


def test_low_rank_in_one_block():
    G = _spd(80, 12, 3, scale=1e4)
    om = np.random.default_rng(4).standard_normal((80, 32 * 3))
    ritz, k, used = O.range_finder(G, om, 32, rho=1.0)
    lam = np.sort(np.linalg.eigvalsh(G))[::-1]
    # FP64 resolves each eigenvalue to about eps * lambda_max in absolute terms
    np.testing.assert_allclose(ritz[:12], lam[:12], rtol=1e-10, atol=1e-13 * lam[0])
    assert np.all(np.abs(ritz[12:]) <= 1e-13 * lam[0])
    assert used == 2  # the second block adds nothing above rho^2


def test_ritz_values_interlace():
    G = _spd(120, 120, 5, scale=1e9)
    lam = np.sort(np.linalg.eigvalsh(G))[::-1]
    om = np.random.default_rng(6).standard_normal((120, 20 * 2))
    ritz, k, used = O.range_finder(G, om, 20, rho=1e3)
    assert k <= 40
    assert np.all(ritz <= lam[:k] * (1 + 1e-12) + 1e-12 * lam[0])
    assert np.count_nonzero(np.sqrt(np.maximum(ritz, 0)) >= 1e3) <= \
        np.count_nonzero(np.sqrt(np.maximum(lam, 0)) >= 1e3)
