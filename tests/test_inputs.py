"""The seeded input generators (shared by the oracle and the CUDA-path tests,
no method arithmetic): SplitMix64 against its published test vector, the
uniform and normal draws built on it, and the seeded control permutations."""
import numpy as np

from paper_2609_05528_b300 import inputs as I


def test_splitmix64_published_vector():
    """Vigna's SplitMix64 seeded with 1234567: its first five outputs."""
    assert [int(v) for v in I.splitmix64(1234567, 5)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]


def test_uniforms_and_normals():
    u = I.uniforms(7, 200_000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 3e-3 and abs(u.var() - 1.0 / 12.0) < 2e-3
    # uniforms are the top 53 bits of the raw outputs
    raw = I.splitmix64(7, 4)
    assert np.array_equal(u[:4], (raw >> np.uint64(11)).astype(np.float64) / 2.0 ** 53)
    z = I.normals(8, 200_001)
    assert z.size == 200_001 and np.all(np.isfinite(z))
    assert abs(z.mean()) < 1e-2 and abs(z.var() - 1.0) < 1e-2
    assert abs(np.mean(z ** 4) - 3.0) < 0.1  # Gaussian kurtosis
    # the same seed gives the same draws; a different seed does not
    assert np.array_equal(I.normals(8, 10), z[:10])
    assert not np.array_equal(I.normals(9, 10), z[:10])


def test_noise_shape_and_seed():
    a = I.noise((3, 4, 2), 5)
    assert a.shape == (3, 4, 2)
    assert np.array_equal(a.ravel(), I.normals(5, 24))
