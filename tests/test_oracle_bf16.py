"""Pins of the oracle's BF16-weight mode (the GPU tables' precision option):

  * the rounding itself against the definition, brute force: the float
    nearest the value, then the nearer of the two BF16 neighbours of that
    float, ties to the even one; hand-made ties;
  * the BF16 operator is still a pair of exact transposes (dot test);
  * it differs from the FP64-weight operator by at most the rounding of each
    weight, |A_bf16 x - A x| <= 2^-8 (A |x|) elementwise (the weights are
    positive, so A |x| bounds the sum of |terms|), and it does differ.
"""
import struct

import numpy as np
import pytest

import oracle as O
from paper_2609_05528_b300 import inputs as I


def _f32(v):
    return struct.unpack("<f", struct.pack("<f", v))[0]


def _bits(f):
    return struct.unpack("<I", struct.pack("<f", f))[0]


def _from_bits(u):
    return struct.unpack("<f", struct.pack("<I", u & 0xFFFFFFFF))[0]


def _bf16_nearest(v):
    f = _f32(v)
    lo = _from_bits(_bits(f) & 0xFFFF0000)
    # lo: f truncated toward zero; hi: the next BF16 away from zero (one more
    # unit in the magnitude bits, for either sign)
    hi = _from_bits((_bits(f) & 0xFFFF0000) + 0x10000)
    dl, dh = abs(f - lo), abs(hi - f)
    if dl < dh:
        return lo
    if dh < dl:
        return hi
    return lo if ((_bits(lo) >> 16) & 1) == 0 else hi


def test_round_bf16_brute_force():
    rng = np.random.default_rng(5)
    vals = np.concatenate([rng.standard_normal(3000) * 10.0 ** rng.integers(-30, 30, 3000),
                           rng.uniform(0, 1, 2000)])
    for v in vals:
        assert O.round_bf16(v) == _bf16_nearest(float(v)), v


def test_round_bf16_ties_to_even():
    assert O.round_bf16(1.0 + 2.0 ** -8) == 1.0                    # tie, 1.0 is even
    assert O.round_bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6     # tie, rounds up to even
    assert O.round_bf16(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    assert O.round_bf16(-(1.0 + 2.0 ** -8)) == -1.0
    assert O.round_bf16(0.0) == 0.0
    for k in range(-20, 20):
        assert O.round_bf16(2.0 ** k) == 2.0 ** k


@pytest.fixture(scope="module")
def case():
    w = I.small_kerr(spin=0.5, incl_deg=50.0, nx=24, n_r=8, n_phi=12, n_frames=64, n_hats=24, ss=1)
    tab = O.build_table(w, I.screen_samples(w))
    return w, tab, O.scale(tab)


def test_bf16_operator_is_transposed_exactly(case):
    w, tab, scl = case
    x = I.uniform_batch(w, [1, 2])
    y = I.noise((tab.n_rows, w.time.n_frames, 2), 3)
    lhs = np.sum(O.apply_A(w, tab, x, scl, bf16=True) * y)
    rhs = np.sum(x * O.apply_AT(w, tab, y, scl, bf16=True))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_bf16_weights_within_their_rounding(case):
    w, tab, scl = case
    x = I.uniform_batch(w, [4]) - 0.5
    y64 = O.apply_A(w, tab, x, scl)
    y16 = O.apply_A(w, tab, x, scl, bf16=True)
    bound = O.apply_A(w, tab, np.abs(x), scl)
    assert np.all(np.abs(y16 - y64) <= 2.0 ** -8 * bound + 1e-300)
    assert np.max(np.abs(y16 - y64)) > 0.0
    d = I.noise((tab.n_rows, w.time.n_frames, 1), 9)
    g64 = O.apply_AT(w, tab, d, scl)
    g16 = O.apply_AT(w, tab, d, scl, bf16=True)
    gb = O.apply_AT(w, tab, np.abs(d), scl)
    assert np.all(np.abs(g16 - g64) <= 2.0 ** -8 * gb + 1e-300)
