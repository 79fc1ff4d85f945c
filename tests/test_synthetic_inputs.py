"""The integer input generator of the full-size parity fixtures
(synthetic.int_poly): SplitMix64 as published, values in range, a pure
function of (seed, index), so the GPU test and the oracle script draw the
same words on any machine."""
import numpy as np

from paper_2506_18150_gb300 import synthetic as syn


def test_splitmix64_matches_the_published_sequence():
    # SplitMix64 seeded with 0: state advances by the golden gamma, and the
    # first outputs are 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4 (Steele et al.)
    gamma = 0x9E3779B97F4A7C15
    states = np.array([gamma, (2 * gamma) % 2**64], dtype=np.uint64)
    out = syn._splitmix64(states)
    assert int(out[0]) == 0xE220A8397B1DCDAF
    assert int(out[1]) == 0x6E789E6AA1B965F4


def test_int_poly_range_determinism_and_independence():
    a = syn.int_poly(7, 3, 1 << 12, 1 << 20)
    assert a.dtype == np.int64 and a.min() >= -(1 << 20) and a.max() <= (1 << 20)
    assert np.array_equal(a, syn.int_poly(7, 3, 1 << 12, 1 << 20))
    assert not np.array_equal(a, syn.int_poly(7, 4, 1 << 12, 1 << 20))
    assert not np.array_equal(a, syn.int_poly(8, 3, 1 << 12, 1 << 20))
    assert np.array_equal(a[:100], syn.int_poly(7, 3, 100, 1 << 20))      # a prefix of the same stream
    assert abs(a.mean()) < 3 * (1 << 20) / np.sqrt(3 * len(a))           # centred


def test_dyadic_coefficients_are_exact_binary_fractions():
    a = syn.uci_silu_spec(0).act
    b = syn.uci_silu_fixed_spec(0).act
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert abs(x - y) <= 2.0**-21 and float(y * 2**20).is_integer()
    assert syn.dyadic((0.5, -0.25, 1e-9)) == (0.5, -0.25, 0.0)
