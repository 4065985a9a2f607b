"""The seeded input generator follows SplitMix64's published definition."""
import numpy as np

from paper_1709_00178_gb300.synth import splitmix64_words, synth_bytes


def _splitmix64_scalar(state):
    # Steele, Lea, Flood (OOPSLA 2014): advance by gamma, then the mix function.
    M = (1 << 64) - 1
    state = (state + 0x9E3779B97F4A7C15) & M
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
    return z ^ (z >> 31), state


def test_published_first_output():
    # The first output of SplitMix64 seeded with 1234567 is 6457827717110365317.
    assert int(splitmix64_words(1234567, 0, 1)[0]) == 6457827717110365317


def test_counter_mode_matches_sequential():
    s = 0x5059524954
    seq = []
    st = s
    for _ in range(50):
        v, st = _splitmix64_scalar(st)
        seq.append(v)
    assert splitmix64_words(s, 0, 50).tolist() == seq
    assert splitmix64_words(s, 17, 20).tolist() == seq[17:37]


def test_byte_ranges_are_consistent():
    full = synth_bytes(9, 0, 1000)
    for off, n in [(0, 1), (3, 17), (8, 8), (999, 1), (5, 995)]:
        assert np.array_equal(synth_bytes(9, off, n), full[off:off + n])
