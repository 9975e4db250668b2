"""The counter-based generator of the Poisson right-hand-side noise
(Philox4x32-10) against known-answer vectors of its published definition,
and the Box-Muller normals drawn from it.  No GPU needed."""
import numpy as np

from inputs.philox import philox4x32_10, philox_normal

# (counter, key) -> output words: the known-answer vectors published with the
# Random123 implementation of Salmon et al. (SC'11), philox4x32 with 10 rounds
KAT = [
    ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF,) * 4, (0xFFFFFFFF, 0xFFFFFFFF), (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
]


def test_known_answers():
    for ctr, key, want in KAT:
        got = philox4x32_10(np.array([ctr], dtype=np.uint32), key)[0]
        assert tuple(int(v) for v in got) == want


def test_counters_are_independent_of_batching():
    ids = np.arange(1000, dtype=np.uint64) * 7919 + (np.uint64(1) << np.uint64(33))
    whole = philox_normal(ids, 12345)
    parts = np.concatenate([philox_normal(ids[i:i + 37], 12345) for i in range(0, ids.size, 37)])
    assert np.array_equal(whole, parts)
    assert not np.array_equal(whole, philox_normal(ids, 12346))


def test_normal_moments():
    g = philox_normal(np.arange(1 << 20), 3)
    n = g.size
    assert abs(g.mean()) < 5 / np.sqrt(n)
    assert abs(g.var() - 1.0) < 5 * np.sqrt(2.0 / n)
    # tail mass beyond 3 sigma: 0.0027 for a standard normal
    assert abs((np.abs(g) > 3).mean() - 0.0027) < 0.0005
