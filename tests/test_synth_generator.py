"""The seeded input generator (synth/) against the published definition of its parts.

Both the CUDA path and the oracle receive the host arrays synth/ produces, so a wrong generator
would not break parity; these checks pin it to what the design says it is: SplitMix64 (Steele, Lea
and Flood, OOPSLA 2014) in counter mode, 53-bit uniforms strictly inside (0, 1), and Box-Muller
normals.  The mixer is pinned by the first outputs of the reference SplitMix64 sequence seeded
with 0, the C draws by an independent Python transcription of the counter scheme, and the
normals by their moments and by the pairing of two uniforms each."""
import math

import numpy as np

import synth

MASK = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15

# The reference SplitMix64 generator seeded with 0: its first five outputs.
SPLITMIX64_SEED0 = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC,
                    0x1B39896A51A8749B]


def _mix64(z):
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def _key(seed, stream):
    return _mix64(seed ^ _mix64((stream + 0x632BE59BD9B4E019) & MASK))


def test_mixer_gives_the_reference_sequence():
    state, out = 0, []
    for _ in range(5):
        state = (state + GOLDEN) & MASK
        out.append(_mix64(state))
    assert out == SPLITMIX64_SEED0


def test_counter_draws_follow_the_definition():
    for seed, stream in ((13023876, 0), (1, 7), (2**63 + 5, 123456)):
        key = _key(seed, stream)
        got = synth.u64(seed, stream, 64, offset=1000)
        want = [_mix64((key + (1000 + i + 1) * GOLDEN) & MASK) for i in range(64)]
        assert [int(x) for x in got] == want
    # draw i of a stream is the (i + 1)-th output of the reference generator started at its key
    key = _key(5, 3)
    state, seq = key, []
    for _ in range(8):
        state = (state + GOLDEN) & MASK
        seq.append(_mix64(state))
    assert [int(x) for x in synth.u64(5, 3, 8)] == seq
    # any slice is the same draws (no state carried between calls)
    full = synth.u64(9, 2, 100)
    assert np.array_equal(synth.u64(9, 2, 30, offset=40), full[40:70])


def test_uniforms_are_the_top_53_bits_strictly_inside_the_interval():
    z = synth.u64(77, 4, 4096)
    u = synth.uniform(77, 4, 4096, 0.0, 1.0)
    want = ((z >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0**-53
    assert np.array_equal(u, want)
    assert u.min() > 0.0 and u.max() < 1.0
    w = synth.uniform(77, 4, 4096, 0.5, 1.5)
    np.testing.assert_allclose(w, 0.5 + u, rtol=0, atol=1e-15)


def test_normals_are_box_muller_of_consecutive_uniform_pairs():
    seed, stream, rows, cols = 31, 6, 7, 3
    a = synth.normal_matrix(seed, stream, rows, cols)          # shape (cols, rows)
    u = synth.uniform(seed, stream, 2 * rows * cols, 0.0, 1.0)
    for c in range(cols):
        for j in range(rows):
            i = c * rows + j
            want = math.sqrt(-2.0 * math.log(u[2 * i])) * math.cos(2.0 * math.pi * u[2 * i + 1])
            assert abs(a[c, j] - want) <= 1e-12 * max(1.0, abs(want))
    big = synth.normal_matrix(3, 1, 200000, 5).ravel()
    assert abs(big.mean()) < 5e-3
    assert abs(big.var() - 1.0) < 1e-2
    assert abs(np.mean(big**4) - 3.0) < 5e-2                     # the normal's fourth moment
    scaled = synth.normal_matrix(3, 1, 4, 2, mean=2.0, std=0.5, row_scale=np.array([1.0, 2.0, 3.0, 4.0]))
    base = synth.normal_matrix(3, 1, 4, 2)
    np.testing.assert_allclose(scaled, 2.0 + 0.5 * np.array([1.0, 2.0, 3.0, 4.0]) * base, rtol=1e-15)
