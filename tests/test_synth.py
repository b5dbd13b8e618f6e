"""The seeded input generator: SplitMix64 restated with Python integers, and
the structural properties of the generated systems."""
import numpy as np

from paper_2501_05938_gb300 import synth

MASK = (1 << 64) - 1
G = 0x9E3779B97F4A7C15


def mix64_int(z):
    z &= MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def test_splitmix64_counter_form_matches_sequential_generator():
    seed, stream = 1002, 3
    key = mix64_int(seed + stream * G)
    # a sequential SplitMix64 seeded with key: state += G, output mix64(state)
    state, seq = key, []
    for _ in range(10):
        state = (state + G) & MASK
        seq.append(mix64_int(state))
    assert [int(v) for v in synth.raw(seed, stream, 0, 10)] == seq
    assert [int(v) for v in synth.raw(seed, stream, 4, 3)] == seq[4:7]


def test_uniforms_in_unit_interval_and_roughly_uniform():
    u = synth.uniform(1, 1, 0, 200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5e-3
    assert np.all(np.diff(np.sort(u * 2**53)) % 1 == 0)


def test_paper_system_structure():
    n = 10000
    s = synth.system(1001, n)
    a, b, c, d, x = s["a"], s["b"], s["c"], s["d"], s["x_true"]
    assert a[0] == 0.0 and c[-1] == 0.0
    assert np.all(b - (np.abs(a) + np.abs(c)) >= 1.0)
    assert np.all(b - (np.abs(a) + np.abs(c)) < 2.0 + 1e-15)
    assert np.all(np.abs(x) <= 1.0)
    # d equals A x_true up to rounding of three products and two sums
    Ax = b * x
    Ax[1:] += a[1:] * x[:-1]
    Ax[:-1] += c[:-1] * x[1:]
    assert np.max(np.abs(d - Ax)) < 1e-14


def test_batched_offsets_and_decoupling():
    sizes = synth.batch_sizes(1003, 64, 8, 20)
    assert sizes.min() >= 256 and sizes.max() < 2**20
    off = synth.offsets_from_sizes(sizes)
    s = synth.system(1003, int(off[-1]), offsets=off)
    assert np.all(s["a"][off[:-1]] == 0.0)
    assert np.all(s["c"][off[1:] - 1] == 0.0)


def test_ratio_system_dominance():
    s = synth.system(9, 5000, kind=synth.KIND_RATIO, ratio=1.1)
    off = np.abs(s["a"]) + np.abs(s["c"])
    np.testing.assert_allclose(s["b"], 1.1 * np.maximum(off, synth.RATIO_FLOOR), rtol=1e-15)


def test_same_seed_same_arrays_prefix_property():
    s1 = synth.system(42, 1000)
    s2 = synth.system(42, 2000)
    # elements depend only on (seed, stream, index), except the boundary row
    np.testing.assert_array_equal(s1["a"], s2["a"][:1000])
    np.testing.assert_array_equal(s1["b"][:999], s2["b"][:999])
