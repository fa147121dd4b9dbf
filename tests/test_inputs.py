"""The seeded input generator follows the published SplitMix64 definition
(Steele, Lea & Flood 2014): checked against a scalar big-integer transcription
and the stream's well-known first output for seed 0."""
import numpy as np

from paper_1711_02473_gb300 import inputs

MASK = (1 << 64) - 1


def scalar_stream(seed, count):
    out, state = [], seed
    for _ in range(count):
        state = (state + 0x9E3779B97F4A7C15) & MASK
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
        out.append(z ^ (z >> 31))
    return out


def test_splitmix64_matches_definition():
    for seed in (0, 1, 2, 12345, 2 ** 63 + 7):
        v = inputs.splitmix64(seed, 0, 50)
        assert [int(t) for t in v] == scalar_stream(seed, 50)
        assert [int(t) for t in inputs.splitmix64(seed, 20, 5)] == scalar_stream(seed, 25)[20:]
    assert int(inputs.splitmix64(0, 0, 1)[0]) == 0xE220A8397B1DCDAF


def test_box_coords_perturbation():
    nx, ny, nz = 4, 3, 5
    X = inputs.box_coords(nx, ny, nz, perturb=0.1, seed=0)
    X0 = inputs.box_coords(nx, ny, nz, perturb=0.0)
    d = X - X0
    h = np.array([1 / nx, 1 / ny, 1 / nz])
    assert np.all(np.abs(d) <= 0.1 * h + 1e-17)
    I, J, K = np.unravel_index(np.arange(len(X)), (nx + 1, ny + 1, nz + 1))
    bnd = (I == 0) | (I == nx) | (J == 0) | (J == ny) | (K == 0) | (K == nz)
    assert np.all(d[bnd] == 0) and np.all(d[~bnd] != 0)
    # draws are consumed in interior-vertex order, x then y then z
    u = inputs.uniform01(0, 3)
    first = np.flatnonzero(~bnd)[0]
    np.testing.assert_array_equal(X[first], X0[first] + 0.1 * h * (2 * u - 1))


def test_vectors_and_degrees():
    v = inputs.random_vector(10, 3, seed=1)
    assert v.shape == (10, 3) and v.min() >= -1 and v.max() < 1
    np.testing.assert_array_equal(v.reshape(-1), -1 + 2 * inputs.uniform01(1, 30))
    p = inputs.padaptive_degrees(200000, 8, seed=2)
    freq = np.bincount(p, minlength=9)[1:] / len(p)
    w = 1 / np.arange(1, 9)
    np.testing.assert_allclose(freq, w / w.sum(), atol=4e-3)
