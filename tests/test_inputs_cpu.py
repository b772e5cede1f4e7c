"""The seeded input generators: values depend only on (seed, position), so
every size and every chunking of the stream gives the same numbers, and the
states they build are normalised on the grid."""
import numpy as np

import gpe_inputs as gi


def test_uniform_and_normal_depend_only_on_the_stream_position():
    u = gi.uniform(5, 1000)
    assert np.array_equal(gi.uniform(5, 400, offset=600), u[600:])
    assert np.all((u >= 0.0) & (u < 1.0))
    n_big = gi.normal(7, (1 << 22) + 6)            # crosses the 2^21-pair chunk boundary
    assert np.array_equal(gi.normal(7, 10), n_big[:10])
    i = 1 << 22
    pair = gi.uniform(7, 2, offset=i)               # the pair that makes normals i, i+1
    r = np.sqrt(-2.0 * np.log(1.0 - pair[0]))
    assert np.allclose(n_big[i:i + 2], [r * np.cos(2 * np.pi * pair[1]), r * np.sin(2 * np.pi * pair[1])],
                       rtol=0, atol=1e-12)
    assert abs(np.mean(n_big)) < 3e-3 and abs(np.std(n_big) - 1.0) < 3e-3


def test_gaussian_state_is_normalised_and_seeded():
    a = gi.gaussian_state(64, 32, 16.0, 8.0, 1.5, 1e-2, seed=3)
    b = gi.gaussian_state(64, 32, 16.0, 8.0, 1.5, 1e-2, seed=3)
    c = gi.gaussian_state(64, 32, 16.0, 8.0, 1.5, 1e-2, seed=4)
    assert a.shape == (32, 64)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert abs(np.sum(np.abs(a) ** 2) * (16.0 / 64) * (8.0 / 32) - 1.0) < 1e-12
