"""The seeded serving trace: reproducible, Poisson arrivals at the stated
mean rate, excitation counts in range, unit-modulus weights, and a scene pool
within the stated size ranges (spheres 1k-5k, ribs 10k-40k, kidneys 20k-60k
triangles)."""
import numpy as np

from synth import serving


def test_trace_is_reproducible_and_in_range():
    r1, w1 = serving.trace(200, rate=20.0, max_exc=64)
    r2, w2 = serving.trace(200, rate=20.0, max_exc=64)
    assert r1 == r2
    t = np.array([a for a, _, _ in r1])
    assert t[0] == 0 and np.all(np.diff(t) >= 0)
    assert abs(len(t) / t[-1] - 20.0) < 4.0          # mean rate within sampling noise
    n = np.array([ne for _, _, ne in r1])
    assert n.min() >= 1 and n.max() <= 64
    W = w1(3, 16)
    assert W.shape == (r1[3][2], 16) and np.allclose(np.abs(W), 1.0)
    assert np.array_equal(W, w2(3, 16))


def test_pool_sizes():
    ranges = {"sphere": (1000, 5200), "rib": (10000, 40000), "kidney": (19000, 60000)}
    for key, make in serving.POOL.items():
        s = make()
        lo, hi = ranges[key.split("_")[0]]
        assert lo <= s.n_triangles <= hi, (key, s.n_triangles)
        assert s.transducer is not None and s.meta["omega_rho0"] > 0 and s.meta["r_eps"] > 0
