"""The seeded input generators: determinism, ranges and shapes."""
import numpy as np

import workloads as W


def test_grid_and_filters():
    x = W.wavelength_grid()
    assert x.size == 149 and x[0] == -740.0 and x[-1] == 740.0
    T = W.hmi_filters(x)
    assert T.shape == (6, 149)
    np.testing.assert_allclose(T.sum(1), 1.0, rtol=1e-14)
    peaks = x[T.argmax(1)]
    np.testing.assert_allclose(peaks, W.HMI_CENTRES_mA, atol=5.0)


def test_param_draws_deterministic_and_in_range():
    a = W.quiet_and_active_params(5000, 0)
    b = W.quiet_and_active_params(5000, 0)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, W.quiet_and_active_params(5000, 1))
    lo = [0, 0, 0, 1, 20, 0, -7, 0.1, 0.6, 1]
    hi = [3000, 180, 180, 50, 50, 0.5, 7, 0.4, 0.9, 1]
    assert np.all(a >= np.array(lo) - 1e-12) and np.all(a <= np.array(hi) + 1e-12)
    # cos(gamma) uniform: mean of cos ~ 0
    assert abs(np.cos(np.radians(a[:, 1])).mean()) < 0.05


def test_noise_and_weights():
    p = W.quiet_and_active_params(1000, 2)
    s = np.zeros((1000, 24))
    o, w = W.observe(s, p, W.noise(1000, 24, 2))
    z = o / (1e-3 * W.continuum(p))[:, None]
    assert abs(z.std() - 1) < 0.02
    np.testing.assert_allclose(w, 1.0 / (1e-3 * W.continuum(p))[:, None] ** 2 * np.ones((1, 24)))


def test_disk_geometry():
    m = W.disk_mask()
    n = int(m.sum())
    # ~13.5 million on-disk pixels (the r = 2073 disk is clipped slightly by the 4096 frame)
    assert 13.4e6 < n < np.pi * 2073 ** 2
    # a scaled-down disk keeps the recipe: blobs cover >= 10 % with weight > 0.5
    p, idx = W.full_disk_params(2, side=1024, radius=518.0)
    assert p.shape == (idx.size, 10)
    assert p[:, 0].max() <= 3500.0 and (p[:, 0] > 750).mean() >= 0.10
    quiet = p[:, 0] <= 200
    assert quiet.mean() > 0.3
