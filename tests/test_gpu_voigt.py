"""Device Voigt/Faraday-Voigt functions vs the oracle's library Faddeeva
function, and the paper's Taylor-table experiment E1 (Sec. 3.2, Fig. 2):
first-order extrapolation from a 500 x 100 table stays below 1e-4 at a = 1."""
import numpy as np
import pytest

from oracle import me
from gpu_common import vf  # noqa: F401

pytestmark = pytest.mark.gpu


def test_rational_series_vs_oracle(vf):
    v, h, torch = vf
    rng = np.random.default_rng(0)
    a = np.concatenate([np.zeros(2000), rng.uniform(0, 5, 20000), rng.uniform(0, 1e-3, 2000)])
    u = np.concatenate([rng.uniform(-60, 60, 2000), rng.uniform(-60, 60, 20000),
                        rng.uniform(-3, 3, 2000)])
    a32, u32 = a.astype(np.float32), u.astype(np.float32)
    H, F = v.vfisv_voigt(h, a32, u32, 0)
    Hr, Fr = me.voigt_faraday(a32.astype(np.float64), u32.astype(np.float64))
    assert np.abs(H - Hr).max() < 1e-6 and np.abs(F - Fr).max() < 1e-6


@pytest.mark.parametrize("order,tol", [(1, 1e-4), (2, 2e-6)])
def test_taylor_table_at_unit_damping(vf, order, tol):
    """E1: 10^6 frequencies, a = 1 (the paper's Fig. 2 setting)."""
    v, h, torch = vf
    u = np.linspace(-20, 20, 1_000_001)[:-1].astype(np.float32)
    a = np.ones_like(u)
    H, F = v.vfisv_voigt(h, a, u, order)
    Hr, Fr = me.voigt_faraday(1.0, u.astype(np.float64))
    assert np.abs(H - Hr).max() < tol and np.abs(F - Fr).max() < tol


def test_taylor_table_exact_at_nodes_and_outside(vf):
    v, h, torch = vf
    u = np.array([0.0, 0.04 * 7, -0.04 * 123, 12.0, 25.0, -40.0], np.float32)
    a = np.array([0.05 * 3, 0.0, 0.05 * 40, 7.0, 0.3, 0.1], np.float32)
    H1, F1 = v.vfisv_voigt(h, a, u, 1)
    H0, F0 = v.vfisv_voigt(h, a, u, 0)
    # at table nodes both orders reduce to the tabulated (rational-series) value
    np.testing.assert_allclose(H1[:3], H0[:3], atol=2e-7)
    np.testing.assert_allclose(F1[:3], F0[:3], atol=2e-7)
    # outside the table (a >= 5 or |u| >= 20) the rational series is used
    assert np.array_equal(H1[[3, 4, 5]], H0[[3, 4, 5]])
