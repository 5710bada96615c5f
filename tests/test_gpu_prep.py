"""Full-disk weights (Eqs. 14-15) on the GPU vs the oracle."""
import numpy as np
import pytest

import workloads as W
from oracle import lm, me
from gpu_common import LINE, T, X, f32, vf  # noqa: F401

pytestmark = pytest.mark.gpu


def test_limb_weights_vs_oracle(vf):
    v, h, torch = vf
    p, idx = W.full_disk_params(2, side=512, radius=259.0)
    sel = np.linspace(0, len(idx) - 1, 3000).astype(int)
    p, idx = f32(p[sel]), idx[sel]
    mu = f32(W.disk_mu(idx, side=512, radius=259.0))
    # darken the continuum with the centre-to-limb law
    p[:, 7] *= lm.icont_mu(mu)
    p[:, 8] *= lm.icont_mu(mu)
    obs = f32(me.synth(p, f32(T), f32(X), LINE).reshape(len(p), -1))
    sig = [1e-3, 2e-3, 2e-3, 1.5e-3]
    w = v.vfisv_limb_weights(h, obs.astype(np.float32), mu.astype(np.float32), 1.0, sig)
    ref = lm.limb_weights(obs, mu, 1.0, sig)
    # FP32 kernel: about ten roundings in w_I, doubled by the square
    np.testing.assert_allclose(w, ref, rtol=4e-6)
