"""Pins of the learned-solver oracle: the 3-D convolution against
scipy.ndimage.correlate, and the analytic gradients of the unrolled loss
against central finite differences in FP64."""

import numpy as np
import pytest
from scipy import ndimage

from oracle import learned as ln
from oracle import operators as op
from oracle import physics as ph
from oracle import solvers as so


def test_conv3d_is_zero_padded_correlation():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 5, 6, 7))
    w = rng.standard_normal((3, 2, 27))
    b = rng.standard_normal(3)
    y = ln.conv3d(x, w, b)
    for o in range(3):
        want = np.full(x.shape[1:], b[o])
        for c in range(2):
            want += ndimage.correlate(x[c], w[o, c].reshape(3, 3, 3), mode="constant", cval=0.0)
        assert np.abs(y[o] - want).max() <= 1e-12


def test_param_count():
    assert ln.param_count(10) == 14688 + 49 + 10


def _tiny_problem(stages=3):
    g = op.Grid(6, 3, 10, 1.0, 1.0, 1.0, 50.0)
    med = ph.Medium(0.01, 1.0, 1.4, r_min=0.5)
    wh = op.kernel_spectrum(op.kernel_offsets(g, med), g)
    s = so.spectral_norm(wh)
    fwd = lambda v: op.forward_fft(wh / s, v, g)
    adj = lambda r: op.adjoint_fft(wh / s, r, g)
    rng = np.random.default_rng(1)
    mu = rng.uniform(0, 0.02, (g.nz, g.n, g.n)) * (rng.uniform(size=(g.nz, g.n, g.n)) < 0.4)
    m_n = fwd(mu)
    theta = ln.init_params(stages, seed=5)
    theta[-stages:] = [0.9, 1.1, 0.8][:stages]
    return theta, stages, fwd, adj, m_n, mu


def test_gradients_match_finite_differences():
    theta, stages, fwd, adj, m_n, mu = _tiny_problem()
    loss, grad = ln.loss_and_grad(theta, stages, fwd, adj, m_n, mu)
    rng = np.random.default_rng(2)
    idx = list(rng.choice(len(theta) - stages, 12, replace=False)) + list(range(len(theta) - stages, len(theta)))
    for i in idx:
        h = 1e-6 * max(1.0, abs(theta[i]))
        tp = theta.copy()
        tm = theta.copy()
        tp[i] += h
        tm[i] -= h
        lp = ln.loss_and_grad(tp, stages, fwd, adj, m_n, mu)[0]
        lm = ln.loss_and_grad(tm, stages, fwd, adj, m_n, mu)[0]
        fd = (lp - lm) / (2 * h)
        assert grad[i] == pytest.approx(fd, rel=1e-5, abs=1e-9 * max(1.0, abs(loss)))
