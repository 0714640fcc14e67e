"""Pins of the multiplexed composite operator (Section 5, Eq. 12) in the oracle."""

import numpy as np
import pytest
from scipy import linalg

from oracle import multiplex as mx
from oracle import operators as op
from oracle import physics as ph
from oracle import solvers as so


def test_hadamard_is_sylvester_and_orthogonal():
    h = mx.hadamard(64)
    assert np.array_equal(h, linalg.hadamard(64))
    assert np.array_equal(h @ h.T, 64 * np.eye(64))
    assert np.array_equal(h, h.T)


def _grid(n=16, nz=2, nt=10):
    g = op.Grid(n, nz, nt, 1.0, 1.0, 1.0, 50.0)
    wh = op.kernel_spectrum(op.kernel_offsets(g, ph.Medium(0.01, 1.0, 1.4, r_min=0.5)), g)
    return g, wh


def test_block_multiplex_equals_dense_block_matrix():
    """y = S m with S built entry by entry: scan point (r, c) of block (br, bc) is
    source index 8 (r mod 8) + (c mod 8) within that block."""
    rng = np.random.default_rng(1)
    m = rng.standard_normal((3, 16, 16))
    h = mx.hadamard(64)
    n = 16
    s_full = np.zeros((n * n, n * n))
    for r in range(n):
        for c in range(n):
            for r2 in range(n):
                for c2 in range(n):
                    if r // 8 == r2 // 8 and c // 8 == c2 // 8:
                        s_full[r * n + c, r2 * n + c2] = h[8 * (r % 8) + c % 8, 8 * (r2 % 8) + c2 % 8]
    want = np.einsum("ij,tj->ti", s_full, m.reshape(3, -1)).reshape(m.shape)
    assert np.allclose(mx.block_multiplex(m), want, rtol=1e-13, atol=1e-12)


def test_composite_adjoint_identity_and_norm():
    g, wh = _grid()
    rng = np.random.default_rng(2)
    x = rng.standard_normal((g.nz, g.n, g.n))
    y = rng.standard_normal((g.nt, g.n, g.n))
    lhs = np.vdot(mx.composite_forward(wh, x, g), y)
    rhs = np.vdot(x, mx.composite_adjoint(wh, y, g))
    assert lhs == pytest.approx(rhs, rel=1e-12)
    # S^T S = 64 I: ||S A x|| = 8 ||A x||
    ax = op.forward_fft(wh, x, g)
    assert np.linalg.norm(mx.composite_forward(wh, x, g)) == pytest.approx(8 * np.linalg.norm(ax), rel=1e-12)


def test_multiplexed_fista_lam0_is_least_squares_of_s_j():
    """lam = 0 on one depth: the composite FISTA converges to the least-squares
    solution of the dense S J (with S J = 8 Q J, Q orthogonal, the same as J's)."""
    g = op.Grid(8, 1, 16, 1.0, 1.0, 2.0, 50.0)
    med = ph.Medium(0.01, 1.0, 1.4, r_min=0.5)
    wh = op.kernel_spectrum(op.kernel_offsets(g, med), g)
    J = op.dense_jacobian(g, med)
    rng = np.random.default_rng(3)
    mu = rng.uniform(0, 0.02, (1, 8, 8))
    y = mx.composite_forward(wh, mu, g)
    y = y + 0.02 * np.abs(y).max() * rng.standard_normal(y.shape)
    x, info = so.fista_l1(wh, y, g, 20000, lam=0.0, multiplexed=True)
    assert info["scale"] == pytest.approx(8 * so.spectral_norm(wh), rel=1e-12)
    h = mx.hadamard(64)
    sj = np.kron(np.eye(g.nt), h) @ J  # one 8 x 8 block per time bin
    want, *_ = np.linalg.lstsq(sj, y.ravel(), rcond=None)
    assert np.abs(x.ravel() - want).max() <= 1e-8 * np.abs(want).max()
