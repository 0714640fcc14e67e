"""Pins of the oracle's convolutional operator (Eq. 9, Eq. 11) against brute force.

The dense Jacobian is assembled entry by entry from scan-point and voxel
positions (Eq. 2, Eq. 6) without any offset table or FFT; the FFT operator,
the direct quadruple sum and the library 2-D convolution must all agree
with it.
"""

import json
import os

import numpy as np
import pytest
from scipy import signal

from oracle import operators as op
from oracle import physics as ph

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def cfg1_medium():
    return ph.Medium(0.01, 1.0, 1.4, r_min=0.5)


def sub_grid(mode="linear"):
    """The 8 x 8 (1 mm) x first 4 depths (1-4 mm) x first 16 bins (50 ps) sub-grid of config 1."""
    return op.Grid(8, 4, 16, 1.0, 1.0, 1.0, 50.0, mode=mode)


@pytest.fixture(scope="module", params=["linear", "circular"])
def small(request):
    g = sub_grid(request.param)
    m = cfg1_medium()
    w = op.kernel_offsets(g, m)
    return g, m, w, op.kernel_spectrum(w, g), op.dense_jacobian(g, m)


def test_dense_jacobian_columns_equal_forward(small):
    """J e_q == forward(e_q) for every voxel q (shift-invariance of the confocal J, Section 4)."""
    g, _, _, wh, J = small
    nvox = g.nz * g.n * g.n
    scale = np.abs(J).max()
    for q in range(nvox):
        e = np.zeros(nvox)
        e[q] = 1.0
        col = op.forward_fft(wh, e.reshape(g.nz, g.n, g.n), g).ravel()
        assert np.abs(col - J[:, q]).max() <= 1e-13 * scale


def test_dense_jacobian_transpose_equals_adjoint(small):
    g, _, _, wh, J = small
    rng = np.random.default_rng(3)
    m = rng.standard_normal((g.nt, g.n, g.n))
    a = op.adjoint_fft(wh, m, g).ravel()
    b = J.T @ m.ravel()
    assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()


def test_fft_equals_direct(small):
    g, _, w, wh, _ = small
    rng = np.random.default_rng(4)
    mu = rng.standard_normal((g.nz, g.n, g.n))
    a = op.forward_fft(wh, mu, g)
    b = op.forward_direct(w, mu, g)
    assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()
    m = rng.standard_normal((g.nt, g.n, g.n))
    c = op.adjoint_fft(wh, m, g)
    d = op.adjoint_direct(w, m, g)
    assert np.abs(c - d).max() <= 1e-13 * np.abs(d).max()


@pytest.mark.slow
def test_fft_equals_direct_cfg1():
    """Config 1 (32 x 32 x 16 x 64): FFT operator == direct summation to 1e-12."""
    g = op.Grid(32, 16, 64, 1.0, 1.0, 1.0, 50.0)
    w = op.kernel_offsets(g, cfg1_medium())
    wh = op.kernel_spectrum(w, g)
    rng = np.random.default_rng(5)
    mu = np.zeros((16, 32, 32))
    mu[:, 4:28:3, 6:30:5] = rng.uniform(0, 0.02, size=(16, 8, 5))
    a = op.forward_fft(wh, mu, g)
    b = op.forward_direct(w, mu, g)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def test_adjoint_identity(small):
    g, _, _, wh, _ = small
    rng = np.random.default_rng(6)
    x = rng.standard_normal((g.nz, g.n, g.n))
    y = rng.standard_normal((g.nt, g.n, g.n))
    ax = op.forward_fft(wh, x, g)
    aty = op.adjoint_fft(wh, y, g)
    lhs = float(np.sum(ax * y))
    rhs = float(np.sum(x * aty))
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(ax) * np.linalg.norm(y)


def test_single_depth_is_2d_convolution():
    """Z = 1 reduces to Eq. 9: each time bin is a plain 2-D linear convolution."""
    g = op.Grid(12, 1, 8, 1.0, 1.0, 3.0, 50.0)
    w = op.kernel_offsets(g, cfg1_medium())
    wh = op.kernel_spectrum(w, g)
    rng = np.random.default_rng(7)
    mu = rng.uniform(0, 1, (1, 12, 12))
    m = op.forward_fft(wh, mu, g)
    for k in range(g.nt):
        full = signal.convolve2d(mu[0], w[k, 0], mode="full")  # offsets -(N-1)..(N-1)
        want = full[g.n - 1: 2 * g.n - 1, g.n - 1: 2 * g.n - 1]
        assert np.abs(m[k] - want).max() <= 1e-13 * np.abs(want).max()


def test_shift_equivariance():
    """Shifting a point absorber shifts the measurement (away from the scan edges)."""
    g = sub_grid()
    wh = op.kernel_spectrum(op.kernel_offsets(g, cfg1_medium()), g)
    a = np.zeros((g.nz, g.n, g.n))
    a[2, 3, 2] = 1.0
    b = np.roll(a, (1, 2), axis=(1, 2))
    ma = op.forward_fft(wh, a, g)
    mb = op.forward_fft(wh, b, g)
    assert np.abs(mb[:, 1:, 2:] - ma[:, :-1, :-2]).max() <= 1e-14 * np.abs(ma).max()


def test_kernel_spectrum_is_real_and_symmetric():
    """The kernel is even in each lateral axis (and x<->y for dx == dy): W_hat is real, symmetric."""
    g = op.Grid(16, 3, 8, 0.5, 0.5, 0.5, 25.0)
    wh = op.kernel_spectrum(op.kernel_offsets(g, cfg1_medium()), g)
    assert np.abs(wh.imag).max() <= 1e-15 * np.abs(wh.real).max()
    assert np.abs(wh - np.swapaxes(wh, -1, -2)).max() <= 1e-15 * np.abs(wh).max()
    assert np.abs(wh - np.roll(wh[..., ::-1], 1, axis=-1)).max() <= 1e-15 * np.abs(wh).max()


def test_paper_dimensions():
    """The Jacobian sizes the paper prints (Section 3 and Section 6) follow N_meas x N_vox."""
    with open(os.path.join(GOLDEN, "paper_dimensions.json")) as f:
        facts = json.load(f)
    d = facts["dense_tof_dot"]
    n_meas = d["sources"] * d["detectors"] * d["time_bins"]
    n_vox = int(round(d["extent_mm"][0] / d["voxel_mm"])) * int(round(d["extent_mm"][1] / d["voxel_mm"])) \
        * int(round(d["extent_mm"][2] / d["voxel_mm"]))
    assert n_meas == d["jacobian_rows"]
    assert abs(n_vox - d["jacobian_cols"]) <= 0.01 * d["jacobian_cols"]
    c = facts["confocal_scan"]
    g = op.Grid(c["side"], 1, 1, 1.0, 1.0, 1.0, 50.0)
    J = op.dense_jacobian(op.Grid(4, 1, 2, 1.0, 1.0, 1.0, 50.0), cfg1_medium())
    assert J.shape == (2 * 16, 16)  # rows = bins x scan points, cols = voxels
    assert g.n * g.n == c["scan_points"]
