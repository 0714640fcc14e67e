"""Pins of the fluorescence-mode response (Section 5, simulator paragraph).

The oracle evaluates f = Phi0_ex (*) L_tau (*) R_em through the product of
Laplace transforms and a fixed-Talbot inversion.  These tests hold it to
facts that do not go through that route: known inverse transforms, the
closed-form absorption convolution (tau = 0, one medium), brute-force time
quadrature of the double convolution with two media and a lifetime, the CW
product Phi0_CW(ex) R_CW(em) as the total time integral, and the mean
arrival time growing by exactly tau.
"""

import numpy as np
import pytest
from scipy import integrate

from oracle import operators as op
from oracle import physics as ph

EX = dict(mua=0.01, musp=1.0, n=1.4)
EM = dict(mua=0.005, musp=0.8, n=1.4)


def medium(p, r_min=0.0):
    return ph.Medium(p["mua"], p["musp"], p["n"], r_min=r_min)


@pytest.mark.parametrize("t", [0.3, 2.0, 17.0, 250.0])
def test_talbot_inverts_known_transforms(t):
    a = 0.013
    assert ph.talbot_inverse(lambda s: 1.0 / (s + a), t) == pytest.approx(np.exp(-a * t), rel=1e-10)
    assert ph.talbot_inverse(lambda s: 1.0 / s**2, t) == pytest.approx(t, rel=1e-10)
    # L[a/(2 sqrt(pi) t^1.5) exp(-a^2/(4t))] = exp(-a sqrt(s))
    b = 2.5
    want = b / (2 * np.sqrt(np.pi) * t**1.5) * np.exp(-b * b / (4 * t))
    got = ph.talbot_inverse(lambda s: np.exp(-b * np.sqrt(s)), t)
    assert abs(got - want) <= 1e-10 * max(want, 1e-3)


@pytest.mark.parametrize("rho,z", [(0.0, 1.0), (1.5, 2.0), (4.0, 6.0), (0.0, 0.5)])
def test_instantaneous_one_medium_is_absorption_convolution(rho, z):
    """tau = 0 and one medium: f equals the closed-form Phi0 (*) R of Eq. 5."""
    m = medium(EX, r_min=0.5)
    ts = np.array([5.0, 40.0, 120.0, 400.0, 1500.0])
    want = np.array([float(ph.conv_closed(rho, z, t, m)) for t in ts])
    got = np.array([float(ph.fluorescence_response(rho, z, t, m, m, 0.0)) for t in ts])
    assert np.abs(got - want).max() <= 1e-9 * np.abs(want).max()


def test_binned_is_exact_bin_integral():
    """The edge differences equal adaptive quadrature of the closed form over each bin."""
    m = medium(EX, r_min=0.5)
    rho, z, dt, nt = 1.0, 1.0, 50.0, 24
    got = ph.binned_fluorescence(rho, z, nt, dt, m, m, 0.0)
    want = np.array([integrate.quad(lambda t: float(ph.conv_closed(rho, z, t, m)), k * dt, (k + 1) * dt,
                                    epsabs=0.0, epsrel=1e-12, limit=200)[0] for k in range(nt)])
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()


def _double_convolution(rho, z, t, mx, mm, tau):
    """f(t) = int_0^t L_tau(t-u) int_0^u Phi0_ex(v) R_em(u-v) dv du by nested adaptive quadrature."""
    def inner(u):
        if u <= 0:
            return 0.0
        g = lambda v: float(ph.fluence(rho, z, v, mx) * ph.reflectance(rho, z, u - v, mm))
        return integrate.quad(g, 0.0, u, points=[0.5 * u], limit=300, epsabs=0.0, epsrel=1e-11)[0]
    h = lambda u: np.exp(-(t - u) / tau) / tau * inner(u)
    return integrate.quad(h, 0.0, t, limit=300, epsabs=0.0, epsrel=1e-9)[0]


@pytest.mark.parametrize("rho,z,t,tau", [(1.0, 3.0, 600.0, 300.0), (3.0, 5.0, 1200.0, 1000.0)])
def test_two_media_and_lifetime_match_brute_force(rho, z, t, tau):
    """Separate excitation / emission optics and a lifetime against the time-domain definition."""
    mx, mm = medium(EX), medium(EM)
    want = _double_convolution(rho, z, t, mx, mm, tau)
    got = float(ph.fluorescence_response(rho, z, t, mx, mm, tau))
    assert got == pytest.approx(want, rel=1e-7)
    # the media are not interchangeable: swapping them changes the response
    swapped = float(ph.fluorescence_response(rho, z, t, mm, mx, tau))
    assert abs(swapped - want) > 1e-3 * abs(want)


@pytest.mark.parametrize("rho,z,tau", [(0.0, 2.0, 0.0), (2.0, 4.0, 500.0), (5.0, 3.0, 2000.0)])
def test_total_is_cw_product(rho, z, tau):
    """int_0^inf f dt = Phi0_CW(excitation) * R_CW(emission): the lifetime density integrates to one."""
    mx, mm = medium(EX), medium(EM)
    want = float(ph.fluence_cw(rho, z, mx) * ph.reflectance_cw(rho, z, mm))
    got = float(ph.fluorescence_cumulative(rho, z, 4e4, mx, mm, tau))
    assert got == pytest.approx(want, rel=1e-9)


def _mean_time(f, t_end=3e4):
    pts = [50.0, 200.0, 1000.0, 5000.0]
    m0 = integrate.quad(f, 0.0, t_end, points=pts, limit=400, epsabs=0.0, epsrel=1e-10)[0]
    m1 = integrate.quad(lambda t: t * f(t), 0.0, t_end, points=pts, limit=400, epsabs=0.0, epsrel=1e-10)[0]
    return m1 / m0


def test_mean_arrival_time_adds_lifetime():
    """Mean time of a convolution = sum of the factors' mean times (tau for the lifetime density)."""
    mx, mm = medium(EX), medium(EM)
    rho, z, tau = 1.0, 2.0, 700.0
    t_phi = _mean_time(lambda t: float(ph.fluence(rho, z, t, mx)))
    t_r = _mean_time(lambda t: float(ph.reflectance(rho, z, t, mm)))
    got = _mean_time(lambda t: float(ph.fluorescence_response(rho, z, t, mx, mm, tau)) if t > 0 else 0.0)
    assert got == pytest.approx(t_phi + t_r + tau, rel=1e-6)


def test_kernel_table_layout_and_symmetry():
    """Offset table: mirror-symmetric, non-negative, bins sum to the cumulative at the last edge."""
    g = op.Grid(6, 3, 10, 1.0, 1.0, 1.0, 50.0)
    mx, mm = medium(EX, 0.5), medium(EM, 0.5)
    w = op.kernel_offsets_fluorescence(g, mx, mm, 400.0)
    assert w.shape == (10, 3, 11, 11)
    assert np.array_equal(w, w[:, :, ::-1, :]) and np.array_equal(w, w[:, :, :, ::-1])
    assert np.array_equal(w, np.swapaxes(w, 2, 3))
    assert w.min() >= -1e-12 * w.max()
    rho = np.hypot(2.0, 1.0)
    cum = float(ph.fluorescence_cumulative(rho, g.depths[1], 10 * g.dt, mx, mm, 400.0))
    assert w[:, 1, 5 + 1, 5 + 2].sum() == pytest.approx(cum * g.voxel_volume, rel=1e-9)
