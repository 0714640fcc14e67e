"""Pins of the oracle's diffusion physics against facts fixed by the mathematics.

Each test checks the oracle against something other than itself: a boundary
condition, a numerical derivative or integral of the defining expression,
or an independently derived closed form.  A dropped term, a wrong sign, a
misplaced image source or a wrong prefactor in oracle/physics.py fails one
of them.
"""

import numpy as np
import pytest
from scipy import integrate

from oracle import physics as ph

CFG1 = dict(mua=0.01, musp=1.0, n=1.4)


def med(**kw):
    p = dict(CFG1)
    p.update(kw)
    return ph.Medium(p["mua"], p["musp"], p["n"], z0=p.get("z0", 0.0), r_min=p.get("r_min", 0.0))


def test_constants_cfg1():
    """Textbook diffusion constants for mua=0.01, musp'=1.0, n=1.4."""
    m = med()
    assert m.c == pytest.approx(0.299792458 / 1.4, rel=1e-15)
    assert m.D == pytest.approx(1.0 / 3.03, rel=1e-15)
    assert m.z0 == pytest.approx(1.0 / 1.01, rel=1e-15)
    # Groenhuis fit at n = 1.4 and A = (1+R)/(1-R)
    assert m.Reff == pytest.approx(0.52948898, abs=1e-8)
    assert m.A == pytest.approx(3.2506975, abs=1e-6)
    assert m.zb == pytest.approx(2.0 * m.A * m.D, rel=1e-15)
    assert m.mueff == pytest.approx(np.sqrt(0.01 * 3.03), rel=1e-14)


@pytest.mark.parametrize("rho", [0.0, 1.0, 4.0])
@pytest.mark.parametrize("t", [20.0, 200.0, 2000.0])
def test_fluence_vanishes_on_extrapolated_boundary(rho, t):
    """Phi0 = 0 on the plane z = -zb: the image source sits at the mirror of z0."""
    m = med()
    scale = float(ph.fluence(rho, m.z0, t, m))
    assert abs(float(ph.fluence(rho, -m.zb, t, m))) <= 1e-14 * max(scale, 1e-300)


def _point_fluence(x, y, zp, zs, t, m):
    """Fluence at (x,y,zp) of a unit impulse at (0,0,zs) with negative image at -(zs+2zb)."""
    ra = np.sqrt(x * x + y * y + (zp - zs) ** 2)
    rb = np.sqrt(x * x + y * y + (zp + zs + 2 * m.zb) ** 2)
    return np.exp(-m.mua * m.c * t) * (ph.green_inf(ra, t, m) - ph.green_inf(rb, t, m))


@pytest.mark.parametrize("rho,z,t", [(0.0, 3.0, 150.0), (2.0, 5.0, 400.0), (6.0, 2.0, 900.0)])
def test_reflectance_is_fick_flux(rho, z, t):
    """R(rho,z,t) = D dPhi/dz at the surface, Phi from a source at the voxel depth."""
    m = med()
    h = 1e-4
    d = (_point_fluence(rho, 0.0, h, z, t, m) - _point_fluence(rho, 0.0, -h, z, t, m)) / (2 * h)
    assert float(ph.reflectance(rho, z, t, m)) == pytest.approx(m.D * float(d), rel=1e-7)


@pytest.mark.parametrize("t", [30.0, 300.0])
def test_green_conserves_photons(t):
    """The infinite-medium impulse response integrates to c over space."""
    m = med()
    val, _ = integrate.quad(lambda r: 4 * np.pi * r * r * float(ph.green_inf(r, t, m)), 0, np.inf,
                            epsabs=0, epsrel=1e-12, limit=400)
    assert val == pytest.approx(m.c, rel=1e-10)


@pytest.mark.parametrize("r", [0.5, 3.0, 10.0])
def test_green_time_integral(r):
    """int_0^inf g(r,t) dt = 1 / (4 pi D r) (steady state of the diffusion equation)."""
    m = med()
    k = m.D * m.c
    tp = r * r / (6 * k)
    f = lambda t: float(ph.green_inf(r, t, m))
    v1, _ = integrate.quad(f, 0, tp, epsabs=0, epsrel=1e-12, limit=400)
    v2, _ = integrate.quad(f, tp, np.inf, epsabs=0, epsrel=1e-12, limit=400)
    assert v1 + v2 == pytest.approx(1.0 / (4 * np.pi * m.D * r), rel=1e-9)


def _total_escape(z, m):
    """int over the surface plane and all time of R for a source at depth z.

    Both image terms of R carry the same lateral factor exp(-rho^2/(4Dct)),
    whose plane integral is 4 pi D c t (Gaussian integral); the remaining
    time integral is done by adaptive quadrature.
    """
    k = m.D * m.c
    f = lambda t: float(ph.reflectance(0.0, z, t, m)) * 4 * np.pi * k * t
    tp = z * z / (10 * k)
    v1, _ = integrate.quad(f, 0, tp, epsabs=0, epsrel=1e-12, limit=400)
    v2, _ = integrate.quad(f, tp, np.inf, epsabs=0, epsrel=1e-12, limit=400)
    return v1 + v2


def test_escape_fraction_lossless_is_one():
    """With mua = 0 every photon eventually leaves through the surface: total flux = 1."""
    m = med(mua=0.0)
    assert _total_escape(4.0, m) == pytest.approx(1.0, rel=1e-7)


def test_escape_fraction_absorbing():
    """With absorption the escaping fraction is 1/2 [exp(-mueff z) + exp(-mueff (z + 2 zb))]."""
    m = med()
    z = 5.0
    want = 0.5 * (np.exp(-m.mueff * z) + np.exp(-m.mueff * (z + 2 * m.zb)))
    assert _total_escape(z, m) == pytest.approx(want, rel=1e-7)


@pytest.mark.parametrize("rho,z,t,rmin", [
    (0.0, 5.0, 300.0, 0.0), (3.0, 2.0, 100.0, 0.0), (1.0, 9.0, 1500.0, 0.0),
    (0.0, 1.0, 50.0, 0.5), (5.0, 16.0, 3000.0, 0.5), (0.25, 0.5, 12.0, 0.25)])
def test_closed_form_equals_numerical_convolution(rho, z, t, rmin):
    """Closed-form time convolution (Eq. 5) equals adaptive quadrature of its definition."""
    m = med(r_min=rmin)
    a = float(ph.conv_closed(rho, z, t, m))
    b = ph.conv_numeric(rho, z, t, m)
    assert a == pytest.approx(b, rel=1e-10)


@pytest.mark.parametrize("rho,z", [(0.0, 4.0), (3.0, 6.0), (8.0, 3.0)])
def test_cw_limit_of_time_domain_kernel(rho, z):
    """Time integral of Phi0 (*) R equals the CW Jacobian Phi0_CW * R_CW (Eq. 4 vs Eq. 5).

    The CW forms are the s = 0 Laplace transforms written independently:
    Phi0_CW = [exp(-mueff r1)/r1 - exp(-mueff r2)/r2] / (4 pi D),
    R_CW = [z (mueff + 1/r3) exp(-mueff r3)/r3^2 + (z+2zb)(mueff + 1/r4) exp(-mueff r4)/r4^2] / (4 pi).
    The sum over 400 bins of 50 ps (20 ns, > 40 absorption times) uses the
    same composite Gauss-Legendre bin rule as the kernel.
    """
    m = med()
    w = ph.binned_conv(rho, z, 400, 50.0, m)
    want = float(ph.fluence_cw(rho, z, m) * ph.reflectance_cw(rho, z, m))
    assert float(np.sum(w)) == pytest.approx(want, rel=1e-9)


def test_cw_forms_are_time_integrals():
    """Phi0_CW and R_CW are the time integrals of Phi0 and R (quadrature)."""
    m = med()
    rho, z = 2.0, 4.0
    f = integrate.quad(lambda t: float(ph.fluence(rho, z, t, m)), 0, np.inf, epsabs=0, epsrel=1e-12, limit=400)[0]
    r = integrate.quad(lambda t: float(ph.reflectance(rho, z, t, m)), 0, np.inf, epsabs=0, epsrel=1e-12, limit=400)[0]
    assert float(ph.fluence_cw(rho, z, m)) == pytest.approx(f, rel=1e-9)
    assert float(ph.reflectance_cw(rho, z, m)) == pytest.approx(r, rel=1e-9)


def test_bin_rule_integrates_polynomials_exactly():
    """8-node x 4-sub-interval Gauss-Legendre is exact for degree <= 15 on each piece."""
    ts, ws = ph.bin_nodes(3, 50.0)
    a, b = 150.0, 200.0
    for deg in (0, 5, 15):
        want = (b ** (deg + 1) - a ** (deg + 1)) / (deg + 1)
        assert float(np.sum(ws * ts**deg)) == pytest.approx(want, rel=1e-12)


def test_clamp_only_changes_near_singular_distances():
    """The r_min clamp leaves every distance >= r_min untouched."""
    m0 = med()
    m1 = med(r_min=0.5)
    rho = np.array([0.0, 0.0, 0.3, 2.0])
    z = np.array([1.0, 5.0, 1.0, 1.0])
    a = m0.distances(rho, z)
    b = m1.distances(rho, z)
    for ra, rb in zip(a, b):
        keep = ra >= 0.5
        assert np.array_equal(ra[keep], rb[keep])
        assert np.all(rb[~keep] == 0.5)
