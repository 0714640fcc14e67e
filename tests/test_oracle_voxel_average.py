"""Pins of the voxel-averaged kernel (time-domain forward model integrated over each voxel).

The oracle averages the binned kernel over the voxel with a tensor
Gauss-Legendre rule.  The tests hold that rule to facts fixed elsewhere: the
one-node rule is the centre value, the rule integrates low-degree
polynomials in (x, y, z) exactly over the right box, and it matches an
adaptive cubature of the CW Jacobian Phi0_CW R_CW over near-surface voxels.
"""

import numpy as np
import pytest
from scipy import integrate

from oracle import operators as op
from oracle import physics as ph


def med():
    return ph.Medium(0.01, 1.0, 1.4, r_min=0.5)


def test_one_node_is_centre_value():
    g = op.Grid(6, 3, 8, 1.0, 1.0, 1.0, 50.0)
    w0 = op.kernel_offsets(g, med())
    w1 = op.kernel_offsets_averaged(g, med(), 3, 1)
    assert np.allclose(w1, w0, rtol=1e-14, atol=0.0)


@pytest.mark.parametrize("nodes", [2, 3, 5])
def test_rule_is_exact_for_polynomials(nodes):
    """(1/V) int (x^2 + y^2) z^3 over the box = (<x^2> + <y^2>) <z^3>, <x^2> = x0^2 + h^2/12,
    <z^3> = z0^3 + z0 hz^2/4 (degree <= 3 per axis: exact from two nodes)."""
    g = op.Grid(4, 2, 1, 0.7, 0.9, 1.2, 10.0, dy=1.1)
    qx, qy, z0 = 3, 2, 1.7
    got = op.voxel_average(lambda rho, z: rho**2 * z**3, qx, qy, z0, g, nodes)
    x0, y0 = qx * g.dx, qy * g.dy
    want = (x0**2 + g.dx**2 / 12 + y0**2 + g.dy**2 / 12) * (z0**3 + z0 * g.dz**2 / 4)
    assert got == pytest.approx(want, rel=1e-14)


@pytest.mark.parametrize("qx,qy", [(1, 0), (2, 1), (3, 3)])
def test_cw_jacobian_average_matches_cubature(qx, qy):
    """Top-layer voxels next to the source: the 8-node rule against adaptive cubature."""
    g = op.Grid(4, 1, 1, 1.0, 1.0, 1.0, 50.0)
    m = ph.Medium(0.01, 1.0, 1.4)  # no distance clamp: the voxels do not contain the source
    cw = lambda rho, z: ph.fluence_cw(rho, z, m) * ph.reflectance_cw(rho, z, m)
    got = float(op.voxel_average(cw, qx, qy, g.depths[0], g, 8))
    f = lambda z, y, x: float(cw(np.hypot(x, y), z))
    want, _ = integrate.tplquad(f, qx - 0.5, qx + 0.5, qy - 0.5, qy + 0.5, 0.5, 1.5, epsabs=0.0, epsrel=1e-10)
    assert got == pytest.approx(want, rel=1e-6)
    # and the centre value is measurably off there (the reason for averaging)
    assert abs(float(cw(np.hypot(qx, qy), 1.0)) - want) > 1e-3 * want


def test_only_the_requested_layers_change():
    g = op.Grid(5, 4, 6, 1.0, 1.0, 1.0, 50.0)
    w0 = op.kernel_offsets(g, med())
    w2 = op.kernel_offsets_averaged(g, med(), 2, 3)
    assert np.array_equal(w2[:, 2:], w0[:, 2:])
    assert np.abs(w2[:, :2] - w0[:, :2]).max() > 1e-3 * np.abs(w0).max()
    # mirror symmetry and the x <-> y swap survive the averaging (dx == dy)
    assert np.array_equal(w2, w2[:, :, ::-1, :])
    assert np.allclose(w2, np.swapaxes(w2, 2, 3), rtol=1e-13, atol=0.0)  # node sums in another order
