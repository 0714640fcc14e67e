"""Diffusion-theory physics of the confocal sensitivity (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper builds its Jacobian from the analytic diffusion approximation of a
homogeneous semi-infinite slab (Section 3, "Computation of the Sensitivity
Matrix", Eq. 3-6) but does not print the Green's functions; it cites the
standard forms.  This module writes those textbook forms out:

* medium constants: c = c0/n, D = 1/(3(mua+musp')), mueff = sqrt(mua/D),
  isotropic source at depth z0 = 1/(mua+musp'), extrapolated boundary at
  z = -zb with zb = 2 A D and A = (1+Reff)/(1-Reff) (Groenhuis fit for Reff);
* Phi0(rho,z,t): fluence from a unit-energy impulse at (0,0,z0) with a
  negative image source at (0,0,-z0-2zb)  (first factor of Eq. 5);
* R(rho,z,t): Fick flux leaving the surface z=0 at the scan point from a unit
  point source at the voxel (depth z), image at -(z+2zb) (second factor of
  Eq. 5);
* their time convolution (Eq. 5), both by a closed form obtained from the
  Laplace transforms of the two factors and by direct numerical quadrature;
* the CW limits Phi0_CW, R_CW whose product is the CW Jacobian of Eq. 4;
* the composite Gauss-Legendre rule that integrates the convolution over a
  TCSPC time bin.

Units: mm, ps, 1/mm.  Distances r1..r4 are optionally clamped below at
r_min (a reading: the diffusion form diverges at the source point, and the
paper notes it fails near the surface, Section 3).
"""

import numpy as np
from scipy import integrate

C0_MM_PER_PS = 0.299792458  # speed of light in vacuum [mm/ps]


class Medium:
    """Background optics and the constants derived from them.

    mua, musp: absorption and reduced scattering [1/mm]; n: refractive index;
    z0: source depth (<=0 selects 1/(mua+musp)); r_min: distance clamp (0 =
    off).
    """

    def __init__(self, mua, musp, n, z0=0.0, r_min=0.0):
        self.mua = float(mua)
        self.musp = float(musp)
        self.n = float(n)
        self.c = C0_MM_PER_PS / self.n
        self.D = 1.0 / (3.0 * (self.mua + self.musp))
        self.mueff = np.sqrt(self.mua / self.D)
        n_ = self.n
        self.Reff = -1.440 / n_**2 + 0.710 / n_ + 0.668 + 0.0636 * n_
        self.A = (1.0 + self.Reff) / (1.0 - self.Reff)
        self.zb = 2.0 * self.A * self.D
        self.z0 = float(z0) if z0 > 0 else 1.0 / (self.mua + self.musp)
        self.r_min = float(r_min)

    def distances(self, rho, z):
        """(r1, r2, r3, r4) for lateral offset rho and voxel depth z.

        r1: source (0,0,z0) -> voxel;  r2: image source (0,0,-z0-2zb) -> voxel;
        r3: voxel -> scan point on the surface;  r4: voxel image
        (depth -(z+2zb)) -> scan point.  Each is clamped to >= r_min.
        """
        rho = np.asarray(rho, dtype=np.float64)
        z = np.asarray(z, dtype=np.float64)
        r1 = np.sqrt(rho**2 + (z - self.z0) ** 2)
        r2 = np.sqrt(rho**2 + (z + self.z0 + 2.0 * self.zb) ** 2)
        r3 = np.sqrt(rho**2 + z**2)
        r4 = np.sqrt(rho**2 + (z + 2.0 * self.zb) ** 2)
        rm = self.r_min
        return (np.maximum(r1, rm), np.maximum(r2, rm),
                np.maximum(r3, rm), np.maximum(r4, rm))


def green_inf(r, t, med):
    """Infinite-medium diffusion fluence (no absorption) of a unit impulse.

    g(r,t) = c (4 pi D c t)^(-3/2) exp(-r^2 / (4 D c t)), zero for t <= 0.
    """
    t = np.asarray(t, dtype=np.float64)
    k = med.D * med.c
    tt = np.where(t > 0, t, 1.0)
    out = med.c * (4.0 * np.pi * k * tt) ** -1.5 * np.exp(-np.asarray(r) ** 2 / (4.0 * k * tt))
    return np.where(t > 0, out, 0.0)


def fluence(rho, z, t, med):
    """Phi0(rho,z,t): fluence at the voxel from the scan-point source (Eq. 5).

    Semi-infinite medium, extrapolated boundary: real source at depth z0,
    negative image at -(z0 + 2 zb); absorption as exp(-mua c t).
    """
    r1, r2, _, _ = med.distances(rho, z)
    return np.exp(-med.mua * med.c * np.asarray(t)) * (green_inf(r1, t, med) - green_inf(r2, t, med))


def reflectance(rho, z, t, med):
    """R(rho,z,t): flux detected at the scan point from a unit source at the voxel.

    Fick flux D dPhi/dz at z = 0 of a unit impulse at depth z with its negative
    image at -(z + 2 zb):
      R = 1/2 (4 pi D c)^(-3/2) t^(-5/2) exp(-mua c t)
          [ z exp(-r3^2/4Dct) + (z + 2 zb) exp(-r4^2/4Dct) ].
    """
    _, _, r3, r4 = med.distances(rho, z)
    z = np.asarray(z, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    k = med.D * med.c
    tt = np.where(t > 0, t, 1.0)
    val = (0.5 * (4.0 * np.pi * k) ** -1.5 * tt**-2.5 * np.exp(-med.mua * med.c * tt)
           * (z * np.exp(-r3**2 / (4 * k * tt)) + (z + 2 * med.zb) * np.exp(-r4**2 / (4 * k * tt))))
    return np.where(t > 0, val, 0.0)


def conv_numeric(rho, z, t, med, epsrel=1e-13):
    """(Phi0 (*)_t R)(rho,z,t) = int_0^t Phi0(t') R(t - t') dt' by adaptive quadrature (Eq. 5).

    Scalar rho, z, t.  Used only to pin the closed form.
    """
    if t <= 0:
        return 0.0
    f = lambda tp: float(fluence(rho, z, tp, med) * reflectance(rho, z, t - tp, med))
    # both factors vanish smoothly at their t -> 0 ends; split at the midpoint
    # and at the two transit-time peaks so the adaptive rule sees them
    r1, r2, r3, r4 = med.distances(rho, z)
    k = med.D * med.c
    pts = sorted({x for x in (r1**2 / (6 * k), t - r3**2 / (10 * k), 0.5 * t) if 0 < x < t})
    val, _ = integrate.quad(f, 0.0, t, points=pts or None, limit=500, epsabs=0.0, epsrel=epsrel)
    return val


def conv_closed(rho, z, t, med):
    """Closed form of (Phi0 (*)_t R)(rho,z,t) (Eq. 5).

    With q = sqrt(s/(Dc)) the Laplace transforms of the two factors (without
    the common absorption factor, which leaves the convolution as exp(-mua c t))
    are
        L[g(r_i)] = exp(-r_i q) / (4 pi D r_i),
        L[R_j]    = z_j (1 + r_j q) exp(-r_j q) / (4 pi r_j^3),
    so each product inverts with L^-1[exp(-a q)] = h0(a,t) and
    L^-1[q exp(-a q)] = h1(a,t) = -dh0/da:
        h0(a,t) = a / (2 sqrt(pi Dc)) t^(-3/2) exp(-a^2/(4Dct))
        h1(a,t) = 1 / (2 sqrt(pi Dc)) t^(-3/2) exp(-a^2/(4Dct)) (a^2/(2Dct) - 1)
    Result: exp(-mua c t) sum_{i in (1,2)} sum_{j in (3,4)} sigma_i z_j /
    (16 pi^2 D r_i r_j^3) [h0(r_i + r_j, t) + r_j h1(r_i + r_j, t)], with
    sigma_1 = +1, sigma_2 = -1, z_3 = z, z_4 = z + 2 zb.
    """
    r1, r2, r3, r4 = med.distances(rho, z)
    z = np.asarray(z, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    k = med.D * med.c
    tt = np.where(t > 0, t, 1.0)
    base = 1.0 / (2.0 * np.sqrt(np.pi * k)) * tt**-1.5
    total = 0.0
    for sig, ri in ((1.0, r1), (-1.0, r2)):
        for zj, rj in ((z, r3), (z + 2 * med.zb, r4)):
            a = ri + rj
            e = np.exp(-a**2 / (4 * k * tt))
            h0 = a * base * e
            h1 = base * e * (a**2 / (2 * k * tt) - 1.0)
            total = total + sig * zj / (16 * np.pi**2 * med.D * ri * rj**3) * (h0 + rj * h1)
    return np.where(t > 0, np.exp(-med.mua * med.c * tt) * total, 0.0)


def fluence_cw(rho, z, med):
    """Phi0_CW: time integral of Phi0 (CW fluence of the Eq. 4 Jacobian)."""
    r1, r2, _, _ = med.distances(rho, z)
    m = med.mueff
    return (np.exp(-m * r1) / r1 - np.exp(-m * r2) / r2) / (4 * np.pi * med.D)


def reflectance_cw(rho, z, med):
    """R_CW: time integral of R (CW reflectance of the Eq. 4 Jacobian)."""
    _, _, r3, r4 = med.distances(rho, z)
    z = np.asarray(z, dtype=np.float64)
    m = med.mueff
    zz = z + 2 * med.zb
    return (z * (m + 1 / r3) * np.exp(-m * r3) / r3**2 + zz * (m + 1 / r4) * np.exp(-m * r4) / r4**2) / (4 * np.pi)


def gauss_legendre(nodes):
    """Nodes and weights of the n-point Gauss-Legendre rule on [-1, 1]."""
    return np.polynomial.legendre.leggauss(nodes)


def bin_nodes(k, dt, nodes=8, sub=4):
    """Abscissae and weights of the composite rule for bin [k dt, (k+1) dt).

    The bin is split into `sub` equal sub-intervals, each integrated with an
    `nodes`-point Gauss-Legendre rule.  (Reading: the measurement of bin k is
    the integral of the response over the bin, as a TCSPC histogram counts
    every photon arriving in it.)
    """
    x, w = gauss_legendre(nodes)
    h = dt / sub
    ts, ws = [], []
    for s in range(sub):
        a = k * dt + s * h
        ts.append(a + 0.5 * h * (x + 1.0))
        ws.append(0.5 * h * w)
    return np.concatenate(ts), np.concatenate(ws)


def binned_conv(rho, z, nt, dt, med, nodes=8, sub=4):
    """int over bin k of (Phi0 (*) R)(rho, z, t) dt for k = 0..nt-1.

    rho, z broadcastable arrays; returns shape (nt,) + broadcast shape.
    """
    rho = np.asarray(rho, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    shape = np.broadcast(rho, z).shape
    out = np.empty((nt,) + shape)
    for k in range(nt):
        ts, ws = bin_nodes(k, dt, nodes, sub)
        acc = np.zeros(shape)
        for t, w in zip(ts, ws):
            acc += w * conv_closed(rho, z, t, med)
        out[k] = acc
    return out


# ---------------------------------------------------------------------------
# Fluorescence mode (Section 5, simulator paragraph: separate excitation and
# emission optics, the response convolved with an exponential of the
# fluorescence lifetime).
#
# Reading: a fluorophore at the voxel is excited by the fluence Phi0 of the
# excitation light (excitation optics, source depth z0 and extrapolated
# boundary of the excitation medium), re-emits with the normalised lifetime
# density L_tau(t) = exp(-t/tau)/tau (quantum yield and concentration are the
# unknown), and the emission reaches the scan point as the flux R of the
# emission medium.  The time response is the double convolution
#     f(t) = (Phi0_ex (*)_t L_tau (*)_t R_em)(rho, z, t),
# tau = 0 meaning instantaneous emission (L_tau = delta).  It is evaluated
# through the convolution theorem: the Laplace transform of f is the product
# of the three factors' transforms (each in closed form, below), inverted
# numerically with the fixed-Talbot rule.  The bin integral is the difference
# of the cumulative response int_0^t f at the bin edges, inverted from F(s)/s.
# ---------------------------------------------------------------------------

TALBOT_TERMS = 24


def fluorescence_laplace(s, rho, z, med_ex, med_em, tau):
    """F(s) = L[Phi0_ex](s) L[L_tau](s) L[R_em](s) for complex s (Re s > -min absorption rate).

    With q = sqrt((s + mua c)/(D c)) of each medium (absorption exp(-mua c t)
    shifts s), the transforms are
        L[Phi0_ex] = exp(-r1 q_ex)/(4 pi D_ex r1) - exp(-r2 q_ex)/(4 pi D_ex r2),
        L[R_em]    = sum_{j in (3,4)} z_j (1 + r_j q_em) exp(-r_j q_em)/(4 pi r_j^3),
        L[L_tau]   = 1/(1 + s tau),
    r1, r2 from the excitation medium, r3, r4 (z_3 = z, z_4 = z + 2 zb_em)
    from the emission medium.
    """
    s = np.asarray(s, dtype=np.complex128)
    r1, r2, _, _ = med_ex.distances(rho, z)
    _, _, r3, r4 = med_em.distances(rho, z)
    z = np.asarray(z, dtype=np.float64)
    q_ex = np.sqrt((s + med_ex.mua * med_ex.c) / (med_ex.D * med_ex.c))
    q_em = np.sqrt((s + med_em.mua * med_em.c) / (med_em.D * med_em.c))
    src = (np.exp(-r1 * q_ex) / r1 - np.exp(-r2 * q_ex) / r2) / (4.0 * np.pi * med_ex.D)
    z4 = z + 2.0 * med_em.zb
    det = (z * (1.0 + r3 * q_em) * np.exp(-r3 * q_em) / r3**3
           + z4 * (1.0 + r4 * q_em) * np.exp(-r4 * q_em) / r4**3) / (4.0 * np.pi)
    return src * det / (1.0 + s * tau)


def talbot_inverse(F, t, m=TALBOT_TERMS):
    """Inverse Laplace transform f(t) by the fixed-Talbot rule (Abate and Valko, 2004).

    The Bromwich contour is deformed to s(theta) = r theta (cot theta + i),
    -pi < theta < pi, r = 2m/(5t), which encloses every singularity on the
    negative real axis; by conjugate symmetry f(t) = (r/pi) int_0^pi
    Re[exp(t s) F(s) (1 + i sigma(theta))] dtheta with sigma(theta) = theta +
    (theta cot theta - 1) cot theta, and the trapezoidal rule with step pi/m
    gives
        f(t) ~ (r/m) [ exp(r t) F(r)/2 + sum_{k=1}^{m-1} Re(exp(t s_k) F(s_k) (1 + i sigma_k)) ].
    F maps a complex scalar to an array (or scalar); t > 0 scalar.
    """
    t = float(t)
    r = 2.0 * m / (5.0 * t)
    total = 0.5 * np.exp(r * t) * np.real(F(complex(r, 0.0)))
    for k in range(1, m):
        th = k * np.pi / m
        cot = np.cos(th) / np.sin(th)
        s = r * th * complex(cot, 1.0)
        sigma = th + (th * cot - 1.0) * cot
        total = total + np.real(np.exp(t * s) * F(s) * complex(1.0, sigma))
    return r / m * total


def fluorescence_response(rho, z, t, med_ex, med_em, tau, m=TALBOT_TERMS):
    """f(rho, z, t) = (Phi0_ex (*) L_tau (*) R_em)(t) for scalar t > 0."""
    return talbot_inverse(lambda s: fluorescence_laplace(s, rho, z, med_ex, med_em, tau), t, m)


def fluorescence_cumulative(rho, z, t, med_ex, med_em, tau, m=TALBOT_TERMS):
    """int_0^t f(rho, z, t') dt' (the transform F(s)/s), scalar t >= 0."""
    if t <= 0:
        return np.zeros(np.broadcast(np.asarray(rho), np.asarray(z)).shape)
    return talbot_inverse(lambda s: fluorescence_laplace(s, rho, z, med_ex, med_em, tau) / s, t, m)


def binned_fluorescence(rho, z, nt, dt, med_ex, med_em, tau, m=TALBOT_TERMS):
    """int over bin k of f(rho, z, t) dt for k = 0..nt-1 (cumulative differences at the edges).

    rho, z broadcastable arrays; returns shape (nt,) + broadcast shape.
    """
    edges = [fluorescence_cumulative(rho, z, k * dt, med_ex, med_em, tau, m) for k in range(nt + 1)]
    return np.stack([edges[k + 1] - edges[k] for k in range(nt)])
