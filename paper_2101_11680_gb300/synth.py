"""Seeded synthetic inputs: absorbing phantoms and Poisson measurement noise.

This module is the one piece shared by the CUDA path's tests/bench and the
FP64 oracle.  It holds no part of the reconstruction method: it voxelises
geometric shapes and draws counting noise, nothing else.  All randomness
comes from ``numpy.random.Generator(PCG64(seed))``.

Voxel centres: lateral x_i = i*dx, y_i = i*dy (i < n); depth
z_j = z_first + j*dz (j < nz).  A voxel takes a shape's value when its centre
lies inside the shape; overlapping shapes take the maximum.

The paper's own phantoms (vasculature, discs and lines at several depths,
Section 6 "3D Image Reconstruction"; spheres are not used there) are not
available; these seeded shapes stand in for them.
"""

import numpy as np


def _rng(seed):
    return np.random.Generator(np.random.PCG64(int(seed)))


def _centres(n, nz, dx, dy, dz, z_first):
    x = np.arange(n) * dx
    y = np.arange(n) * dy
    z = z_first + np.arange(nz) * dz
    return np.meshgrid(z, y, x, indexing="ij")  # each [nz][n][n]


def phantom_spheres(n, nz, dx, dz, z_first, seed, radius=1.5, value=0.01,
                    depths=(5.0, 9.0), dy=None):
    """Spheres of `radius` mm and `value` 1/mm, one per entry of `depths` [mm].

    Lateral centres are continuous uniform in [radius+1, (n-1)*dx - radius - 1].
    Returns float64 [nz][n][n].
    """
    dy = dx if dy is None else dy
    rng = _rng(seed)
    zz, yy, xx = _centres(n, nz, dx, dy, dz, z_first)
    vol = np.zeros((nz, n, n))
    lo = radius + 1.0
    for zc in depths:
        xc = rng.uniform(lo, (n - 1) * dx - lo)
        yc = rng.uniform(lo, (n - 1) * dy - lo)
        inside = (xx - xc) ** 2 + (yy - yc) ** 2 + (zz - zc) ** 2 <= radius**2
        vol = np.where(inside, np.maximum(vol, value), vol)
    return vol


def _rotation(rng):
    """Uniform random 3-D rotation (QR of a Gaussian matrix, sign-fixed)."""
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def phantom_shapes(n, nz, dx, dz, z_first, seed, max_shapes=8,
                   value_range=(0.005, 0.02), dy=None):
    """1..max_shapes random ellipsoids and tubes (each with probability 1/2).

    Ellipsoid: centre uniform in the volume, semi-axes U[1,4] mm, random
    rotation.  Tube: the segment between two uniform interior points, radius
    U[0.5,2] mm.  Value U[value_range] 1/mm.  Returns float64 [nz][n][n].
    """
    dy = dx if dy is None else dy
    rng = _rng(seed)
    zz, yy, xx = _centres(n, nz, dx, dy, dz, z_first)
    pts = np.stack([xx, yy, zz], axis=-1)  # [nz][n][n][3]
    lo = np.array([0.0, 0.0, z_first])
    hi = np.array([(n - 1) * dx, (n - 1) * dy, z_first + (nz - 1) * dz])
    vol = np.zeros((nz, n, n))
    count = int(rng.integers(1, max_shapes + 1))
    for _ in range(count):
        val = rng.uniform(*value_range)
        if rng.uniform() < 0.5:
            c = rng.uniform(lo, hi)
            ax = rng.uniform(1.0, 4.0, size=3)
            rot = _rotation(rng)
            loc = (pts - c) @ rot  # coordinates in the ellipsoid frame
            inside = np.sum((loc / ax) ** 2, axis=-1) <= 1.0
        else:
            a = rng.uniform(lo, hi)
            b = rng.uniform(lo, hi)
            r = rng.uniform(0.5, 2.0)
            ab = b - a
            L2 = float(ab @ ab)
            s = np.clip(((pts - a) @ ab) / max(L2, 1e-30), 0.0, 1.0)
            d = pts - (a + s[..., None] * ab)
            inside = np.sum(d * d, axis=-1) <= r * r
        vol = np.where(inside, np.maximum(vol, val), vol)
    return vol


def poisson_noise(m, peak, seed):
    """Counting noise at a given peak: Poisson(m * peak / max m) * max m / peak.

    (Reading of "Poisson noise at peak P counts": the largest clean bin is
    scaled to P expected counts.)  m must be non-negative.  float64 out.
    """
    m = np.asarray(m, dtype=np.float64)
    mx = float(m.max())
    if mx <= 0:
        return m.copy()
    rng = _rng(seed)
    lam = np.clip(m, 0.0, None) * (peak / mx)
    return rng.poisson(lam).astype(np.float64) * (mx / peak)


def dark_count_noise(m, rate_cps, integration_s, dark_cps, seed):
    """Photon counting with detector dark counts (the noise of the paper's
    multiplexing simulations, Section 5: Poisson photon noise at a detected
    count rate, plus dark counts at a fixed rate, 200 counts/s for its SPAD).

    m [T][...]: clean non-negative measurement, time bins on the first axis.
    Reading: the brightest measurement (largest sum over its T bins) collects
    rate_cps * integration_s photons; every measurement collects
    dark_cps * integration_s dark counts, spread evenly over its T bins.
    Returns (counts, unit, dark_per_bin): counts ~ Poisson(m / unit +
    dark_per_bin) (int64), with unit = max_x sum_t m / (rate_cps *
    integration_s); (counts - dark_per_bin) * unit is an unbiased estimate of m.
    """
    m = np.asarray(m, dtype=np.float64)
    nt = m.shape[0]
    total = m.reshape(nt, -1).sum(axis=0).max()
    photons = float(rate_cps) * float(integration_s)
    unit = float(total) / photons if total > 0 and photons > 0 else 1.0
    dark_per_bin = float(dark_cps) * float(integration_s) / nt
    rng = _rng(seed)
    lam = np.clip(m, 0.0, None) / unit + dark_per_bin
    return rng.poisson(lam), unit, dark_per_bin


# (input channels, output channels) of the four 3x3x3 layers of the learned prox
LEARNED_LAYERS = ((1, 16), (16, 16), (16, 16), (16, 1))


def learned_init(stages, seed):
    """Random starting parameters of the learned solver, flat float64.

    He-normal weights std sqrt(2 / (27 ci)) (the last layer's scaled by 0.1, so
    the untrained prox is close to the identity), zero biases, step sizes 1.
    Layout: w1 [16][1][27], b1 [16], w2 [16][16][27], b2 [16], w3 [16][16][27],
    b3 [16], w4 [1][16][27], b4 [1], eta [stages].
    """
    rng = _rng(seed)
    parts = []
    for li, (ci, co) in enumerate(LEARNED_LAYERS):
        std = np.sqrt(2.0 / (ci * 27))
        if li == len(LEARNED_LAYERS) - 1:
            std *= 0.1
        parts += [np.ravel(rng.standard_normal((co, ci, 27)) * std), np.zeros(co)]
    parts.append(np.ones(int(stages)))
    return np.concatenate(parts)
