"""Confocal sensitivity kernel and the convolutional forward/adjoint (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Geometry.  The confocal scan points (source = detector, Section 4 "Confocal
ToF-DOT") sit on the lateral voxel-column centres x_i = i dx, y_i = i dy,
i < N, at the surface z = 0.  Voxel depths are z_j = z_first + j dz, j < Z.
Time bin k covers [k dt, (k+1) dt) with t = 0 at pulse emission.

The Jacobian of Eq. 6 restricted to confocal measurements is
    J[(k,y,x), (j,y',x')] = dx dy dz * int_bin_k (Phi0 (*)_t R)(rho, z_j, t) dt,
    rho = |(x - x', y - y')|,
which depends only on the lateral offset: the convolutional approximation
(Eq. 9 for one depth, Eq. 11 summed over depth).  Two lateral boundary modes:

* linear (default): m[k][y][x] = sum_j sum_{y',x' < N} W[k][j][y-y'][x-x'] mu[j][y'][x'],
  offsets in [-(N-1), N-1], no truncation; evaluated by FFT on a P x P grid,
  P = max(32, smallest power of two >= 2N), with the kernel placed at offset index
  p -> p mod P (zero at every index no offset reaches), then cropped to N x N;
* circular: P = N, minimum-image offsets (the paper's "doubly circulant"
  statement, Section 4).
"""

import numpy as np

from .physics import binned_conv, binned_fluorescence


class Grid:
    """Lateral N x N scan, Z depths, T bins; pitches in mm, dt in ps."""

    def __init__(self, n, nz, nt, dx, dz, z_first, dt, dy=None, mode="linear"):
        self.n = int(n)
        self.nz = int(nz)
        self.nt = int(nt)
        self.dx = float(dx)
        self.dy = float(dx if dy is None else dy)
        self.dz = float(dz)
        self.z_first = float(z_first)
        self.dt = float(dt)
        if mode not in ("linear", "circular"):
            raise ValueError(mode)
        self.mode = mode
        if mode == "linear":
            # any P >= 2N-1 gives the same linear convolution; the solvers work
            # on the P x P periodic grid, so P is fixed here: the smallest power
            # of two >= 2N, and at least 32.
            p = 32
            while p < 2 * self.n:
                p *= 2
            self.p = p
        else:
            self.p = self.n

    @property
    def depths(self):
        return self.z_first + self.dz * np.arange(self.nz)

    @property
    def voxel_volume(self):
        return self.dx * self.dy * self.dz


def kernel_offsets(grid, med, nodes=8, sub=4):
    """W[k][j][oy + N-1][ox + N-1] for lateral offsets oy, ox in [-(N-1), N-1].

    Evaluated on the quadrant |oy|, |ox| < N (rho depends on |offset| only)
    and mirrored.  Scaled by the voxel volume (Born: absorbed power is
    dmua * Phi0 * volume).
    """
    n = grid.n
    a = np.arange(n)
    rho = np.sqrt((a[None, :] * grid.dx) ** 2 + (a[:, None] * grid.dy) ** 2)  # [qy][qx]
    z = grid.depths[:, None, None]
    quad = binned_conv(rho[None, :, :], z, grid.nt, grid.dt, med, nodes, sub) * grid.voxel_volume
    return _mirror(quad, n)


def _mirror(quad, n):
    """[T][Z][|oy|][|ox|] quadrant -> [T][Z][2N-1][2N-1] full offsets."""
    idx = np.abs(np.arange(-(n - 1), n))
    return quad[:, :, idx][:, :, :, idx]


def voxel_average(point, qx, qy, z, grid, nodes):
    """(1/V) int over the voxel of point(rho(x, y), z') dV, tensor Gauss-Legendre rule.

    The voxel at lateral offset (qx dx, qy dy) from the scan point and centre
    depth z spans +-dx/2, +-dy/2, +-dz/2 around that centre; ``nodes``
    Gauss-Legendre nodes per axis (weights sum to 2 on [-1, 1], so the
    average divides by 8).  point(rho, z) may return extra leading axes.
    """
    x, w = np.polynomial.legendre.leggauss(nodes)
    acc = 0.0
    for a in range(nodes):
        for b in range(nodes):
            for c in range(nodes):
                px = qx * grid.dx + 0.5 * grid.dx * x[a]
                py = qy * grid.dy + 0.5 * grid.dy * x[b]
                pz = z + 0.5 * grid.dz * x[c]
                acc = acc + w[a] * w[b] * w[c] / 8.0 * point(np.sqrt(px * px + py * py), pz)
    return acc


def kernel_offsets_averaged(grid, med, layers, nodes, emission=None):
    """Kernel with the first ``layers`` depth layers averaged over the voxel volume.

    Reading of the time-domain forward model m = int_v J mu dr_v with mu
    constant on each voxel: the exact voxel weight is the integral of J over
    the voxel, of which the centre value times the volume is the midpoint
    rule.  Near the surface (and the source) J varies strongly inside one
    voxel, so those layers take the voxel average with ``nodes`` Gauss-Legendre
    nodes per axis; deeper layers keep the centre value.  ``emission`` = None
    for the absorption kernel (``binned_conv``), else (med_em, tau) for the
    fluorescence kernel (``binned_fluorescence``).
    """
    n = grid.n
    if emission is None:
        point = lambda rho, z: binned_conv(rho, z, grid.nt, grid.dt, med)
    else:
        med_em, tau = emission
        point = lambda rho, z: binned_fluorescence(rho, z, grid.nt, grid.dt, med, med_em, tau)
    a = np.arange(n)
    qx, qy = a[None, :], a[:, None]
    rho = np.sqrt((qx * grid.dx) ** 2 + (qy * grid.dy) ** 2)
    z = grid.depths[:, None, None]
    quad = point(rho[None, :, :], z)  # [T][Z][qy][qx]
    for j in range(min(layers, grid.nz)):
        quad[:, j] = voxel_average(point, qx, qy, grid.depths[j], grid, nodes)
    return _mirror(quad * grid.voxel_volume, n)


def kernel_offsets_fluorescence(grid, med_ex, med_em, tau):
    """Fluorescence-mode kernel on the offset grid (same layout as ``kernel_offsets``).

    W[k][j][oy][ox] = dx dy dz * int_bin_k (Phi0_ex (*) L_tau (*) R_em)(rho, z_j, t) dt
    (Section 5: excitation and emission optics, lifetime tau in ps), the bin
    integral taken exactly as differences of the cumulative response.
    """
    n = grid.n
    a = np.arange(n)
    rho = np.sqrt((a[None, :] * grid.dx) ** 2 + (a[:, None] * grid.dy) ** 2)
    z = grid.depths[:, None, None]
    quad = binned_fluorescence(rho[None, :, :], z, grid.nt, grid.dt, med_ex, med_em, tau) * grid.voxel_volume
    return _mirror(quad, n)


def periodic_kernel(w_off, grid):
    """Place the offset kernel on the P x P periodic grid ([T][Z][P][P])."""
    n, p = grid.n, grid.p
    t, z = w_off.shape[:2]
    out = np.zeros((t, z, p, p))
    if grid.mode == "linear":
        o = np.arange(-(n - 1), n)
        pos = np.mod(o, p)
        out[:, :, pos[:, None], pos[None, :]] = w_off
    else:
        o = np.arange(p)
        mi = np.where(o <= p // 2, o, o - p)  # minimum-image offset
        src = mi + (n - 1)
        out[:] = w_off[:, :, src[:, None], src[None, :]]
    return out


def kernel_spectrum(w_off, grid):
    """W_hat[k][j][ky][kx] = 2-D DFT of the periodic kernel (complex128)."""
    return np.fft.fft2(periodic_kernel(w_off, grid), axes=(-2, -1))


def _pad(v, grid):
    p, n = grid.p, grid.n
    out = np.zeros(v.shape[:-2] + (p, p))
    out[..., :n, :n] = v
    return out


def forward_fft(w_hat, mu, grid):
    """m = sum_z W_z (*) mu_z via FFT (Eq. 11): pad, transform, contract over depth, invert, crop."""
    n = grid.n
    mu_hat = np.fft.fft2(_pad(mu, grid), axes=(-2, -1))
    m_hat = np.einsum("tzyx,zyx->tyx", w_hat, mu_hat)
    return np.fft.ifft2(m_hat, axes=(-2, -1)).real[:, :n, :n]


def adjoint_fft(w_hat, m, grid):
    """vol = A^T m via FFT: pad, transform, contract with conj(W_hat) over time, invert, crop."""
    n = grid.n
    m_hat = np.fft.fft2(_pad(m, grid), axes=(-2, -1))
    v_hat = np.einsum("tzyx,tyx->zyx", np.conj(w_hat), m_hat)
    return np.fft.ifft2(v_hat, axes=(-2, -1)).real[:, :n, :n]


def _offset_index(d, grid):
    """Index into the offset axis of kernel_offsets for lateral difference d."""
    n = grid.n
    if grid.mode == "linear":
        return d + (n - 1)
    mi = np.mod(d, n)
    mi = np.where(mi <= n // 2, mi, mi - n)
    return mi + (n - 1)


def forward_direct(w_off, mu, grid):
    """m[k][y][x] = sum_j sum_{y',x'} W[k][j][y-y'][x-x'] mu[j][y'][x'] by direct summation (Eq. 11)."""
    n = grid.n
    y = np.arange(n)
    m = np.zeros((w_off.shape[0], n, n))
    for yp in range(n):
        iy = _offset_index(y - yp, grid)
        for xp in range(n):
            col = mu[:, yp, xp]
            if not np.any(col):
                continue
            ix = _offset_index(y - xp, grid)
            blk = w_off[:, :, iy[:, None], ix[None, :]]  # [T][Z][y][x]
            m += np.einsum("tzyx,z->tyx", blk, col)
    return m


def adjoint_direct(w_off, m, grid):
    """vol[j][y'][x'] = sum_k sum_{y,x} W[k][j][y-y'][x-x'] m[k][y][x] by direct summation."""
    n = grid.n
    y = np.arange(n)
    vol = np.zeros((w_off.shape[1], n, n))
    for yp in range(n):
        iy = _offset_index(y - yp, grid)
        for xp in range(n):
            ix = _offset_index(y - xp, grid)
            blk = w_off[:, :, iy[:, None], ix[None, :]]
            vol[:, yp, xp] = np.einsum("tzyx,tyx->z", blk, m)
    return vol


def dense_jacobian(grid, med, nodes=8, sub=4):
    """Confocal Jacobian J (Eq. 2, Eq. 6) assembled entry by entry from positions.

    Rows: measurement index (k, y, x) flattened k-major; columns: voxel index
    (j, y', x') flattened j-major.  Entry = voxel volume * bin integral of the
    source->voxel->detector time convolution at the scan point (x dx, y dy, 0)
    and voxel centre (x' dx, y' dy, z_j).  No offset table or FFT is used.
    """
    n = grid.n
    iy, ix = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    sy = iy.ravel()
    sx = ix.ravel()
    ddx = sx[:, None] - sx[None, :]
    ddy = sy[:, None] - sy[None, :]
    if grid.mode == "circular":
        ddx = np.mod(ddx, n)
        ddx = np.where(ddx <= n // 2, ddx, ddx - n)
        ddy = np.mod(ddy, n)
        ddy = np.where(ddy <= n // 2, ddy, ddy - n)
    rho = np.sqrt((ddx * grid.dx) ** 2 + (ddy * grid.dy) ** 2)  # [scan][voxel column]
    z = grid.depths[:, None, None]
    vals = binned_conv(rho[None], z, grid.nt, grid.dt, med, nodes, sub) * grid.voxel_volume
    # vals: [T][Z][scan][col] -> J[(k,scan), (j,col)]
    t, zn, s, c = vals.shape
    return vals.transpose(0, 2, 1, 3).reshape(t * s, zn * c)
