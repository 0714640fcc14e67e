"""Reconstruction solvers on the convolutional operator (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper poses reconstruction as the regularised inverse of Eq. 7 (and the
L1 problem of Eq. 8, solved there by FISTA, with one weight per depth in
Eq. 10).  The solvers here are
(a) per-frequency Tikhonov, the closed-form minimiser of
    ||K x - pad(m)||^2 + lam ||x||^2 on the P x P periodic grid, and
(b) scaled-form ADMM for
    min_x 1/2 ||C K x - m||^2 + beta ||D x||_1 + indicator{x >= 0, x = 0 off S}
with C the crop to the measured N x N scan, D forward differences (lateral
periodic on the P grid, axial Neumann), S = [0,N)^2 x all depths, and
(c) FISTA for the layer-weighted L1 problem of Eq. 10,
    min_x 1/2 ||A x - m||^2 + sum_z lam(z) ||x_z||_1,   A = C K.
All are written step by step in the order the algorithm states them.

Conventions: numpy FFT (X[k] = sum x[n] exp(-2 pi i k n / P)), so the
periodic forward difference x[n+1] - x[n] has symbol exp(2 pi i k/P) - 1.
"""

import numpy as np

from .operators import _pad, adjoint_fft, forward_fft


def gram(w_hat):
    """G(f) = W_hat(f)^H W_hat(f), shape [P][P][Z][Z] (per lateral frequency)."""
    w = np.moveaxis(w_hat, (0, 1), (-2, -1))  # [ky][kx][T][Z]
    return np.einsum("yxtz,yxtw->yxzw", np.conj(w), w)


def tikhonov(w_hat, m, grid, lam_rel=1e-3):
    """Per-frequency Tikhonov solve.

    x_hat(f) = (G(f) + lam I)^-1 W_hat(f)^H m_hat(f),  m_hat = FFT2(pad(m)),
    lam = lam_rel * max over f and j of G_jj(f) (reading: the global maximum
    of the Gram diagonal).  Returns (crop(IFFT2(x_hat)), lam, x_hat).
    """
    n = grid.n
    g = gram(w_hat)
    lam = lam_rel * np.max(np.real(np.einsum("yxzz->yxz", g)))
    z = g.shape[-1]
    m_hat = np.fft.fft2(_pad(m, grid), axes=(-2, -1))  # [T][P][P]
    rhs = np.einsum("tzyx,tyx->yxz", np.conj(w_hat), m_hat)
    x_hat = np.linalg.solve(g + lam * np.eye(z), rhs[..., None])[..., 0]  # [P][P][Z]
    x_hat = np.moveaxis(x_hat, -1, 0)
    x = np.fft.ifft2(x_hat, axes=(-2, -1)).real
    return x[:, :n, :n], lam, x_hat


def spectral_norm(w_hat):
    """max over lateral frequencies of sigma_max(W_hat(f)) (exact, per frequency)."""
    ev = np.linalg.eigvalsh(gram(w_hat))
    return float(np.sqrt(np.max(ev)))


def _dz_t_dz(z):
    """D_z^T D_z for the axial forward difference with Neumann boundary ((Z-1) x Z)."""
    d = np.zeros((z - 1, z))
    for j in range(z - 1):
        d[j, j] = -1.0
        d[j, j + 1] = 1.0
    return d.T @ d


def diff_op(x):
    """D x: forward differences (x: lateral periodic on P grid, y: same, z: Neumann).

    Returns [3][Z][P][P]; the last axial plane is identically zero (there are
    Z-1 axial differences).
    """
    dx = np.roll(x, -1, axis=2) - x
    dy = np.roll(x, -1, axis=1) - x
    dz = np.zeros_like(x)
    dz[:-1] = x[1:] - x[:-1]
    return np.stack([dx, dy, dz])


def diff_adj(w):
    """D^T w for the operator of diff_op."""
    ax = np.roll(w[0], 1, axis=2) - w[0]
    ay = np.roll(w[1], 1, axis=1) - w[1]
    wz = w[2].copy()
    wz[-1] = 0.0
    az = np.zeros_like(wz)
    az[1:] += wz[:-1]
    az -= wz
    return ax + ay + az


def soft(v, thr):
    """Soft threshold (proximal map of thr * |.|)."""
    return np.sign(v) * np.maximum(np.abs(v) - thr, 0.0)


def admm(w_hat, m, grid, iters, rho=1.0, beta=None, beta_rel=1e-3, history=False, callback=None):
    """Scaled-form ADMM for nonnegative, TV-regularised reconstruction.

    Splitting: v1 = K x (T planes on the P grid), v2 = D x, v3 = x.
      0. normalise: s = max_f sigma_max(W_hat(f)); W_hat <- W_hat/s, m <- m/s.
         beta (if None) = beta_rel * max |A^T m| over the N x N x Z crop, in
         normalised units (A = C K).
      1. init x = v = u = 0.
      2. repeat `iters` times:
         x  = H^-1 [K^T (v1 - u1) + D^T (v2 - u2) + (v3 - u3)],
              H(f) = W_hat^H W_hat + (|dx(f)|^2 + |dy(f)|^2 + 1) I + D_z^T D_z
         v1 = (C^T m + rho (K x + u1)) / (C^T 1 + rho)     (elementwise)
         v2 = soft(D x + u2, beta / rho)
         v3 = max(x + u3, 0) * 1_S
         u1 += K x - v1;  u2 += D x - v2;  u3 += x - v3
      3. return crop(v3).
    Returns (mu, info) with info = dict(scale, beta, iterates (if history)).
    `callback(i)`, if given, is called after iteration i (a timing hook; it
    sees no data).
    """
    n, p, nt = grid.n, grid.p, w_hat.shape[0]
    nz = w_hat.shape[1]
    s = spectral_norm(w_hat)
    wn = w_hat / s
    mn = m / s
    if beta is None:
        beta = beta_rel * float(np.max(np.abs(adjoint_fft(wn, mn, grid))))
    # H(f)^-1, [P][P][Z][Z]
    k = np.arange(p)
    lap = (np.abs(np.exp(2j * np.pi * k / p) - 1.0) ** 2)
    diag = lap[:, None] + lap[None, :] + 1.0  # [ky][kx]
    h = gram(wn) + diag[..., None, None] * np.eye(nz) + _dz_t_dz(nz)
    h_inv = np.linalg.inv(h)

    cm = _pad(mn, grid)  # C^T m on the P grid
    c1 = _pad(np.ones_like(mn), grid)  # C^T 1
    support = _pad(np.ones((nz, n, n)), grid)

    def K(x):
        xh = np.fft.fft2(x, axes=(-2, -1))
        return np.fft.ifft2(np.einsum("tzyx,zyx->tyx", wn, xh), axes=(-2, -1)).real

    def Kt(r):
        rh = np.fft.fft2(r, axes=(-2, -1))
        return np.fft.ifft2(np.einsum("tzyx,tyx->zyx", np.conj(wn), rh), axes=(-2, -1)).real

    def Hinv(b):
        bh = np.fft.fft2(b, axes=(-2, -1))
        xh = np.einsum("yxzw,wyx->zyx", h_inv, bh)
        return np.fft.ifft2(xh, axes=(-2, -1)).real

    x = np.zeros((nz, p, p))
    v1 = np.zeros((nt, p, p))
    u1 = np.zeros_like(v1)
    v2 = np.zeros((3, nz, p, p))
    u2 = np.zeros_like(v2)
    v3 = np.zeros_like(x)
    u3 = np.zeros_like(x)
    hist = []
    for _ in range(iters):
        x = Hinv(Kt(v1 - u1) + diff_adj(v2 - u2) + (v3 - u3))
        kx = K(x)
        dxx = diff_op(x)
        v1 = (cm + rho * (kx + u1)) / (c1 + rho)
        v2 = soft(dxx + u2, beta / rho)
        v3 = np.maximum(x + u3, 0.0) * support
        u1 = u1 + kx - v1
        u2 = u2 + dxx - v2
        u3 = u3 + x - v3
        if history:
            hist.append(v3[:, :n, :n].copy())
        if callback is not None:
            callback(_)
    info = dict(scale=s, beta=beta, x=x)
    if history:
        info["iterates"] = hist
    return v3[:, :n, :n].copy(), info


def depth_sensitivity(w_hat):
    """sigma(z) = sqrt(G(0)_zz): the norm of depth z's kernel summed over the
    lateral plane (the DC Gram diagonal), which falls with depth."""
    g0 = gram(w_hat[:, :, :1, :1])[0, 0]
    return np.sqrt(np.real(np.diag(g0)))


def fista_l1(w_hat, m, grid, iters, lam=None, lam_rel=1e-2, layerwise=True, history=False, multiplexed=False):
    """FISTA (Beck and Teboulle) for Eq. 10 with the layer-wise weight lam(z).

    Readings: the data term is 1/2 ||A x - m||^2 (the smooth part FISTA needs);
    units are normalised by s = max_f sigma_max(W_hat(f)) (A <- A/s, m <- m/s,
    so the gradient's Lipschitz constant is 1 and the step is 1); the weight
    follows the depth sensitivity, lam(z) = lam0 sigma(z) / max_z sigma(z)
    (layerwise=False: lam(z) = lam0), which lowers the threshold where the
    measurements see less and so counteracts the fading with depth that
    Eq. 10 is introduced for; lam0 (if lam is None) = lam_rel max |A^T m|.
      1. x_0 = y_1 = 0, t_1 = 1.
      2. for k = 1 .. iters:
           x_k     = soft(y_k - A^T (A y_k - m), lam(z))
           t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2
           y_{k+1} = x_k + ((t_k - 1) / t_{k+1}) (x_k - x_{k-1})
      3. return x_iters.
    multiplexed=True solves the composite problem of Eq. 12 with the same
    scheme: A is replaced by S A (``multiplex.composite_forward``), `m` is the
    multiplexed measurement y, and s by the composite norm 8 s (||S|| = 8).
    Returns (mu, info) with info = dict(scale, lam (per depth), iterates).
    """
    from . import multiplex as mx
    s = spectral_norm(w_hat) * (8.0 if multiplexed else 1.0)
    wn = w_hat / s
    mn = m / s
    nz = w_hat.shape[1]
    fwd = (lambda v: mx.composite_forward(wn, v, grid)) if multiplexed else (lambda v: forward_fft(wn, v, grid))
    adj = (lambda r: mx.composite_adjoint(wn, r, grid)) if multiplexed else (lambda r: adjoint_fft(wn, r, grid))
    if lam is None:
        lam = lam_rel * float(np.max(np.abs(adj(mn))))
    sig = depth_sensitivity(wn)
    lam_z = lam * (sig / sig.max() if layerwise else np.ones(nz))
    thr = lam_z[:, None, None]
    x_prev = np.zeros((nz, grid.n, grid.n))
    y = x_prev.copy()
    t = 1.0
    its = []
    for _ in range(iters):
        g = adj(fwd(y) - mn)
        x = soft(y - g, thr)
        t_next = (1.0 + np.sqrt(1.0 + 4.0 * t * t)) / 2.0
        y = x + ((t - 1.0) / t_next) * (x - x_prev)
        x_prev, t = x, t_next
        if history:
            its.append(x.copy())
    return x_prev, dict(scale=s, lam=lam_z, iterates=its)
