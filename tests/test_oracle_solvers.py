"""Pins of the oracle's solvers against independent dense linear algebra and optimisers.

* Tikhonov (circular mode) == a dense solve of (J^T J + lam I) x = J^T m with
  the entry-by-entry Jacobian; and (linear mode) its spatial normal equations
  with the periodic operator applied by direct summation.
* The ADMM normalisation s = max_f sigma_max(W_hat(f)) == ||J||_2 (circular).
* ADMM with beta = 0 converges to the non-negative least-squares solution
  (scipy.optimize.nnls on the dense Jacobian); with beta > 0 to the minimiser
  found by SLSQP on the dense TV problem assembled from its definition.
"""

import numpy as np
import pytest
from scipy import optimize

from oracle import operators as op
from oracle import physics as ph
from oracle import solvers as so
from paper_2101_11680_gb300 import synth


def medium():
    return ph.Medium(0.01, 1.0, 1.4, r_min=0.5)


def test_tikhonov_equals_dense_solve_circular():
    g = op.Grid(8, 4, 16, 1.0, 1.0, 1.0, 50.0, mode="circular")
    m_ = medium()
    w = op.kernel_offsets(g, m_)
    wh = op.kernel_spectrum(w, g)
    J = op.dense_jacobian(g, m_)
    rng = np.random.default_rng(11)
    meas = rng.uniform(0, 1, (g.nt, g.n, g.n)) * np.abs(J).max()
    x, lam, _ = so.tikhonov(wh, meas, g)
    want = np.linalg.solve(J.T @ J + lam * np.eye(J.shape[1]), J.T @ meas.ravel())
    assert np.abs(x.ravel() - want).max() <= 1e-9 * np.abs(want).max()
    # lam is 1e-3 x the largest Gram diagonal = 1e-3 x the largest column norm^2 of the
    # circulant J times P^0 (Parseval: diag G(f) summed over f / P^2 = ||column||^2)
    assert lam > 0


def _periodic_apply(wp, x):
    """K x on the P grid by direct periodic summation (no FFT): wp [T][Z][P][P], x [Z][P][P]."""
    t, z, p, _ = wp.shape
    out = np.zeros((t, p, p))
    for j in range(z):
        for yp in range(p):
            for xp in range(p):
                if x[j, yp, xp] != 0.0:
                    out += x[j, yp, xp] * np.roll(wp[:, j], (yp, xp), axis=(1, 2))
    return out


def _periodic_adjoint(wp, r):
    t, z, p, _ = wp.shape
    out = np.zeros((z, p, p))
    for yp in range(p):
        for xp in range(p):
            sh = np.roll(wp, (yp, xp), axis=(2, 3))
            out[:, yp, xp] = np.einsum("tzyx,tyx->z", sh, r)
    return out


def test_tikhonov_normal_equations_linear():
    """(K^T K + lam) x = K^T pad(m) on the P grid, K applied by direct periodic sums."""
    g = op.Grid(6, 3, 8, 1.0, 1.0, 1.0, 50.0)
    w = op.kernel_offsets(g, medium())
    wh = op.kernel_spectrum(w, g)
    wp = op.periodic_kernel(w, g)
    rng = np.random.default_rng(12)
    meas = rng.uniform(0, 1, (g.nt, g.n, g.n)) * np.abs(w).max()
    _, lam, xh = so.tikhonov(wh, meas, g)
    x = np.fft.ifft2(xh, axes=(-2, -1)).real
    padm = np.zeros((g.nt, g.p, g.p))
    padm[:, :g.n, :g.n] = meas
    lhs = _periodic_adjoint(wp, _periodic_apply(wp, x)) + lam * x
    rhs = _periodic_adjoint(wp, padm)
    assert np.abs(lhs - rhs).max() <= 1e-10 * np.abs(rhs).max()


def test_normalisation_is_operator_norm():
    g = op.Grid(8, 4, 16, 1.0, 1.0, 1.0, 50.0, mode="circular")
    m_ = medium()
    wh = op.kernel_spectrum(op.kernel_offsets(g, m_), g)
    J = op.dense_jacobian(g, m_)
    assert so.spectral_norm(wh) == pytest.approx(np.linalg.norm(J, 2), rel=1e-10)


def test_normalisation_attained_at_dc():
    """W >= 0 elementwise, so |W_hat(f)| <= W_hat(0) entrywise and the max is at f = 0."""
    g = op.Grid(8, 4, 16, 1.0, 1.0, 1.0, 50.0)
    wh = op.kernel_spectrum(op.kernel_offsets(g, medium()), g)
    s0 = np.linalg.norm(wh[:, :, 0, 0].real, 2)
    assert so.spectral_norm(wh) == pytest.approx(s0, rel=1e-12)


def _tiny(n=4, nz=1, nt=12, dx=1.0, dz=1.0, z_first=2.0, dt=50.0, seed=5):
    """A small, well-conditioned linear-mode problem with 2 % Gaussian noise."""
    g = op.Grid(n, nz, nt, dx, dz, z_first, dt, mode="linear")
    m_ = medium()
    w = op.kernel_offsets(g, m_)
    wh = op.kernel_spectrum(w, g)
    J = op.dense_jacobian(g, m_)
    rng = np.random.default_rng(seed)
    mu = rng.uniform(0, 0.02, (nz, n, n)) * (rng.uniform(size=(nz, n, n)) < 0.5)
    meas = op.forward_fft(wh, mu, g)
    meas = meas + 0.02 * np.abs(meas).max() * rng.standard_normal(meas.shape)
    return g, wh, J, meas


def test_admm_beta0_converges_to_nnls():
    """beta = 0: ADMM's limit is the non-negative least-squares solution on S.

    (The fixed point does not depend on rho; rho = 0.03 converges fast here.)
    """
    g, wh, J, meas = _tiny()
    x, info = so.admm(wh, meas, g, 3000, beta=0.0, rho=0.03)
    s = info["scale"]
    want, _ = optimize.nnls(J / s, meas.ravel() / s, maxiter=10000)
    assert np.abs(x.ravel() - want).max() <= 1e-9 * np.abs(want).max()


def _tv_matrix(g):
    """Rows of D restricted to the support S for the zero-extended P-grid volume.

    Lateral: periodic forward differences on the P grid; since x = 0 off S each
    lateral line contributes the N-1 interior differences plus |x_first| and
    |x_last| (the two neighbours outside S).  Axial: the Z-1 Neumann differences.
    """
    n, z = g.n, g.nz
    idx = lambda j, y, x: (j * n + y) * n + x
    rows = []
    for j in range(z):
        for y in range(n):
            for x in range(n):
                for (yy, xx) in ((y, x + 1), (y + 1, x)):
                    r = np.zeros(z * n * n)
                    r[idx(j, y, x)] = -1.0
                    if yy < n and xx < n:
                        r[idx(j, yy, xx)] = 1.0
                    rows.append(r)
                # difference entering the support from the zero neighbour at -1
                if x == 0:
                    r = np.zeros(z * n * n)
                    r[idx(j, y, x)] = 1.0
                    rows.append(r)
                if y == 0:
                    r = np.zeros(z * n * n)
                    r[idx(j, y, x)] = 1.0
                    rows.append(r)
                if j + 1 < z:
                    r = np.zeros(z * n * n)
                    r[idx(j, y, x)] = -1.0
                    r[idx(j + 1, y, x)] = 1.0
                    rows.append(r)
    return np.array(rows)


def test_admm_tv_matches_slsqp():
    """beta > 0: ADMM's limit is the minimiser of the dense TV problem (SLSQP from zero)."""
    g, wh, J, meas = _tiny(n=2, nz=3, nt=48, dx=1.5, dz=1.5, z_first=1.5, dt=20.0, seed=5)
    x, info = so.admm(wh, meas, g, 2000, beta_rel=2e-2, rho=0.1)
    s, beta = info["scale"], info["beta"]
    A = J / s
    b = meas.ravel() / s
    E = _tv_matrix(g)
    nv, ne = A.shape[1], E.shape[0]

    def f(v):
        xx, tt = v[:nv], v[nv:]
        r = A @ xx - b
        return 0.5 * r @ r + beta * tt.sum()

    def grad(v):
        xx = v[:nv]
        return np.concatenate([A.T @ (A @ xx - b), beta * np.ones(ne)])

    cons = [{"type": "ineq", "fun": lambda v: v[nv:] - E @ v[:nv], "jac": lambda v: np.hstack([-E, np.eye(ne)])},
            {"type": "ineq", "fun": lambda v: v[nv:] + E @ v[:nv], "jac": lambda v: np.hstack([E, np.eye(ne)])}]
    res = optimize.minimize(f, np.zeros(nv + ne), jac=grad, constraints=cons, method="SLSQP",
                            bounds=[(0, None)] * (nv + ne), options=dict(ftol=1e-16, maxiter=2000))
    assert res.success
    fx = f(np.concatenate([x.ravel(), np.abs(E @ x.ravel())]))
    assert fx <= res.fun * (1 + 1e-10)
    assert np.abs(res.x[:nv] - x.ravel()).max() <= 1e-5 * np.abs(x).max()


def test_admm_fixed_point_residuals_vanish():
    g, wh, _, meas = _tiny(n=2, nz=3, nt=48, dx=1.5, dz=1.5, z_first=1.5, dt=20.0)
    x, info = so.admm(wh, meas, g, 2000, beta_rel=2e-2, rho=0.1)
    xf = info["x"]
    # the x iterate agrees with the feasible output on S and is ~0 off S
    assert np.abs(xf[:, :g.n, :g.n] - x).max() <= 1e-6 * np.abs(x).max()
    off = xf.copy()
    off[:, :g.n, :g.n] = 0.0
    assert np.abs(off).max() <= 1e-6 * np.abs(x).max()


def test_admm_first_iterate_is_zero():
    """From x = v = u = 0 the first x-update sees a zero right-hand side, so v3 = 0."""
    g, wh, J, meas = _tiny()
    v1, _ = so.admm(wh, meas, g, 1)
    assert np.all(v1 == 0.0)


def test_phantom_generators():
    vol = synth.phantom_spheres(32, 16, 1.0, 1.0, 1.0, seed=0)
    assert set(np.unique(vol)) <= {0.0, 0.01}
    # two spheres of radius 1.5 mm centred at depths 5 and 9 mm (voxel depths 1..16 mm):
    # every marked voxel lies within 1.5 mm of one of those depths; volume ~ 2 x 14 voxels
    zs = 1.0 + np.nonzero(vol)[0]
    assert np.all((np.abs(zs - 5.0) <= 1.5) | (np.abs(zs - 9.0) <= 1.5))
    assert 2 * 7 <= np.count_nonzero(vol) <= 2 * 27
    v2 = synth.phantom_shapes(32, 16, 0.5, 0.5, 0.5, seed=3)
    assert v2.max() <= 0.02 and v2.min() >= 0.0 and np.count_nonzero(v2) > 0
    a = synth.phantom_shapes(16, 8, 0.5, 0.5, 0.5, seed=4)
    b = synth.phantom_shapes(16, 8, 0.5, 0.5, 0.5, seed=4)
    assert np.array_equal(a, b)


def test_poisson_noise_statistics():
    m = np.full(200000, 0.25)
    m[0] = 1.0
    y = synth.poisson_noise(m, 1e4, seed=1)
    # counts at 2500 expected: mean 0.25, variance 0.25 * (max/peak)
    assert y[1:].mean() == pytest.approx(0.25, rel=2e-3)
    assert y[1:].var() == pytest.approx(0.25 * 1e-4, rel=2e-2)


def test_dark_count_noise_statistics():
    """Dark-count noise of the multiplexing simulations (Section 5: 200 counts/s dark rate).

    With no light every measurement holds only dark counts: dark_cps x
    integration time per measurement, spread over its bins, Poisson (mean =
    variance).  With light, the brightest measurement collects rate x time
    photons, and the dark-subtracted counts are an unbiased estimate of m.
    """
    nt, n = 64, 24
    dark = synth.dark_count_noise(np.zeros((nt, n, n)), 5e6, 0.5, 200.0, seed=1)
    counts, unit, per_bin = dark
    assert per_bin == pytest.approx(200.0 * 0.5 / nt)
    tot = counts.reshape(nt, -1).sum(axis=0)  # dark counts per measurement: Poisson(100)
    assert tot.mean() == pytest.approx(100.0, rel=0.02)
    assert tot.var() == pytest.approx(100.0, rel=0.1)
    t = np.arange(nt)[:, None, None]
    m = np.exp(-((t - 20.0) / 6.0) ** 2) * np.ones((1, n, n)) * np.linspace(0.2, 1.0, n)[None, None, :]
    est = []
    for seed in range(40):
        c, unit, per_bin = synth.dark_count_noise(m, 5e6, 1e-3, 200.0, seed=100 + seed)
        assert c.dtype.kind == "i"
        assert unit * 5e6 * 1e-3 == pytest.approx(m.sum(axis=0).max())
        est.append((c - per_bin) * unit)
    est = np.array(est)
    assert np.abs(est.mean(axis=0) - m).max() <= 6 * np.sqrt(m.max() * unit / 40 + 1e-30)
    # Poisson: the variance of the counts equals their mean
    lam = m / unit + per_bin
    var = (est / unit).var(axis=0)
    assert float(np.mean(var[lam > 50] / lam[lam > 50])) == pytest.approx(1.0, rel=0.05)


def test_depth_sensitivity_is_response_to_a_constant_plane():
    """Periodic grid: K applied to a constant plane of ones at depth z is the DC
    term alone, so ||K 1_z|| = P sigma(z); sigma falls with depth (Eq. 10's
    motive)."""
    g = op.Grid(8, 4, 16, 1.0, 1.0, 1.0, 50.0, mode="circular")
    wh = op.kernel_spectrum(op.kernel_offsets(g, medium()), g)
    sig = so.depth_sensitivity(wh)
    for z in range(g.nz):
        plane = np.zeros((g.nz, g.n, g.n))
        plane[z] = 1.0
        resp = op.forward_fft(wh, plane, g)
        assert np.linalg.norm(resp) == pytest.approx(g.p * sig[z], rel=1e-12)
    assert np.all(np.diff(sig) < 0)


def test_fista_lam0_converges_to_least_squares():
    """lam = 0: FISTA minimises 1/2 ||A x - m||^2; its limit is the least-squares
    solution (one depth: condition number 13, so it gets there quickly)."""
    g, wh, J, meas = _tiny(nz=1, nt=16)
    x, info = so.fista_l1(wh, meas, g, 6000, lam=0.0)
    s = info["scale"]
    want, *_ = np.linalg.lstsq(J / s, meas.ravel() / s, rcond=None)
    assert np.abs(x.ravel() - want).max() <= 1e-8 * np.abs(want).max()


def test_fista_matches_weighted_lasso_of_sklearn():
    """lam > 0, layer-wise: the FISTA limit equals scikit-learn's coordinate-descent
    Lasso on the dense Jacobian with columns scaled by 1/lam(z)."""
    linear_model = pytest.importorskip("sklearn.linear_model")
    g, wh, J, meas = _tiny(nz=2, nt=16, seed=7)
    x, info = so.fista_l1(wh, meas, g, 6000, lam_rel=0.2)
    s, lam_z = info["scale"], info["lam"]
    assert lam_z[1] < lam_z[0]  # deeper layer, smaller weight
    a = J / s
    y = meas.ravel() / s
    w = np.repeat(lam_z, g.n * g.n)
    model = linear_model.Lasso(alpha=1.0 / len(y), fit_intercept=False, tol=1e-14, max_iter=200000)
    model.fit(a / w[None, :], y)
    want = model.coef_ / w
    assert np.abs(x.ravel() - want).max() <= 1e-9 * np.abs(want).max()
    # optimality (KKT) of the weighted L1 problem
    r = a.T @ (y - a @ x.ravel())
    nzr = np.abs(x.ravel()) > 0
    assert np.all(np.abs(r[~nzr]) <= w[~nzr] * (1 + 1e-6))
    assert np.allclose(r[nzr], w[nzr] * np.sign(x.ravel()[nzr]), rtol=1e-5, atol=1e-9 * w.max())


def test_fista_first_iterate_is_a_thresholded_gradient_step():
    g, wh, J, meas = _tiny(nz=2, nt=16)
    x, info = so.fista_l1(wh, meas, g, 1, lam_rel=0.1)
    s, lam_z = info["scale"], info["lam"]
    step = (J / s).T @ (meas.ravel() / s)  # y_1 = 0: y - grad = A^T m
    thr = np.repeat(lam_z, g.n * g.n)
    want = np.sign(step) * np.maximum(np.abs(step) - thr, 0.0)
    assert np.allclose(x.ravel(), want, rtol=1e-12, atol=1e-15)
