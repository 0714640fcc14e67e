"""Writes the stored oracle results that the GPU parity tests compare with.

Each fixture is an FP64 oracle run (``oracle/`` only) on seeded synthetic
input (``paper_2101_11680_gb300.synth``) at a size whose oracle run takes
minutes, too long to repeat inside the GPU test session.  The noisy
measurement is stored exactly (integer counts and the count unit), so the
test feeds the device the very input the oracle saw.

    python tests/golden/make_oracle_fixtures.py [name ...]

Fixtures:

* ``admm_n32_z48_t256.npz``: ADMM (nonnegativity + anisotropic TV, rho = 1,
  beta = 1e-3 max|A^T m|) for 100 iterations on a 32 x 32 scan at 0.5 mm
  with 48 depths of 0.5 mm and 256 bins of 25 ps (lateral FFT grid P = 64):
  the frequency-class block of the 128 x 128 x 48 x 256 workload (48
  depths x 256 bins per class) on a smaller lateral field.  Phantom: 1-8
  ellipsoids/tubes (seed 3), Poisson noise at peak 1e5 (seed 103).
* ``tikhonov_n32_z64_t512.npz``: per-frequency Tikhonov (lambda 1e-3 max Gram
  diagonal) at 64 depths x 512 bins on a 32 x 32 scan (P = 64, all 2112
  frequencies), the class block of the 256 x 256 x 64 x 512 precision-form
  workload; two sphere phantoms, Poisson peak 1e4.
"""

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import operators as op  # noqa: E402
from oracle import physics as ph  # noqa: E402
from oracle import solvers as so  # noqa: E402
from paper_2101_11680_gb300 import synth  # noqa: E402

OPTICS = dict(mua=0.01, musp=1.0, n=1.4)


def _medium(kw):
    return ph.Medium(OPTICS["mua"], OPTICS["musp"], OPTICS["n"], r_min=0.5 * min(kw["dx"], kw["dz"]))


def _grid(kw):
    return op.Grid(kw["n"], kw["nz"], kw["nt"], kw["dx"], kw["dz"], kw["z_first"], kw["dt"])


def _noisy_counts(wh, g, mu, peak, seed):
    """Poisson counts and the count unit of synth.poisson_noise (same draws)."""
    clean = np.clip(op.forward_fft(wh, mu, g), 0.0, None)
    noisy = synth.poisson_noise(clean, peak, seed)
    unit = float(clean.max()) / peak
    counts = np.rint(noisy / unit).astype(np.int32)
    assert np.array_equal(counts.astype(np.float64) * unit, noisy)
    return counts, unit


def admm_n32_z48_t256():
    kw = dict(n=32, nz=48, nt=256, dx=0.5, dz=0.5, z_first=0.5, dt=25.0)
    g = _grid(kw)
    wh = op.kernel_spectrum(op.kernel_offsets(g, _medium(kw)), g)
    mu = synth.phantom_shapes(g.n, g.nz, g.dx, g.dz, g.z_first, seed=3)
    counts, unit = _noisy_counts(wh, g, mu, 1e5, 103)
    iters = 100
    want, info = so.admm(wh, counts.astype(np.float64) * unit, g, iters)
    np.savez_compressed(os.path.join(HERE, "admm_n32_z48_t256.npz"), counts=counts, unit=unit,
                        grid=np.array([kw["n"], kw["nz"], kw["nt"]]),
                        pitch=np.array([kw["dx"], kw["dz"], kw["z_first"], kw["dt"]]), iters=iters,
                        want=want, beta=info["beta"], scale=info["scale"])


def tikhonov_n32_z64_t512():
    """Precision-form class shape: 64 depths x 512 bins (the 256 x 256 x 64 x 512
    workload's frequency-class block) on a 32 x 32 scan at 0.5 mm (P = 64: all
    2112 half-plane frequencies solved exactly by the FP64 oracle).  Two
    measurement volumes (2 spheres each, seeds 0 and 1; Poisson peak 1e4, seeds
    100 and 101); lambda = 1e-3 max Gram diagonal.  Counts stored as int16."""
    kw = dict(n=32, nz=64, nt=512, dx=0.5, dz=0.5, z_first=0.5, dt=25.0)
    g = _grid(kw)
    wh = op.kernel_spectrum(op.kernel_offsets(g, _medium(kw)), g)
    counts, units, wants = [], [], []
    lam = None
    for i in range(2):
        mu = synth.phantom_spheres(g.n, g.nz, g.dx, g.dz, g.z_first, seed=i)
        c, unit = _noisy_counts(wh, g, mu, 1e4, 100 + i)
        assert c.max() < 32767
        want, lam, _ = so.tikhonov(wh, c.astype(np.float64) * unit, g)
        counts.append(c.astype(np.int16))
        units.append(unit)
        wants.append(want.astype(np.float32))
    np.savez_compressed(os.path.join(HERE, "tikhonov_n32_z64_t512.npz"), counts=np.stack(counts),
                        unit=np.array(units), grid=np.array([kw["n"], kw["nz"], kw["nt"]]),
                        pitch=np.array([kw["dx"], kw["dz"], kw["z_first"], kw["dt"]]), lam=lam,
                        want=np.stack(wants))


FIXTURES = {"admm_n32_z48_t256": admm_n32_z48_t256, "tikhonov_n32_z64_t512": tikhonov_n32_z64_t512}

if __name__ == "__main__":
    for name in sys.argv[1:] or list(FIXTURES):
        FIXTURES[name]()
        print("wrote", name)
