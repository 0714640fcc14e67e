"""Shared set-up of the GPU parity tests: build the library, make matching
oracle / device grids, and build (and cache) device kernels."""

import functools

import numpy as np

from oracle import operators as op
from oracle import physics as ph

CFG1_OPTICS = dict(mua=0.01, musp=1.0, n=1.4)

# name -> grid keywords (lateral n, depths, bins, pitches, first depth, bin width)
CASES = {
    # the 8 x 8 x 4 x 16 sub-grid of config 1 (1 mm voxels, depths 1-4 mm, 16 bins of 50 ps)
    "sub": dict(n=8, nz=4, nt=16, dx=1.0, dz=1.0, z_first=1.0, dt=50.0),
    # config 1: 32 x 32 scan at 1 mm, 16 depths 1-16 mm, 64 bins of 50 ps
    "cfg1": dict(n=32, nz=16, nt=64, dx=1.0, dz=1.0, z_first=1.0, dt=50.0),
    # ragged: n not a power of two, Z and T not multiples of the 8-plane tiles
    "ragged": dict(n=20, nz=5, nt=19, dx=0.7, dz=0.9, z_first=0.9, dt=33.0),
    # anisotropic lateral pitch: only the 4-fold symmetry holds
    "aniso": dict(n=12, nz=3, nt=10, dx=0.8, dy=1.1, dz=1.0, z_first=1.0, dt=40.0),
    # circular (periodic) lateral boundary
    "circ": dict(n=32, nz=4, nt=12, dx=1.0, dz=1.0, z_first=1.0, dt=50.0, mode="circular"),
    # small ADMM case (P = 32)
    "admm16": dict(n=16, nz=6, nt=32, dx=1.0, dz=1.0, z_first=1.0, dt=50.0),
    # full 128-voxel rows (the learned CNN's M tile), four 32-row bands, few depths and bins
    "wide128": dict(n=128, nz=4, nt=32, dx=1.0, dz=1.0, z_first=1.0, dt=50.0),
}


def medium(optics=CFG1_OPTICS, grid_kw=None):
    g = grid_kw or {}
    dy = g.get("dy", g.get("dx", 1.0))
    rmin = 0.5 * min(g.get("dx", 1.0), dy, g.get("dz", 1.0))
    return ph.Medium(optics["mua"], optics["musp"], optics["n"], r_min=rmin)


def oracle_grid(kw):
    return op.Grid(kw["n"], kw["nz"], kw["nt"], kw["dx"], kw["dz"], kw["z_first"], kw["dt"], dy=kw.get("dy"),
                   mode=kw.get("mode", "linear"))


@functools.lru_cache(maxsize=None)
def oracle_kernel(name):
    kw = CASES[name]
    g = oracle_grid(kw)
    w = op.kernel_offsets(g, medium(grid_kw=kw))
    return g, w, op.kernel_spectrum(w, g)


_dev_cache = {}


def device_kernel(name, keep_w=True):
    from paper_2101_11680_gb300 import build as B
    from paper_2101_11680_gb300 import ctof
    key = (name, keep_w)
    if key not in _dev_cache:
        B.build()
        kw = CASES[name]
        grid = ctof.make_grid(kw["n"], kw["nz"], kw["nt"], kw["dx"], kw["dz"], kw["z_first"], kw["dt"],
                              dy=kw.get("dy"), mode=kw.get("mode", "linear"))
        _dev_cache[key] = ctof.Kernel(ctof.make_optics(**CFG1_OPTICS), grid, keep_w=keep_w)
    return _dev_cache[key]


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
