"""Source multiplexing and the composite operator y = S A mu (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 5 ("Composite reconstruction algorithm", Eq. 12) measures y = S m =
S J mu, with S the multiplexing matrix, and solves the L1 problem for the
composite operator with FISTA; the multiplexing study uses an 8 x 8 source
array, hence a 64 x 64 Hadamard matrix.  Readings:
  * the scan grid is tiled into 8 x 8 blocks of scan points; S acts on the
    64 points of each block (row-major inside the block) for every time bin:
    y[t, block] = H_64 m[t, block];
  * S is the Sylvester Hadamard matrix with entries +-1 (H_1 = [1],
    H_2n = [[H_n, H_n], [H_n, -H_n]]); H H^T = 64 I, H = H^T, so the composite
    operator's norm is 8 times that of A.
"""

import numpy as np

from .operators import adjoint_fft, forward_fft

BLOCK = 8


def hadamard(n):
    """Sylvester Hadamard matrix of order n (a power of two)."""
    h = np.ones((1, 1))
    while h.shape[0] < n:
        h = np.block([[h, h], [h, -h]])
    return h


def block_multiplex(m, h=None):
    """y[t] = S m[t]: H applied to the 64 scan points of every 8 x 8 block (row-major)."""
    h = hadamard(BLOCK * BLOCK) if h is None else h
    t, n, _ = m.shape
    nb = n // BLOCK
    blocks = m.reshape(t, nb, BLOCK, nb, BLOCK).transpose(0, 1, 3, 2, 4).reshape(t, nb, nb, BLOCK * BLOCK)
    out = np.einsum("ij,tabj->tabi", h, blocks)
    return out.reshape(t, nb, nb, BLOCK, BLOCK).transpose(0, 1, 3, 2, 4).reshape(t, n, n)


def block_multiplex_adj(y, h=None):
    """S^T y (H is symmetric, so the same map)."""
    h = hadamard(BLOCK * BLOCK) if h is None else h
    return block_multiplex(y, h.T)


def composite_forward(w_hat, mu, grid):
    """y = S A mu (Eq. 12)."""
    return block_multiplex(forward_fft(w_hat, mu, grid))


def composite_adjoint(w_hat, y, grid):
    """A^T S^T y."""
    return adjoint_fft(w_hat, block_multiplex_adj(y), grid)
