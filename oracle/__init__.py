"""FP64 CPU oracle for confocal time-of-flight DOT (arXiv 2101.11680).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It
shares no code, tables or constants with the CUDA library; the only module
both sides use is the seeded input generator ``paper_2101_11680_gb300.synth``,
which holds none of the method's arithmetic.

Layout
------
physics    diffusion Green's functions (Eq. 4, Eq. 5), the source->voxel->
           detector time convolution in closed form and numerically, and the
           time-bin quadrature; the fluorescence-mode response (excitation
           and emission optics, lifetime convolution) by the convolution
           theorem and a fixed-Talbot Laplace inversion.
operators  the sensitivity kernel W on the lateral offset grid, the dense
           confocal Jacobian (Eq. 2, Eq. 6), and the convolutional forward /
           adjoint operators of the 3D convolutional approximation
           (Eq. 11) both by direct summation and by FFT.
solvers    per-frequency Tikhonov (the regularised inverse of Eq. 7) and the
           ADMM (nonnegativity + anisotropic 3D TV) iteration.

Every function is plain NumPy/SciPy in float64 and follows the definition it
cites; none is blocked, fused or reordered for speed.
"""

from . import physics, operators, solvers  # noqa: F401
