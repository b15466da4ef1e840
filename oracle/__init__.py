"""FP64 CPU oracle for plane-wise multi-view Richardson-Lucy deconvolution.

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously-correct
definition that the CUDA path is checked against.  Only the test suite,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it; the library under ``paper_1503_07998_gb300`` never does, and it
shares no code with it.

Modules
-------
rl       the forward method (Supp. Note 1, update equation; Fig. 1a reslicing),
         with optional per-pixel view weights and the padded-domain estimate
adjoint  reverse-mode gradient of a Poisson data fit through unrolled
         iterations with respect to the PSFs (PSF calibration)
variants correlation kernels X_v of the MV-RL variants (Supp. Note 2 sec. 1)
volume3d 3D MV-RL with PSFs a_v(y) P_v(z, x) (views turned about the axis),
         against which the plane-wise approximation is measured

Every function is pinned by ``tests/test_oracle.py`` against brute force,
library routines, closed forms and invariants; none is "parity unpinned".
"""

from .rl import (  # noqa: F401
    flip_psf,
    convolve,
    correlate,
    convolve_fft,
    correlate_fft,
    init_mean,
    rl_step,
    rl_planes,
    reslice,
    embed_padded,
    crop_padded,
    NORM_FLOOR,
)
from .adjoint import poisson_nll, rl_loss, rl_loss_and_psf_grad  # noqa: F401
from .variants import VARIANTS, correlation_kernels  # noqa: F401
from .volume3d import convolve3d, correlate3d, rl3d  # noqa: F401
