"""GB300 (sm_103a) implementation of the HyperSARA primal-dual hot path.

The compute lives in libhypersara.so (CUDA kernels behind the C ABI declared
in include/hypersara.h); `hypersara` is its ctypes binding, `autograd` exposes
Phi and Psi as torch.autograd Functions (backward = the adjoint kernels) and a
checkpointed unrolled PD solve, and `problem` prepares a synthetic problem on
the device with the library's own operators.
Importing this package does not load the library; the first call does, and
raises if it has not been built.
"""

from . import hypersara  # noqa: F401
from .hypersara import (  # noqa: F401
    Plan,
    PDState,
    HSError,
    phi_fwd,
    phi_adj,
    psi_fwd,
    psi_adj,
    prox_l21,
    prox_nuclear,
    proj_l2ball,
    pd_step,
    pd_solve,
    load,
)
