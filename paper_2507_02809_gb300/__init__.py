"""GB300-native solver for the block-triangular-preconditioned all-at-once system of the
time-space fractional inverse source problem (arXiv 2507.02809).

The compute path is the CUDA library ``lib/libtsfde.so`` (sources in ``csrc/``,
C ABI in ``include/tsfde.h``); ``tsfde`` is its ctypes binding and ``autograd`` wraps the
solve and its adjoint as a ``torch.autograd.Function``.  Importing this
package does not load the library; the first call does, and raises if it is
missing.
"""
from .tsfde import (  # noqa: F401
    BLOCK_SOLVE,
    BLOCK_STRANG,
    BLOCK_TAU,
    EXPORTS,
    PREC_FP64,
    PREC_MIXED,
    SIDE_FLEXIBLE,
    SIDE_LEFT,
    SIDE_RIGHT,
    TSFDE_EBREAKDOWN,
    TSFDE_ECUDA,
    TSFDE_EINVAL,
    TSFDE_ENOMEM,
    TSFDE_ETIMEOUT,
    TSFDE_EUNSUPPORTED,
    TSFDE_NOT_CONVERGED,
    TSFDE_OK,
    Solver,
    TsfdeError,
    TsfdeOpts,
    library_path,
    load,
    tsfde_adjoint,
    tsfde_default_opts,
    tsfde_destroy,
    tsfde_device_bytes,
    tsfde_direct_solve,
    tsfde_gmres_solve,
    tsfde_gmres_solve_batch,
    tsfde_matvec,
    tsfde_matvec_1d_noalloc,
    tsfde_matvec_transpose,
    tsfde_precond_apply,
    tsfde_precond_apply_batch,
    tsfde_precond_apply_transpose,
    tsfde_profile,
    tsfde_profile_read,
    tsfde_rhs,
    tsfde_set_opts,
    tsfde_solve,
    tsfde_setup,
)
