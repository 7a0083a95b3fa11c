"""GB300 library for mixed-variational plane-wave band structures of 3-D phononic crystals
and their adjoint design sensitivities (batched over k, FP64 and split-BF16 forms)."""
from . import binding  # noqa: F401
from .binding import (PC_BCC, PC_FCC, PC_FP64, PC_GAP_LAMBDA, PC_GAP_OMEGA, PC_GRAD_ALLBANDS,  # noqa: F401
                      PC_MIXED, PC_SC, PhononicError)


def __getattr__(name):
    if name in ("BandSolver", "GapFn", "gap"):
        from . import solver
        return getattr(solver, name)
    raise AttributeError(name)
