"""GB300 (sm_103a) implementation of the hybrid exponential / semi-implicit
spectral deferred correction (HSDC, "ES-SDC") step for the monodomain equation
of arXiv 2405.19994, behind the C ABI of include/esdc.h."""
from . import inputs  # noqa: F401
from .esdc import Batch, Solver, EsdcError, lib  # noqa: F401
