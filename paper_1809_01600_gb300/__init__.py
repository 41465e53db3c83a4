"""GB300-native solver for ternary (H2-H2O-Ar) diffusion in a porous SOFC
anode: an advection-diffusion lattice Boltzmann model coupled to the
Maxwell-Stefan equations through a local relaxation time (arXiv:1809.01600).

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/lbms.h``); ``lbms.Solver`` is its Python binding.
"""
from .lbms import Batch, LbmsError, Net, Solver, load  # noqa: F401

__all__ = ["Solver", "Batch", "Net", "LbmsError", "load"]
