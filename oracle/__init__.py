"""CPU FP64 oracle of the LBM / Maxwell-Stefan ternary diffusion method.

TEST INFRASTRUCTURE.  This package exists to check the CUDA solver: only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg and the
``--impl reference`` arm of ``bench.py`` may import it.  It shares no code
with the solver (constants, tables and arithmetic are all its own); both
sides take their inputs from ``workloads``.

Every function cites the paper passage it follows (Eqs. 2, 9, 19-43).
Pins (tests/test_oracle_pins.py) tie it to closed forms: the 1-D ternary
Maxwell-Stefan profile with Stefan flux, the exact binary linear profile, the
exact lattice variance law of a diffusing pulse, I = 0 invariance, closed-box
conservation, steady flux balance, D2Q9/D3Q19 agreement on 1-D states and
mirror symmetry; with the literal readings of Eq. 35 (forward gradient) and
Eq. 37 (extrapolated outlet) the 1-D profile is reached at first order.
Porous 2-D/3-D fields have no closed form: beyond those invariants their
parity is unpinned.
"""
from .gas import Scaling, fuller_binary, knudsen, effective_binary, total_concentration
from .lattice import d2q9, d3q19
from .lbm import Oracle

__all__ = ["Oracle", "Scaling", "fuller_binary", "knudsen", "effective_binary",
           "total_concentration", "d2q9", "d3q19"]
