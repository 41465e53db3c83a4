"""Seeded synthetic inputs shared by the CPU oracle and the CUDA solver.

Nothing here computes any part of the transport model: it draws masks and
states the operating points (gas data of Table 1, Eq. 38 stoichiometry).
"""
from .microstructure import overlapping_balls, porosity_of, Microstructure
from . import cases

__all__ = ["overlapping_balls", "porosity_of", "Microstructure", "cases"]
