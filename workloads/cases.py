"""Synthetic workload recipes: gas data, operating point, geometry and seeds.

These are inputs handed to both the CPU oracle and the CUDA solver; nothing
here computes any part of the transport model.

Gas data are Table 1 of the paper (molar mass in kg/kmol, Fuller diffusion
volume); the reaction is Eq. 38 (stoichiometry H2 -1, H2O +1, Ar 0, two
electrons per H2).  The operating point of the synthetic anodes is 1073 K,
1 atm, a 1 um pore diameter for the Knudsen term and inlet mole fractions
H2/H2O/Ar = 0.5/0.1/0.4; the paper's own Table 2 point (1023.15 K,
1.013e5 Pa, eps/tau = 0.46/4.5, d_p = 2.6 um) is ``PAPER_TABLE2``.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

from .microstructure import overlapping_balls

SPECIES = ("H2", "H2O", "Ar")
MOLAR_MASS = (2.016, 18.015, 39.948)      # kg/kmol, Table 1
FULLER_VOLUME = (6.12, 13.1, 16.2)        # Table 1
STOICH = (-1, 1, 0)                       # Eq. 38
ELECTRONS = 2


@dataclass
class Gas:
    T: float = 1073.0               # K
    p: float = 101325.0             # Pa
    pore_diameter: float = 1e-6     # m, Knudsen term; <= 0 disables it
    eps_over_tau: float = 1.0       # porosity/tortuosity factor of Eq. 41
    D_binary: np.ndarray | None = None   # 3x3 m^2/s; None -> Fuller
    molar_mass: tuple = MOLAR_MASS
    fuller_volume: tuple = FULLER_VOLUME
    stoich: tuple = STOICH
    electrons: int = ELECTRONS


PAPER_TABLE2 = Gas(T=1023.15, p=1.013e5, pore_diameter=2.6e-6,
                   eps_over_tau=0.46 / 4.5)


@dataclass
class Case:
    name: str
    solid: np.ndarray                 # [z, y, x] bool, True = solid
    dim: int
    x_in: tuple = (0.5, 0.1, 0.4)
    current_A_cm2: float = 0.5
    length_x: float = 2e-3            # m, inlet node to outlet node
    periodic_x: bool = False          # True: closed box, no inlet/outlet
    gas: Gas = field(default_factory=Gas)
    porosity: float = 1.0
    seed: int | None = None

    @property
    def shape(self):
        return self.solid.shape

    @property
    def n_cells(self) -> int:
        return int(self.solid.size)

    @property
    def n_fluid(self) -> int:
        return int((~self.solid).sum())

    def with_(self, **kw) -> "Case":
        return replace(self, **kw)


def open_channel(nx: int, ny: int = 1, nz: int = 1, **kw) -> Case:
    """All-fluid box: with ny = nz = 1 this is the 1-D anode of Section 4.1."""
    dim = 3 if nz > 1 or kw.pop("dim", 2) == 3 else 2
    solid = np.zeros((nz, ny, nx), dtype=bool)
    return Case(name=kw.pop("name", f"open_{nx}x{ny}x{nz}"), solid=solid,
                dim=dim, **kw)


def porous(shape, radius: int, porosity: float, seed: int, **kw) -> Case:
    ms = overlapping_balls(shape, radius, porosity, seed)
    dim = 2 if ms.solid.shape[0] == 1 and len(shape) == 2 else 3
    return Case(name=kw.pop("name", f"porous_{'x'.join(map(str, shape))}_s{seed}"),
                solid=ms.solid, dim=dim, porosity=ms.porosity, seed=ms.seed_used,
                **kw)


def anode_2d_96x48() -> Case:
    """2-D D2Q9 96x48 anode: disks r = 4, porosity 0.45, seed 1, 0.5 A/cm2."""
    return porous((48, 96), radius=4, porosity=0.45, seed=1,
                  name="anode2d_96x48_r4_eps0.45", current_A_cm2=0.5)


def anode_3d_256x128x128() -> Case:
    """3-D D3Q19 256x128x128 anode: spheres r = 3, porosity 0.40, seed 2, 1.0 A/cm2."""
    return porous((128, 128, 256), radius=3, porosity=0.40, seed=2,
                  name="anode3d_256x128x128_r3_eps0.40", current_A_cm2=1.0)


def anode_3d_small(nx=40, ny=24, nz=20, radius=3, porosity=0.40, seed=2,
                   current=1.0) -> Case:
    """Reduced 3-D anode with the same recipe, for oracle-sized parity runs."""
    return porous((nz, ny, nx), radius=radius, porosity=porosity, seed=seed,
                  name=f"anode3d_{nx}x{ny}x{nz}_r{radius}_s{seed}",
                  current_A_cm2=current)


def gaussian_pulse(shape, axis: int, sigma0: float, amplitude: float,
                   background=(0.3, 0.3, 0.4)) -> np.ndarray:
    """Mole-fraction field with a Gaussian H2 pulse (H2O compensating) along
    ``axis`` (0 = x, 1 = y, 2 = z) of a [z, y, x] grid."""
    nz, ny, nx = shape
    n = (nx, ny, nz)[axis]
    c = (n - 1) / 2.0
    s = np.arange(n, dtype=np.float64) - c
    g = amplitude * np.exp(-s * s / (2.0 * sigma0 * sigma0))
    shp = [1, 1, 1]
    shp[2 - axis] = n
    g = g.reshape(shp)
    X = np.empty((3,) + tuple(shape))
    X[0] = background[0] + g
    X[1] = background[1] - g
    X[2] = background[2]
    return X
