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


def anode_3d_512() -> Case:
    """3-D D3Q19 512^3 anode: spheres r = 4, porosity 0.40, seed 7, 1.0 A/cm2."""
    return porous((512, 512, 512), radius=4, porosity=0.40, seed=7,
                  name="anode3d_512x512x512_r4_eps0.40", current_A_cm2=1.0)


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


def sweep_structures(n2d: int, n3d: int, seed0: int = 100, scale: float = 1.0):
    """Seeded microstructures in the style of the uneven-size sweep: 2-D
    grids from 128x128 to 1024x512, 3-D cubes from 64^3 to 160^3 (sizes
    times ``scale``), radius 2-6 cells, porosity uniform in [0.30, 0.55] in
    3-D and in [0.42, 0.55] in 2-D, where the pore space of overlapping disks
    stops percolating near 0.32 and long strips rarely percolate below 0.4.
    A structure none of whose draws percolates is drawn again with its
    porosity raised by 0.02 until one does (the case records the porosity
    reached).  Returns a list of Cases with default boundary data."""
    rng = np.random.Generator(np.random.PCG64(seed0))
    out = []
    for k in range(n2d + n3d):
        seed = seed0 + k
        por = float(rng.uniform(0.30, 0.55))
        if k < n2d:
            por = 0.42 + (por - 0.30) * (0.55 - 0.42) / 0.25
        rad = int(rng.integers(2, 7))
        if k < n2d:
            nx = int(round(rng.uniform(128, 1024) * scale / 8)) * 8
            ny = int(round(rng.uniform(128, 512) * scale / 8)) * 8
            shape = (max(ny, 16), max(nx, 16))
        else:
            n = int(round(rng.uniform(64, 160) * scale / 8)) * 8
            shape = (max(n, 16),) * 3
        while True:
            try:
                c = porous(shape, radius=rad, porosity=por, seed=seed,
                           name=f"sweep{k}_{'x'.join(map(str, shape[::-1]))}_eps{por:.2f}_r{rad}")
                break
            except RuntimeError:
                if por > 0.7:
                    raise
                por = round(por + 0.02, 4)
        out.append(c)
    return out


def sweep_operating_points(n: int = 8, seed0: int = 7):
    """n (current A/cm2, inlet composition) pairs: currents evenly spread in
    [0, 2], inlet H2 fraction drawn in [0.2, 0.8] at H2:H2O = 4:1 with Ar the
    balance (Section 4.1)."""
    rng = np.random.Generator(np.random.PCG64(seed0))
    pts = []
    for k in range(n):
        I = 2.0 * k / max(n - 1, 1)
        xh = float(rng.uniform(0.2, 0.8))
        pts.append((I, (xh, xh / 4.0, 1.0 - 1.25 * xh)))
    return pts


TABLE2_CURRENTS = (0.3, 0.7, 1.0)            # A/cm2, Figs. 2-4
TABLE2_H2 = (0.8, 0.6, 0.4, 0.3, 0.2)        # inlet H2 fraction; 0.8 (no Ar) is the eta_0 run


def table2_inlet(xh: float) -> tuple:
    """Inlet composition of Section 4.2: H2:H2O = 4:1 diluted by Ar."""
    return (xh, xh / 4.0, 1.0 - 1.25 * xh)


def paper_table2_cases(nx: int = 64):
    """The homogenised anode of Section 4.2 (Table 2 gas point, eps/tau =
    0.46/4.5, d_p = 2.6 um, L = 2 mm) as a 1-D all-fluid D2Q9 strip, for every
    current of ``TABLE2_CURRENTS`` times every inlet of ``TABLE2_H2``
    (current-major order)."""
    out = []
    for I in TABLE2_CURRENTS:
        for xh in TABLE2_H2:
            out.append(open_channel(nx, 1, gas=PAPER_TABLE2, current_A_cm2=I, x_in=table2_inlet(xh),
                                    name=f"table2_nx{nx}_I{I}_xH2{xh}"))
    return out


def warmstart_cases(n: int, seed0: int, shape=(32, 32, 64)):
    """Anodes for the learned warm start, sampled in the style of the
    batched sweep at one grid size: spheres of radius 2-4, porosity
    U(0.35, 0.50), current U(0.25, 1.5) A/cm2, inlet H2 U(0.3, 0.8) at
    H2:H2O = 4:1 with Ar the balance; case k uses seed seed0 + k."""
    out = []
    for k in range(n):
        rng = np.random.Generator(np.random.PCG64(seed0 + k))
        por = float(rng.uniform(0.35, 0.50))
        rad = int(rng.integers(2, 5))
        I = float(rng.uniform(0.25, 1.5))
        xh = float(rng.uniform(0.3, 0.8))
        out.append(porous(shape, radius=rad, porosity=por, seed=seed0 + k, current_A_cm2=I,
                          x_in=(xh, xh / 4.0, 1.0 - 1.25 * xh),
                          name=f"ws{seed0 + k}_{'x'.join(map(str, shape[::-1]))}_eps{por:.2f}_r{rad}"))
    return out
