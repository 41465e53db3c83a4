"""Seeded synthetic porous-anode microstructures (solid voxel masks).

This module only draws geometry: it holds none of the transport arithmetic, so
both the CPU oracle and the CUDA path take their masks from here.

Recipe (the paper resolves no pores itself: its anode in Section 4.1 is a
homogenised 2 mm x 20 mm slab; these masks stand in for a resolved anode):

* overlapping disks (2-D) or spheres (3-D) of a fixed radius, centres drawn
  uniformly on integer lattice sites by a PCG64 generator seeded with ``seed``;
* y (and z) are periodic, x is not: balls are clipped at x = 0 and x = nx-1;
* balls are added one at a time until the solid fraction first reaches
  ``1 - porosity`` (the last ball may overshoot);
* the inlet column x = 0 and the outlet column x = nx-1 are forced fluid, so
  the Dirichlet inlet and the reacting outlet act on every boundary node;
* fluid that is not face-connected to the inlet column (periodic wrap
  included) is turned solid; if the outlet column is not reached, the draw is
  repeated with ``seed + 1000 * k``.

Arrays are indexed ``[z, y, x]`` (``nz == 1`` in 2-D), ``True`` = solid.
"""
from __future__ import annotations

import numpy as np

__all__ = ["overlapping_balls", "porosity_of", "Microstructure"]


class Microstructure:
    """A solid mask with the parameters it was drawn from."""

    def __init__(self, solid: np.ndarray, radius: int, target_porosity: float,
                 seed: int, seed_used: int):
        self.solid = solid
        self.radius = radius
        self.target_porosity = target_porosity
        self.seed = seed
        self.seed_used = seed_used

    @property
    def porosity(self) -> float:
        return porosity_of(self.solid)

    @property
    def n_fluid(self) -> int:
        return int((~self.solid).sum())


def porosity_of(solid: np.ndarray) -> float:
    return float((~solid).sum()) / solid.size


def _ball_offsets(radius: int, dim: int) -> np.ndarray:
    r = int(radius)
    rng = np.arange(-r, r + 1)
    if dim == 2:
        dy, dx = np.meshgrid(rng, rng, indexing="ij")
        keep = dx * dx + dy * dy <= r * r
        return np.stack([np.zeros(keep.sum(), np.int64), dy[keep], dx[keep]], axis=1)
    dz, dy, dx = np.meshgrid(rng, rng, rng, indexing="ij")
    keep = dx * dx + dy * dy + dz * dz <= r * r
    return np.stack([dz[keep], dy[keep], dx[keep]], axis=1)


def _paint(shape, radius, porosity, seed):
    nz, ny, nx = shape
    dim = 2 if nz == 1 else 3
    rng = np.random.Generator(np.random.PCG64(seed))
    off = _ball_offsets(radius, dim)
    solid = np.zeros(shape, dtype=bool)
    flat = solid.reshape(-1)
    target = (1.0 - porosity) * solid.size
    count = 0
    while count < target:
        cz = int(rng.integers(0, nz)) if dim == 3 else 0
        cy = int(rng.integers(0, ny))
        cx = int(rng.integers(0, nx))
        z = (cz + off[:, 0]) % nz
        y = (cy + off[:, 1]) % ny
        x = cx + off[:, 2]
        inside = (x >= 0) & (x < nx)
        idx = np.unique((z[inside] * ny + y[inside]) * nx + x[inside])
        count += int((~flat[idx]).sum())
        flat[idx] = True
    return solid


def _connected_to_inlet(fluid: np.ndarray) -> np.ndarray:
    """Fluid cells face-connected to the x = 0 column, y/z periodic."""
    from scipy import ndimage
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components

    nz, ny, nx = fluid.shape
    structure = ndimage.generate_binary_structure(3, 1)
    labels, nlab = ndimage.label(fluid, structure=structure)
    if nlab == 0:
        return np.zeros_like(fluid)
    pairs = []
    # glue labels across the periodic y faces (and z faces in 3-D)
    a, b = labels[:, 0, :], labels[:, ny - 1, :]
    m = (a > 0) & (b > 0)
    pairs.append(np.stack([a[m], b[m]], 1))
    if nz > 1:
        a, b = labels[0, :, :], labels[nz - 1, :, :]
        m = (a > 0) & (b > 0)
        pairs.append(np.stack([a[m], b[m]], 1))
    p = np.concatenate(pairs, 0) if pairs else np.zeros((0, 2), np.int64)
    n = nlab + 1
    g = coo_matrix((np.ones(len(p)), (p[:, 0], p[:, 1])), shape=(n, n))
    _, comp = connected_components(g, directed=False)
    inlet_labels = np.unique(labels[:, :, 0])
    inlet_labels = inlet_labels[inlet_labels > 0]
    keep_comp = np.unique(comp[inlet_labels])
    keep_label = np.isin(comp, keep_comp)
    keep_label[0] = False
    return keep_label[labels]


def overlapping_balls(shape, radius: int, porosity: float, seed: int,
                      max_tries: int = 20) -> Microstructure:
    """Draw a percolating mask of overlapping disks/spheres.

    ``shape`` is ``(ny, nx)`` for 2-D or ``(nz, ny, nx)`` for 3-D.
    """
    shape = tuple(int(s) for s in shape)
    if len(shape) == 2:
        shape = (1,) + shape
    nz, ny, nx = shape
    if nx < 3:
        raise ValueError("nx must be >= 3")
    for k in range(max_tries):
        s = seed + 1000 * k
        solid = _paint(shape, radius, porosity, s)
        solid[:, :, 0] = False
        solid[:, :, nx - 1] = False
        keep = _connected_to_inlet(~solid)
        if keep[:, :, nx - 1].all():
            return Microstructure(~keep, radius, porosity, seed, s)
    raise RuntimeError("no percolating draw found")
