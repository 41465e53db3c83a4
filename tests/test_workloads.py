"""The seeded microstructure generator: determinism and the stated recipe."""
import numpy as np

from workloads import cases, overlapping_balls


def test_deterministic_and_recipe():
    a = overlapping_balls((24, 40), radius=3, porosity=0.45, seed=1)
    b = overlapping_balls((24, 40), radius=3, porosity=0.45, seed=1)
    c = overlapping_balls((24, 40), radius=3, porosity=0.45, seed=2)
    assert np.array_equal(a.solid, b.solid)
    assert not np.array_equal(a.solid, c.solid)
    for m in (a, c):
        assert not m.solid[:, :, 0].any() and not m.solid[:, :, -1].any()
        assert 0.3 < m.porosity < 0.6


def test_fluid_is_connected_to_inlet():
    from scipy import ndimage
    m = overlapping_balls((10, 12, 20), radius=2, porosity=0.5, seed=3)
    fluid = ~m.solid
    # periodic tiling in y and z then label: every fluid cell of the centre
    # tile must share a label with the inlet column
    t = np.tile(fluid, (3, 3, 1))
    lab, _ = ndimage.label(t, structure=ndimage.generate_binary_structure(3, 1))
    nz, ny, nx = fluid.shape
    centre = lab[nz:2 * nz, ny:2 * ny, :]
    inlet = set(np.unique(lab[:, :, 0])) - {0}
    assert set(np.unique(centre[fluid])) <= inlet


def test_named_workloads_shapes():
    c1 = cases.anode_2d_96x48()
    assert c1.solid.shape == (1, 48, 96) and c1.dim == 2
    assert abs(c1.porosity - 0.45) < 0.05
