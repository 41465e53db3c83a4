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


def test_table2_cases_follow_section_4_2():
    cs = cases.paper_table2_cases(32)
    assert len(cs) == len(cases.TABLE2_CURRENTS) * len(cases.TABLE2_H2)
    for k, c in enumerate(cs):
        I = cases.TABLE2_CURRENTS[k // len(cases.TABLE2_H2)]
        xh = cases.TABLE2_H2[k % len(cases.TABLE2_H2)]
        assert c.current_A_cm2 == I
        assert c.x_in == cases.table2_inlet(xh)
        assert abs(sum(c.x_in) - 1.0) < 1e-15 and c.x_in[0] == 4.0 * c.x_in[1]
        assert c.gas is cases.PAPER_TABLE2 and not c.solid.any()
    assert cs[0].x_in[2] == 0.0           # the eta_0 inlet has no Ar


def test_warmstart_cases_are_seeded_and_in_range():
    a = cases.warmstart_cases(3, 1000, shape=(8, 8, 16))
    b = cases.warmstart_cases(3, 1000, shape=(8, 8, 16))
    for x, y in zip(a, b):
        assert np.array_equal(x.solid, y.solid) and x.x_in == y.x_in and x.current_A_cm2 == y.current_A_cm2
    for c in a:
        assert 0.25 <= c.current_A_cm2 <= 1.5
        assert 0.3 <= c.x_in[0] <= 0.8 and abs(c.x_in[0] - 4 * c.x_in[1]) < 1e-15
        assert not c.solid[:, :, 0].any() and not c.solid[:, :, -1].any()
