"""Batched stepping: every case of a batch evolves as the same case in a
handle of its own, to rounding (the autotuner may pick another tile shape,
whose instantiation can contract floating-point operations differently);
per-case residuals, convergence counts and overpotentials."""
import numpy as np
import pytest

from oracle import Oracle
from workloads import cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_01600_gb300 import lbms
    lbms.load()
    return lbms


def _cases_2d():
    shapes = [(24, 40), (17, 33), (40, 64)]
    out = []
    for k, sh in enumerate(shapes):
        c = cases.porous(sh, radius=3, porosity=0.55, seed=40 + k)
        out.append(c)
    return out


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 1e-7), ("fp16", 1e-6)])
def test_batch_equals_single_cases_2d(L, precision, tol):
    cs = _cases_2d()
    ops = [(0.5, (0.5, 0.1, 0.4)), (1.5, (0.3, 0.075, 0.625)), (1.0, (0.6, 0.15, 0.25))]
    b = L.Batch.from_cases(cs, precision=precision)
    for k, (I, x) in enumerate(ops):
        b.set_bc(x, I, case=k)
    info = b.info()
    assert info.n_cases == 3 and info.tile_cells in (32, 64)
    b.step(137)
    eta_b, xo_b = b.overpotentials()
    for k, (c, (I, x)) in enumerate(zip(cs, ops)):
        s = L.Solver.from_case(c, precision=precision)
        s.set_bc(x, I)
        s.step(137)
        Xs = s.fields()
        Xb = b.fields(k)
        assert np.abs(Xs - Xb).max() <= tol, f"case {k}: {np.abs(Xs - Xb).max():.3e}"
        eta, xo = s.overpotential()
        assert eta_b[k] == pytest.approx(eta, rel=max(tol, 1e-12) * 100, abs=1e-15)
        s.close()


def test_batch_3d_matches_oracle_and_residuals(L):
    cs = [cases.porous((10, 12, 20), radius=2, porosity=0.5, seed=51),
          cases.porous((8, 8, 16), radius=2, porosity=0.6, seed=52)]
    b = L.Batch.from_cases(cs, precision="fp64")
    b.set_bc((0.5, 0.1, 0.4), 1.0, case=0)
    b.set_bc((0.4, 0.1, 0.5), 2.0, case=1)
    b.residuals(1)
    b.step(50)
    r = b.residuals(50)
    assert r.shape == (2,) and np.all(r > 0)
    o = Oracle(cs[1].with_(current_A_cm2=2.0, x_in=(0.4, 0.1, 0.5)))
    o.step(50)
    f = ~cs[1].solid
    assert np.abs(b.fields(1) - o.X)[:, f].max() <= 1e-11


def test_batch_run_to_residual_reports_each_case(L):
    small = cases.porous((8, 12), radius=2, porosity=0.6, seed=61)
    large = cases.porous((16, 48), radius=2, porosity=0.6, seed=62)
    b = L.Batch.from_cases([small, large], precision="fp64")
    b.set_bc((0.5, 0.1, 0.4), 1.0)
    n, steps, r, st = b.run_to_residual(1e-9, 400000)
    assert st == L.LBMS_OK
    assert 0 < steps[0] < steps[1] <= n
    assert np.all(r <= 1e-9)


def test_batch_rejects_mixed_dims(L):
    a = cases.porous((8, 12), radius=2, porosity=0.6, seed=61)
    c = cases.porous((8, 8, 12), radius=2, porosity=0.6, seed=63)
    with pytest.raises(L.LbmsError) as e:
        L.Batch([a.solid, c.solid], dim=None)
    assert e.value.status == L.LBMS_EINVAL


@pytest.mark.parametrize("variant", list(range(1, 11)))
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 1e-7)])
def test_every_step_variant_gives_the_same_fields(L, variant, precision, tol):
    """All tile shapes, all three neighbour lookups (32-bit indices, 16-bit
    offsets, row bitmasks) and both thread mappings (one thread per cell and
    species, one per cell) the autotuner may pick compute the same step (to
    rounding of FMA contraction)."""
    c = cases.porous((12, 14, 30), radius=2, porosity=0.5, seed=71, current_A_cm2=1.5)
    ref = L.Solver.from_case(c, precision=precision, step_variant=1)
    s = L.Solver.from_case(c, precision=precision, step_variant=variant)
    for h in (ref, s):
        h.set_bc(c.x_in, c.current_A_cm2)
        h.step(77)
    i = s.info()
    assert i.neighbour_bits == (16 if 4 <= variant <= 6 else (1 if variant >= 9 else 32))
    assert i.threads_per_cell == (1 if variant >= 7 else 3)
    assert np.abs(s.fields() - ref.fields()).max() <= tol


@pytest.mark.parametrize("variant", [1, 4])
def test_far_links_of_the_16_bit_table(L, variant):
    """A box long in z: the periodic wrap in z gives offsets beyond 16 bits,
    which the 16-bit table sends to the 32-bit table."""
    c = cases.porous((96, 40, 24), radius=2, porosity=0.5, seed=72, current_A_cm2=1.0)
    o = Oracle(c)
    s = L.Solver.from_case(c, precision="fp64", step_variant=variant)
    s.set_bc(c.x_in, c.current_A_cm2)
    s.step(40)
    o.step(40)
    assert s.info().neighbour_bits == (16 if variant >= 4 else 32)
    f = ~c.solid
    assert np.abs(s.fields() - o.X)[:, f].max() <= 1e-11


@pytest.mark.parametrize("variant", [9, 10])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 1e-6), ("fp16", 2e-5)])
def test_row_bitmask_decode_against_oracle(L, variant, precision, tol):
    """The neighbour decode from per-row fluid bitmasks (variants 9-10): a
    batch of a 3-D anode wider than one 32-voxel word (x = 70, so windows
    straddle words), with periodic wraps in y and z, and a 2-D strip one
    voxel high (ny = 1: every y neighbour is the cell itself), against the
    oracle."""
    for cs in ([cases.porous((6, 9, 70), radius=2, porosity=0.5, seed=73, current_A_cm2=1.5),
                cases.porous((5, 7, 33), radius=2, porosity=0.6, seed=74, current_A_cm2=0.5)],
               [cases.open_channel(40, 1, current_A_cm2=2.0),
                cases.porous((11, 65), radius=2, porosity=0.55, seed=75, current_A_cm2=1.0)]):
        b = L.Batch.from_cases(cs, precision=precision, step_variant=variant)
        for k, c in enumerate(cs):
            b.set_bc(c.x_in, c.current_A_cm2, case=k)
        assert b.info().neighbour_bits == 1
        b.step(60)
        for k, c in enumerate(cs):
            o = Oracle(c)
            o.step(60)
            f = ~c.solid
            assert np.abs(b.fields(k) - o.X)[:, f].max() <= tol, (c.name, precision)
        b.close()


def test_row_bitmask_variant_needs_a_box_open_in_x(L):
    c = cases.porous((8, 12), radius=2, porosity=0.6, seed=61).with_(periodic_x=True)
    s = L.Solver.from_case(c, precision="fp64", step_variant=9)
    with pytest.raises(L.LbmsError) as e:
        s.set_bc(c.x_in, 0.0)
    assert e.value.status == L.LBMS_EINVAL and "row-bitmask" in str(e.value)
    s.close()
    s = L.Solver.from_case(c, precision="fp64")      # the autotuner skips those variants
    s.set_bc(c.x_in, 0.0)
    assert s.info().neighbour_bits in (16, 32)
    s.close()


@pytest.mark.slow
def test_full_sweep_launch_sampled_cases_against_oracle(L):
    """A full-size batched sweep (8 2-D + 8 3-D seeded microstructures of the
    benchmark's recipe x 8 operating points, 128 cases, ~61M fluid cells, one
    FP32 launch per lattice and step; the benchmark itself runs 32 + 32):
    two sampled cases - the largest 3-D and the largest 2-D grid - start
    from non-uniform fields, and after two batched steps every one of their
    cells matches the oracle run on that case alone."""
    import bench
    args = type("A", (), dict(sweep_2d=8, sweep_3d=8, sweep_scale=1.0, sweep_points=8))()
    groups = bench.sweep_cases(args)
    for dim in (3, 2):
        cs = groups[dim]
        k = int(np.argmax([c.n_cells for c in cs]))
        b = L.Batch.from_cases(cs, precision="fp32")
        for j, c in enumerate(cs):
            b.set_bc(c.x_in, c.current_A_cm2, case=j)
        c = cs[k]
        rng = np.random.Generator(np.random.PCG64(90 + dim))
        nz, ny, nx = c.shape
        x = np.arange(nx)[None, None, :]
        y = np.arange(ny)[None, :, None]
        X0 = np.empty((3,) + c.shape)
        X0[0] = c.x_in[0] + 0.02 * np.sin(2 * np.pi * x / nx + rng.random()) * np.cos(2 * np.pi * y / ny)
        X0[2] = c.x_in[2] + 0.01 * np.cos(2 * np.pi * x / nx)
        X0[1] = 1.0 - X0[0] - X0[2]
        b.set_fields(k, X0)
        b.step(2)
        X = b.fields(k)
        b.close()
        o = Oracle(c)
        o.init(X0)
        o.step(2)
        f = ~c.solid
        assert np.abs(X - o.X)[:, f].max() <= 1e-6, (dim, c.name)
