"""GPU parity: the CUDA solver (through the C ABI) against the FP64 oracle on
the same seeded inputs, element by element.

Tolerances: FP64 kernels agree with the oracle to rounding (the two sum in
different orders), bounded here by 1e-11 absolute on mole fractions after up
to a few thousand steps; FP32 kernels to 1e-6 absolute on mole fractions
(the stated single-precision target), tau to 5e-4; FP16-stored populations
(FP32 arithmetic) to 2e-5 absolute on mole fractions over a few hundred
steps and 1e-4 relative on the overpotential at steady state.
"""
import numpy as np
import pytest

from oracle import Oracle
from workloads import cases

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11
FP32_TOL = 1e-6
FP16_TOL = 2e-5


@pytest.fixture(scope="module")
def lbms():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_01600_gb300 import lbms as L
    L.load()
    return L


def make_pair(L, case, precision="fp64", X0=None, **kw):
    s = L.Solver.from_case(case, precision=precision, **kw)
    s.set_bc(case.x_in, case.current_A_cm2)
    o = Oracle(case, dt=kw.get("dt") or None, tau_min=kw.get("tau_min", 1.0),
               tau_max=kw.get("tau_max", 5.0), coupling=kw.get("coupling", "ms"))
    if X0 is not None:
        s.set_fields(X0)
        o.init(X0)
    return s, o


def smooth_field(shape, seed, amp=0.05):
    rng = np.random.Generator(np.random.PCG64(seed))
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    X = np.empty((3,) + tuple(shape))
    ph = rng.random(6) * 2 * np.pi
    X[0] = 0.5 + amp * np.sin(2 * np.pi * x / nx + ph[0]) * np.cos(2 * np.pi * y / ny + ph[1])
    X[2] = 0.35 + amp * np.cos(2 * np.pi * x / nx + ph[2]) * np.sin(2 * np.pi * (y / ny + z / max(nz, 1)) + ph[3])
    X[1] = 1.0 - X[0] - X[2]
    return X


def compare(s, o, tol, what=""):
    X, u, tau = s.fields(u=True, tau=True)
    f = ~o.solid
    Xo, uo, tauo = o.fields()
    err = np.abs(X - Xo)[:, f].max()
    assert err <= tol, f"{what}: max |dX| = {err:.3e}"
    scale_u = max(np.abs(uo).max(), 1e-30)
    assert np.abs(u - uo)[:, :, f].max() <= max(1e3 * tol, 1e-6) * scale_u + 1e-300, what
    assert np.abs(tau - tauo)[:, f].max() <= max(1e3 * tol, 1e-4) * 5.0, what
    return err


# ------------------------------------------------------------ FP64 steps
STEP_CASES = [
    ("open1d_d2q9", lambda: cases.open_channel(40, 1, current_A_cm2=2.0)),
    ("open1d_d3q19", lambda: cases.open_channel(40, 1, dim=3, current_A_cm2=2.0)),
    ("porous2d_48x40", lambda: cases.porous((40, 48), radius=3, porosity=0.55, seed=21, current_A_cm2=1.5)),
    ("porous3d_20x16x12", lambda: cases.porous((12, 16, 20), radius=2, porosity=0.5, seed=22, current_A_cm2=1.5)),
]


@pytest.mark.parametrize("name,make", STEP_CASES, ids=[c[0] for c in STEP_CASES])
def test_fp64_step_parity(lbms, name, make):
    case = make()
    X0 = smooth_field(case.solid.shape, 5)
    s, o = make_pair(lbms, case, "fp64", X0=X0)
    done = 0
    for n in (1, 9, 190, 800):
        s.step(n)
        o.step(n)
        done += n
        compare(s, o, FP64_TOL, f"{name} after {done} steps")
    eta, xo = s.overpotential()
    assert eta == pytest.approx(o.overpotential(), rel=1e-10, abs=1e-14)
    assert np.allclose(xo, o.outlet_mean(), rtol=0, atol=1e-12)
    s.close()


def test_fp64_step_parity_cfg_96x48(lbms):
    """The 2-D D2Q9 96x48 anode (disks r = 4, porosity 0.45, 0.5 A/cm2) from
    the uniform inlet start, 3000 steps."""
    case = cases.anode_2d_96x48()
    s, o = make_pair(lbms, case, "fp64")
    s.step(3000)
    o.step(3000)
    compare(s, o, FP64_TOL, "96x48 after 3000 steps")
    eta, _ = s.overpotential()
    assert eta == pytest.approx(o.overpotential(), rel=1e-9)


def test_tau_only_coupling_parity(lbms):
    case = cases.porous((24, 32), radius=3, porosity=0.55, seed=23, current_A_cm2=1.0)
    s, o = make_pair(lbms, case, "fp64", X0=smooth_field(case.solid.shape, 6), coupling="tau_only")
    s.step(300)
    o.step(300)
    compare(s, o, FP64_TOL, "tau_only")


def test_closed_box_conservation_and_parity(lbms):
    case = cases.porous((10, 12, 18), radius=2, porosity=0.55, seed=24).with_(periodic_x=True)
    X0 = smooth_field(case.solid.shape, 7)
    s, o = make_pair(lbms, case, "fp64", X0=X0)
    _, tot0 = s.boundary_flux()
    s.step(400)
    o.step(400)
    compare(s, o, FP64_TOL, "closed box")
    _, tot = s.boundary_flux()
    assert np.allclose(tot, tot0, rtol=1e-13)
    assert np.allclose(tot, o.total(), rtol=1e-13)


def test_pulse_variance_on_gpu(lbms):
    """Exact lattice variance law with equal diffusivities (tau = 2)."""
    import sys
    from closed_forms import pulse_variance
    n = 600
    shape = (1, 1, n)
    gas = cases.Gas(D_binary=np.full((3, 3), 2e-4), pore_diameter=0.0)
    case = cases.Case(name="pulse", solid=np.zeros(shape, bool), dim=3, periodic_x=True, gas=gas,
                      length_x=1e-3 * n)
    dt = 3.0 * (1e-3) ** 2 / (6.0 * 2e-4)
    X0 = cases.gaussian_pulse(shape, 0, sigma0=3.0, amplitude=0.05)
    s, o = make_pair(lbms, case, "fp64", X0=X0, dt=dt)
    s.step(1000)
    X, tau = s.fields(tau=True)
    assert np.allclose(tau[0], 2.0, rtol=1e-12)
    pulse = X[0].reshape(-1) - 0.3
    x = np.arange(n) - (n - 1) / 2.0
    var = (x * x * pulse).sum() / pulse.sum()
    assert var == pytest.approx(pulse_variance(1000, 9.0, 2.0), rel=1e-9)


def test_graph_replay_equals_single_steps(lbms):
    case = cases.porous((20, 30), radius=3, porosity=0.55, seed=25, current_A_cm2=1.0)
    X0 = smooth_field(case.solid.shape, 8)
    # one forced kernel variant for both handles: the autotuner times each
    # handle separately and may pick variants that round differently
    a = lbms.Solver.from_case(case, precision="fp32", step_variant=7)
    b = lbms.Solver.from_case(case, precision="fp32", step_variant=7)
    for s in (a, b):
        s.set_bc(case.x_in, case.current_A_cm2)
        s.set_fields(X0)
    a.step(101)                 # 3 graph replays of 32 steps + 5 single steps
    for _ in range(101):
        b.step(1)
    assert np.array_equal(a.fields(), b.fields())
    assert a.info().steps == b.info().steps == 101


# ------------------------------------------------------------ FP32 steps
def test_fp32_parity_porous_3d(lbms):
    """Reduced 3-D anode with the 256x128x128 recipe (spheres r = 3,
    porosity 0.40, seed 2, 1 A/cm2): FP32 against the FP64 oracle."""
    case = cases.anode_3d_small()
    X0 = smooth_field(case.solid.shape, 9, amp=0.02)
    s, o = make_pair(lbms, case, "fp32", X0=X0)
    for n in (1, 49, 250):
        s.step(n)
        o.step(n)
    X, tau = s.fields(tau=True)
    f = ~case.solid
    assert np.abs(X - o.X)[:, f].max() <= FP32_TOL
    assert np.abs(tau - o.tau)[:, f].max() <= 1e-4 * 5.0
    eta, _ = s.overpotential()
    assert eta == pytest.approx(o.overpotential(), rel=1e-4)


def test_fp32_parity_2d(lbms):
    case = cases.anode_2d_96x48()
    s, o = make_pair(lbms, case, "fp32")
    s.step(2000)
    o.step(2000)
    X = s.fields()
    f = ~case.solid
    assert np.abs(X - o.X)[:, f].max() <= FP32_TOL


@pytest.mark.parametrize("dim", [2, 3])
def test_fp16_step_parity(lbms, dim):
    """FP16-stored populations (FP32 arithmetic) against the FP64 oracle."""
    if dim == 2:
        case = cases.porous((40, 48), radius=3, porosity=0.55, seed=21, current_A_cm2=1.5)
    else:
        case = cases.anode_3d_small()
    X0 = smooth_field(case.solid.shape, 12, amp=0.02)
    s, o = make_pair(lbms, case, "fp16", X0=X0)
    s.step(300)
    o.step(300)
    X = s.fields()
    f = ~case.solid
    assert np.abs(X - o.X)[:, f].max() <= FP16_TOL


# ------------------------------------------------------ steady states
def test_steady_state_parity_and_flux_balance(lbms):
    """Both sides run to residual 1e-12 (FP64); fields, eta and the inlet flux
    (which must equal the Eq. 39 outlet flux; zero for Ar) agree."""
    case = cases.porous((12, 20), radius=2, porosity=0.6, seed=7, current_A_cm2=1.0)
    s, o = make_pair(lbms, case, "fp64")
    n, r, st = s.run_to_residual(1e-12, 400000)
    no, ro = o.run_to_residual(1e-12, 400000, 100)
    assert r <= 1e-12 and ro <= 1e-12
    X = s.fields()
    f = ~case.solid
    assert np.abs(X - o.X)[:, f].max() <= 1e-9
    eta, _ = s.overpotential()
    assert eta == pytest.approx(o.overpotential(), rel=1e-7)
    flux, _ = s.boundary_flux()
    info = s.info()
    n_out = case.solid.shape[0] * case.solid.shape[1]
    assert flux[0] == pytest.approx(info.q_lat[0] * n_out, rel=1e-7)
    assert flux[1] == pytest.approx(info.q_lat[1] * n_out, rel=1e-7)
    assert abs(flux[2]) < 1e-7 * abs(info.q_lat[0]) * n_out
    assert np.allclose(flux, o.plane_flux()[:, 0], rtol=1e-6, atol=1e-12)


@pytest.mark.parametrize("precision,xtol", [("fp32", FP32_TOL), ("fp16", 1e-5)])
def test_steady_state_single_and_half_precision(lbms, precision, xtol):
    """Steady state in FP32 (mole fractions within 1e-6 of the FP64 oracle)
    and with FP16 storage (overpotential within 1e-4 relative)."""
    case = cases.porous((12, 20), radius=2, porosity=0.6, seed=7, current_A_cm2=1.0)
    s = lbms.Solver.from_case(case, precision=precision)
    s.set_bc(case.x_in, case.current_A_cm2)
    # the FP32 pair state jitters by about one FP32 ulp at steady state
    # (residual floor ~1e-10 at K = 100); FP16 storage by more
    tol = 1e-9 if precision == "fp32" else 1e-8
    n, r, st = s.run_to_residual(tol, 400000, raise_on_fail=False)
    s.step(20000)      # well past the tolerance: the state stays put
    o = Oracle(case)
    o.run_to_residual(1e-12, 400000, 100)
    X = s.fields()
    f = ~case.solid
    err = np.abs(X - o.X)[:, f].max()
    eta, _ = s.overpotential()
    assert eta == pytest.approx(o.overpotential(), rel=1e-4)
    assert st == lbms.LBMS_OK and r <= tol
    assert err <= xtol


def test_lattice_constants_match_oracle(lbms):
    case = cases.anode_3d_small()
    s = lbms.Solver.from_case(case)
    s.set_bc(case.x_in, case.current_A_cm2)
    o = Oracle(case)
    i = s.info()
    assert i.n_fluid == case.n_fluid and i.q == 19
    assert i.dx_m == pytest.approx(o.sc.dx, rel=1e-15)
    assert i.dt_s == pytest.approx(o.sc.dt, rel=1e-14)
    assert i.C_t == pytest.approx(o.sc.C_t, rel=1e-15)
    assert np.allclose(np.array(i.D_eff_m2s).reshape(3, 3), o.sc.D_eff, rtol=1e-14)
    assert np.allclose(np.array(i.q_lat), o.sc.q_lat, rtol=1e-14, atol=0)


# -------------------------------------------- full size (256x128x128)
@pytest.mark.slow
def test_full_size_fp32_two_steps_against_oracle(lbms):
    """At the full 256x128x128 size, in the FP32 launch configuration the
    benchmark times: two steps from a non-uniform start, every cell."""
    case = cases.anode_3d_256x128x128()
    X0 = smooth_field(case.solid.shape, 10, amp=0.02)
    s, o = make_pair(lbms, case, "fp32", X0=X0)
    s.step(2)
    o.step(2)
    X = s.fields()
    f = ~case.solid
    assert np.abs(X - o.X)[:, f].max() <= FP32_TOL


@pytest.mark.slow
def test_full_size_fp32_closed_box_conservation(lbms):
    case = cases.anode_3d_256x128x128().with_(periodic_x=True)
    s = lbms.Solver.from_case(case, precision="fp32")
    s.set_bc(case.x_in, 0.0)
    s.set_fields(smooth_field(case.solid.shape, 11, amp=0.02))
    _, tot0 = s.boundary_flux()
    s.step(1000)
    _, tot = s.boundary_flux()
    assert np.allclose(tot, tot0, rtol=1e-9)


@pytest.mark.parametrize("precision,rtol", [("fp32", 3e-10), ("fp16", 1e-7)])
def test_closed_box_conservation_low_precision(lbms, precision, rtol):
    """Streaming exchanges w_k (X(src) - X(x)) + h_k terms that cancel
    exactly between cells, and the rest population closes sum_k h_k = 0 on
    the stored values: each species is conserved to rounding."""
    case = cases.porous((10, 12, 18), radius=2, porosity=0.55, seed=24).with_(periodic_x=True)
    s = lbms.Solver.from_case(case, precision=precision)
    s.set_bc(case.x_in, 0.0)
    s.set_fields(smooth_field(case.solid.shape, 7))
    _, tot0 = s.boundary_flux()
    s.step(1000)
    _, tot = s.boundary_flux()
    # relative bounds a few times the measured drift (1.2e-10 FP32, 2.9e-8
    # FP16): the roundings that do not cancel are u * sum|d_k| per cell and
    # step, summed over cells and the ~100 steps the start takes to smooth out
    assert np.all(np.abs(tot / tot0 - 1.0) <= rtol)


# ------------------------------------------------------ error handling
def test_nan_field_is_reported_unstable(lbms):
    case = cases.open_channel(16, 4)
    s = lbms.Solver.from_case(case)
    s.set_bc(case.x_in, 1.0)
    X = np.empty((3,) + case.solid.shape)
    X[:] = np.array(case.x_in).reshape(3, 1, 1, 1)
    X[0, 0, 2, 5] = np.nan
    s.set_fields(X)
    s.step(3)
    with pytest.raises(lbms.LbmsError) as e:
        s.residual(3)
    assert e.value.status == lbms.LBMS_EUNSTABLE
    n, r, st = s.run_to_residual(1e-8, 200, raise_on_fail=False)
    assert st == lbms.LBMS_EUNSTABLE


def test_out_of_order_and_bad_bc(lbms):
    case = cases.open_channel(16, 4)
    s = lbms.Solver.from_case(case)
    with pytest.raises(lbms.LbmsError) as e:
        s.step(1)
    assert e.value.status == lbms.LBMS_ESTATE
    with pytest.raises(lbms.LbmsError) as e:
        s.set_bc((0.5, 0.5, 0.5), 1.0)
    assert e.value.status == lbms.LBMS_EINVAL
    with pytest.raises(lbms.LbmsError) as e:
        s.set_bc((0.5, 0.1, 0.4), -1.0)
    assert e.value.status == lbms.LBMS_EINVAL


def test_depletion_is_reported(lbms):
    """Eq. 43 needs X_H2O,in > 0 and X_H2,out > 0; without inlet steam the
    logarithm is undefined and the call says so."""
    case = cases.open_channel(16, 1, current_A_cm2=0.5, x_in=(0.6, 0.0, 0.4))
    s = lbms.Solver.from_case(case, precision="fp64")
    s.set_bc(case.x_in, case.current_A_cm2)
    s.step(10)
    with pytest.raises(lbms.LbmsError) as e:
        s.overpotential()
    assert e.value.status == lbms.LBMS_EDEPLETED


def test_extrapolation_keeps_the_steady_state_and_saves_steps(lbms):
    """Aitken extrapolation of the slowest mode (extrapolate_every) reaches
    the same steady state in fewer steps."""
    case = cases.anode_2d_96x48()
    runs = {}
    for W in (0, 2000):
        s = lbms.Solver.from_case(case, precision="fp64", extrapolate_every=W)
        s.set_bc(case.x_in, case.current_A_cm2)
        n, r, st = s.run_to_residual(1e-11, 2_000_000)
        assert st == lbms.LBMS_OK and r <= 1e-11
        runs[W] = (n, s.fields(), s.overpotential()[0])
        s.close()
    (n0, X0, eta0), (n1, X1, eta1) = runs[0], runs[2000]
    f = ~case.solid
    assert n1 < 0.8 * n0
    assert np.abs(X0 - X1)[:, f].max() < 1e-6
    assert eta1 == pytest.approx(eta0, rel=1e-5)


@pytest.mark.parametrize("modes", [2, 4])
def test_reduced_rank_extrapolation_keeps_the_steady_state(lbms, modes):
    """Reduced-rank extrapolation (extrapolate_modes >= 2) over snapshots W
    steps apart reaches the same steady state as plain stepping, with fewer
    steps than the plain run, on the 96x48 anode (FP64) and on a batch of
    two anodes whose cases extrapolate separately."""
    case = cases.anode_2d_96x48()
    f = ~case.solid
    ref = lbms.Solver.from_case(case, precision="fp64")
    ref.set_bc(case.x_in, case.current_A_cm2)
    n0, r0, st = ref.run_to_residual(1e-11, 2_000_000)
    assert st == lbms.LBMS_OK
    X0, eta0 = ref.fields(), ref.overpotential()[0]
    ref.close()
    s = lbms.Solver.from_case(case, precision="fp64", extrapolate_every=2000, extrapolate_modes=modes)
    s.set_bc(case.x_in, case.current_A_cm2)
    n1, r1, st = s.run_to_residual(1e-11, 2_000_000)
    assert st == lbms.LBMS_OK and r1 <= 1e-11
    assert n1 < 0.8 * n0
    assert np.abs(s.fields() - X0)[:, f].max() < 1e-6
    assert s.overpotential()[0] == pytest.approx(eta0, rel=1e-5)
    s.close()
    other = cases.porous((30, 60), radius=3, porosity=0.55, seed=27, current_A_cm2=1.5)
    b = lbms.Batch.from_cases([case, other], precision="fp64", extrapolate_every=2000, extrapolate_modes=modes)
    b.set_bc(case.x_in, case.current_A_cm2, case=0)
    b.set_bc(other.x_in, other.current_A_cm2, case=1)
    n, steps, r, st = b.run_to_residual(1e-11, 2_000_000)
    assert st == lbms.LBMS_OK and np.all(r <= 1e-11)
    assert np.abs(b.fields(0) - X0)[:, f].max() < 1e-6
    o = lbms.Solver.from_case(other, precision="fp64")
    o.set_bc(other.x_in, other.current_A_cm2)
    o.run_to_residual(1e-11, 2_000_000)
    g = ~other.solid
    assert np.abs(b.fields(1) - o.fields())[:, g].max() < 1e-6
    b.close()
    o.close()
