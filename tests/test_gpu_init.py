"""The initial state of Section 4.1 (init_mode "profile1d"): every column at
the 1-D profile of Eq. 19 with the fluxes held at their outlet values,
checked against the closed-form ternary profile, and its effect on the
number of steps to steady state."""
import numpy as np
import pytest

from closed_forms import ternary_1d
from oracle.gas import Scaling
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


def _profile(c):
    nx = c.shape[-1]
    sc = Scaling(c.gas, nx, c.length_x, c.current_A_cm2)
    x = np.arange(nx) * sc.dx
    return ternary_1d(x, c.x_in, sc.N_out[0], sc.C_t, sc.D_eff[0, 1], sc.D_eff[0, 2], sc.D_eff[1, 2])


@pytest.mark.parametrize("gas", [cases.Gas(), cases.PAPER_TABLE2])
def test_initial_field_is_the_closed_form_profile(L, gas):
    c = cases.open_channel(48, 3, current_A_cm2=1.0, gas=gas)
    s = L.Solver.from_case(c, precision="fp64", init_mode="profile1d")
    s.set_bc(c.x_in, c.current_A_cm2)
    X = s.fields()
    Xc = _profile(c)
    assert np.abs(X - Xc[:, None, None, :]).max() < 1e-12


def test_porous_columns_share_the_profile(L):
    c = cases.anode_3d_small(nx=32, ny=12, nz=10)
    s = L.Solver.from_case(c, precision="fp32", init_mode="profile1d")
    s.set_bc(c.x_in, c.current_A_cm2)
    X = s.fields()
    Xc = _profile(c)
    f = ~c.solid
    want = np.broadcast_to(Xc[:, None, None, :], X.shape)
    assert np.abs(X - want)[:, f].max() < 1e-7
    assert np.all(X[:, c.solid] == 0.0)


def test_profile_start_reaches_steady_state_sooner(L):
    c = cases.open_channel(48, 1, current_A_cm2=1.0)
    n = {}
    for mode in ("uniform", "profile1d"):
        s = L.Solver.from_case(c, precision="fp64", init_mode=mode)
        s.set_bc(c.x_in, c.current_A_cm2)
        n[mode], r, _ = s.run_to_residual(1e-11, 2_000_000)
        n[mode + "_eta"] = s.overpotential()[0]
    assert n["profile1d"] < 0.5 * n["uniform"]
    assert n["profile1d_eta"] == pytest.approx(n["uniform_eta"], rel=1e-6)


def test_depleting_profile_is_an_error(L):
    """At 3 A/cm2 with little H2 the held-flux profile crosses zero."""
    c = cases.open_channel(24, 1, current_A_cm2=3.0, x_in=(0.05, 0.1, 0.85))
    s = L.Solver.from_case(c, precision="fp64", init_mode="profile1d")
    with pytest.raises(L.LbmsError) as e:
        s.set_bc(c.x_in, c.current_A_cm2)
    assert e.value.status == L.LBMS_EDEPLETED
