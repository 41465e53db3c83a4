"""The literal readings of Eqs. 35 and 37 as options of the CUDA solver
(grad_stencil="forward", outlet_bc="extrapolated") against the same options
of the FP64 oracle, element by element, on porous 2-D and 3-D anodes."""
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


CASES = [
    ("porous2d_48x40", lambda: cases.porous((40, 48), radius=3, porosity=0.55, seed=21, current_A_cm2=1.5)),
    ("porous3d_30x14x12", lambda: cases.porous((12, 14, 30), radius=2, porosity=0.5, seed=23, current_A_cm2=1.5)),
]
OPTIONS = [("forward", "flux"), ("central", "extrapolated"), ("forward", "extrapolated")]


@pytest.mark.parametrize("gs,ob", OPTIONS)
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 1e-6)])
def test_option_parity(L, name, make, gs, ob, precision, tol):
    c = make()
    s = L.Solver.from_case(c, precision=precision, grad_stencil=gs, outlet_bc=ob)
    s.set_bc(c.x_in, c.current_A_cm2)
    o = Oracle(c, grad_stencil=gs, outlet_bc=ob)
    for n in (1, 299):
        s.step(n)
        o.step(n)
    f = ~c.solid
    X, u, tau = s.fields(u=True, tau=True)
    Xo, uo, tauo = o.fields()
    assert np.abs(X - Xo)[:, f].max() <= tol
    assert np.abs(tau - tauo)[:, f].max() <= max(1e3 * tol, 1e-4) * 5.0
    assert np.abs(u - uo)[:, :, f].max() <= max(1e3 * tol, 1e-6) * max(np.abs(uo).max(), 1e-30)


def test_options_change_the_result(L):
    """Each option acts: the three settings give different fields."""
    c = CASES[1][1]()
    out = {}
    for gs, ob in [("central", "flux")] + OPTIONS:
        s = L.Solver.from_case(c, precision="fp64", grad_stencil=gs, outlet_bc=ob)
        s.set_bc(c.x_in, c.current_A_cm2)
        s.step(300)
        out[(gs, ob)] = s.fields()
    keys = list(out)
    for i in range(len(keys)):
        for j in range(i + 1, len(keys)):
            assert np.abs(out[keys[i]] - out[keys[j]]).max() > 1e-9


def test_forward_stencil_on_every_kernel_mapping(L):
    c = CASES[1][1]()
    ref = None
    for v in (1, 4, 7, 8):
        s = L.Solver.from_case(c, precision="fp64", grad_stencil="forward", step_variant=v)
        s.set_bc(c.x_in, c.current_A_cm2)
        s.step(100)
        X = s.fields()
        ref = X if ref is None else ref
        assert np.abs(X - ref).max() <= 1e-13


def test_extrapolated_outlet_needs_the_per_cell_kernel(L):
    c = CASES[1][1]()
    with pytest.raises(L.LbmsError) as e:
        L.Solver.from_case(c, precision="fp32", outlet_bc="extrapolated", step_variant=1)
    assert e.value.status == L.LBMS_EINVAL
    s = L.Solver.from_case(c, precision="fp32", outlet_bc="extrapolated")
    s.set_bc(c.x_in, c.current_A_cm2)
    assert s.info().threads_per_cell == 1
