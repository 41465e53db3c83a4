"""Residual parity (the K-step relative L2 change that decides when every run
stops; the paper defines none, so both sides take the same definition:
r = max_i ||X_i(t) - X_i(t-K)||_2 / (K ||X_i(t)||_2) over fluid cells, FP64).

Three checks, through the C ABI:

* the reduction itself: the GPU residual of a state equals Oracle.residual(K)
  evaluated on that same state (the GPU's X fields at the snapshot and at t,
  handed to the oracle), to 1e-12 relative, for FP64, FP32 and FP16 storage,
  single handles and batches, 2-D and 3-D porous anodes, several K;
* the trajectory: GPU FP64 and the oracle each evolve from the same start and
  their residuals agree within the bound that the X parity (1e-11 absolute
  per cell) implies;
* the stopping decision: per-case step counts of the batched run_to_residual
  equal the oracle's run_to_residual on each case alone.
"""
import numpy as np
import pytest

from oracle import Oracle
from workloads import cases

pytestmark = pytest.mark.gpu

X_TOL_FP64 = 1e-11     # per-cell |X_gpu - X_oracle| after a few thousand FP64 steps


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_01600_gb300 import lbms
    lbms.load()
    return lbms


def _oracle_residual_of(case, X_now, X_snap, K):
    """Oracle.residual(K) evaluated on a given state (dense [3, z, y, x])."""
    o = Oracle(case)
    o.X = np.where(o.fluid, X_now, 0.0)
    o.snap = np.where(o.fluid, X_snap, 0.0)
    return o.residual(K)


CASES = [
    ("porous2d_48x40", lambda: cases.porous((40, 48), radius=3, porosity=0.55, seed=61, current_A_cm2=1.5)),
    ("porous3d_24x16x12", lambda: cases.porous((12, 16, 24), radius=2, porosity=0.5, seed=62, current_A_cm2=1.0)),
]


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_residual_reduction_matches_oracle_on_same_state(L, name, make, precision):
    case = make()
    s = L.Solver.from_case(case, precision=precision)
    s.set_bc(case.x_in, case.current_A_cm2)
    s.step(40)
    s.residual(40)                      # the snapshot is now X(40)
    snap = s.fields()
    for K in (1, 7, 100, 333):
        s.step(K)
        now = s.fields()
        r = s.residual(K)
        ro = _oracle_residual_of(case, now, snap, K)
        assert ro > 0
        assert r == pytest.approx(ro, rel=1e-12), f"K={K}: gpu {r:.17e} oracle {ro:.17e}"
        snap = now
    s.close()


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_residual_trajectory_fp64(L, name, make):
    case = make()
    s = L.Solver.from_case(case, precision="fp64")
    s.set_bc(case.x_in, case.current_A_cm2)
    o = Oracle(case)
    nf = case.n_fluid
    for K in (1, 10, 100, 250):
        s.step(K)
        o.step(K)
        r = s.residual(K)
        ro = o.residual(K)
        # |dr| <= ||dX_now - dX_snap||_2 / (K ||X||_2) with |dX| <= X_TOL_FP64 per cell
        xn = min(np.sqrt((o.X[i] ** 2).sum()) for i in range(3))
        bound = 2.0 * X_TOL_FP64 * np.sqrt(nf) / (K * xn) + 1e-12 * ro
        assert abs(r - ro) <= bound, f"K={K}: gpu {r:.6e} oracle {ro:.6e} bound {bound:.2e}"
    s.close()


def _batch_cases():
    return [cases.porous((20, 28), radius=2, porosity=0.6, seed=71, current_A_cm2=0.5),
            cases.porous((16, 36), radius=3, porosity=0.55, seed=72, current_A_cm2=1.5, x_in=(0.3, 0.075, 0.625)),
            cases.open_channel(24, 6, current_A_cm2=1.0)]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_residuals_match_oracle_on_same_state(L, precision):
    cs = _batch_cases()
    b = L.Batch.from_cases(cs, precision=precision)
    for k, c in enumerate(cs):
        b.set_bc(c.x_in, c.current_A_cm2, case=k)
    b.step(25)
    b.residuals(25)
    snaps = [b.fields(k) for k in range(len(cs))]
    for K in (3, 64):
        b.step(K)
        now = [b.fields(k) for k in range(len(cs))]
        r = b.residuals(K)
        for k, c in enumerate(cs):
            ro = _oracle_residual_of(c, now[k], snaps[k], K)
            assert r[k] == pytest.approx(ro, rel=1e-12), f"case {k}, K={K}"
        snaps = now
    b.close()


def test_batch_stop_steps_match_oracle(L):
    """The per-case stopping step of the batched run equals the oracle's
    run_to_residual on each case alone (checks every K = 100 steps)."""
    cs = _batch_cases()
    tol = 5e-6
    b = L.Batch.from_cases(cs, precision="fp64")
    for k, c in enumerate(cs):
        b.set_bc(c.x_in, c.current_A_cm2, case=k)
    n, steps, r, st = b.run_to_residual(tol, 200000)
    assert st == L.LBMS_OK
    for k, c in enumerate(cs):
        o = Oracle(c)
        no, ro = o.run_to_residual(tol, 200000, 100)
        assert ro <= tol
        assert steps[k] == no, f"case {k}: gpu stops at {steps[k]}, oracle at {no}"
    assert n == max(steps)
    b.close()
