"""Pins of the CPU oracle against results fixed by the paper and by mathematics.

Each test names the passage or closed form it checks and would fail on a
plausible slip in the oracle (a dropped term, a wrong sign, a swapped index).
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import closed_forms as cf
from closed_forms import binary_linear, nernst_overpotential, pulse_variance, ternary_1d
from oracle import Oracle, d2q9, d3q19, effective_binary, fuller_binary, knudsen
from oracle.gas import R_GAS, total_concentration
from workloads import cases

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------- lattices
def test_d2q9_matches_eq2_eq9():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "d2q9_eq2_eq9.txt"))
            if l.strip() and not l.startswith("#")]
    E, W, opp = d2q9()
    for a, ex, ey, w in rows:
        a = int(a)
        assert tuple(E[a]) == (int(ex), int(ey), 0)
        assert W[a] == pytest.approx(float(Fraction(w)), abs=1e-16)
    for a in range(9):
        assert tuple(E[opp[a]]) == tuple(-E[a])


@pytest.mark.parametrize("make", [d2q9, d3q19])
def test_lattice_isotropy(make):
    """Zeroth, second and fourth moments of an isotropic lattice with
    c_s^2 = 1/3 (the conditions under which Eq. 28 recovers Eq. 18)."""
    E, W, opp = make()
    dim = 2 if len(W) == 9 else 3
    assert W.sum() == pytest.approx(1.0, abs=1e-15)
    for a in range(dim):
        assert (W * E[:, a]).sum() == pytest.approx(0.0, abs=1e-15)
        for b in range(dim):
            m2 = (W * E[:, a] * E[:, b]).sum()
            assert m2 == pytest.approx(1.0 / 3.0 if a == b else 0.0, abs=1e-15)
    for a in range(dim):
        assert (W * E[:, a] ** 4).sum() == pytest.approx(1.0 / 3.0, abs=1e-15)
        for b in range(dim):
            if a != b:
                assert (W * E[:, a] ** 2 * E[:, b] ** 2).sum() == pytest.approx(1.0 / 9.0, abs=1e-15)
    assert len({tuple(e) for e in E}) == len(W)


# ------------------------------------------------------------ gas data
def _table1():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table1_gas_data.txt"))
            if l.strip() and not l.startswith("#")]
    return [float(r[1]) for r in rows], [float(r[2]) for r in rows]


def test_table1_inputs_match_workloads():
    M, V = _table1()
    assert tuple(M) == cases.MOLAR_MASS
    assert tuple(V) == cases.FULLER_VOLUME


def test_fuller_invariants():
    """Eq. 40: symmetric, proportional to T^1.75 / p, and larger for lighter
    pairs at equal volumes."""
    M, V = _table1()
    D1 = fuller_binary(1000.0, 1e5, M, V)
    D2 = fuller_binary(2000.0, 2e5, M, V)
    assert np.allclose(D1, D1.T, rtol=0, atol=0)
    off = ~np.eye(3, dtype=bool)
    assert np.allclose(D2[off] / D1[off], 2.0 ** 1.75 / 2.0, rtol=1e-14)
    D3 = fuller_binary(1000.0, 1e5, [1.0, 4.0, 4.0], [10.0, 10.0, 10.0])
    assert D3[0, 1] > D3[1, 2]
    assert D3[0, 1] / D3[1, 2] == pytest.approx(math.sqrt((1 + 0.25) / 0.5), rel=1e-14)
    # order of magnitude of gas-phase diffusivities at SOFC temperatures
    assert 1e-4 < D1[0, 1] < 1e-2


def test_knudsen_and_effective_invariants():
    """Eq. 42 scales as d_p sqrt(T/M); Eq. 41 is symmetric, tends to
    (eps/tau) D_ij when the pores are wide and to the harmonic mean of the
    molecular and Knudsen terms when both species share D_K."""
    M, V = _table1()
    K1 = knudsen(1000.0, M, 1e-6)
    K2 = knudsen(4000.0, M, 2e-6)
    assert np.allclose(K2 / K1, 2.0 * 2.0, rtol=1e-14)
    assert K1[0] / K1[2] == pytest.approx(math.sqrt(M[2] / M[0]), rel=1e-14)
    assert K1[0] == pytest.approx(1e-6 / 3 * math.sqrt(8 * R_GAS * 1000.0 / (math.pi * 2.016e-3)), rel=1e-14)
    D = fuller_binary(1000.0, 1e5, M, V)
    E = effective_binary(D, K1, 0.5)
    assert np.allclose(E, E.T, rtol=1e-15)
    Einf = effective_binary(D, np.full(3, np.inf), 0.3)
    off = ~np.eye(3, dtype=bool)
    assert np.allclose(Einf[off], 0.3 * D[off], rtol=1e-15)
    Eeq = effective_binary(D, np.full(3, 2e-4), 1.0)
    assert Eeq[0, 1] == pytest.approx(1.0 / (1.0 / D[0, 1] + 1.0 / 2e-4), rel=1e-14)
    assert total_concentration(1000.0, 1e5) == pytest.approx(1e5 / (R_GAS * 1000.0), rel=1e-15)


def test_gas_data_against_independent_closed_form():
    """Eqs. 39-42 and C_t = p/RT of the oracle against closed_forms, which
    computes them with its own constants and unit conversions: a wrong
    Fuller constant, exponent or pressure unit, Knudsen factor, Eq. 41
    weighting or Eq. 39 scale (n, F, the A/cm^2 factor) fails here."""
    for T, p, dp, phi in ((1073.0, 101325.0, 1e-6, 1.0), (1023.15, 1.013e5, 2.6e-6, 0.46 / 4.5),
                          (900.0, 2.0e5, 0.0, 0.3)):
        gas = cases.Gas(T=T, p=p, pore_diameter=dp, eps_over_tau=phi)
        c = cases.open_channel(11, 1, current_A_cm2=0.7, length_x=2e-3, gas=gas)
        sc = Oracle(c).sc
        D, Ct = cf.gas_point(T, p, dp, phi)
        assert np.allclose(sc.D_eff, D, rtol=1e-13, atol=0)
        assert sc.C_t == pytest.approx(Ct, rel=1e-14)
        assert np.allclose(sc.N_out, cf.outlet_flux(0.7), rtol=1e-14, atol=0)
        assert sc.dx == pytest.approx(2e-3 / 10, rel=1e-15)
        assert np.allclose(sc.q_lat, cf.outlet_flux(0.7) * sc.dt / (Ct * sc.dx), rtol=1e-13, atol=0)


def test_hand_derived_gas_data_and_1d_anode():
    """Values worked out by hand from Table 1 and Eqs. 19 and 39-43 at
    1073 K, 1 atm, d_p = 1 um, eps/tau = 1, X_in = (0.5, 0.1, 0.4),
    L = 2 mm (they are not printed in the paper), to the digits given:
    D_eff = 4.326e-4 (H2-H2O), 3.765e-4 (H2-Ar), 1.607e-4 (H2O-Ar) m^2/s,
    C_t = 11.357 mol/m^3; at 0.5 A/cm^2, N = 2.591e-2 mol/(m^2 s), X_out =
    (0.488829, 0.117626, 0.393545), eta = 8.550 mV; at 1.0 A/cm^2, X_out =
    (0.477668, 0.135138, 0.387193), eta = 16.034 mV.  Checked against the
    closed forms and against the oracle's 1-D steady state (nx = 33, second
    order in dx, so a few 1e-6 from the continuum)."""
    D, Ct = cf.gas_point(1073.0, 101325.0, 1e-6, 1.0)
    assert D[0, 1] == pytest.approx(4.326e-4, abs=0.0005e-4)
    assert D[0, 2] == pytest.approx(3.765e-4, abs=0.0005e-4)
    assert D[1, 2] == pytest.approx(1.607e-4, abs=0.0005e-4)
    assert Ct == pytest.approx(11.357, abs=0.0005)
    assert cf.outlet_flux(0.5)[0] == pytest.approx(2.591e-2, abs=0.0005e-2)
    want = {0.5: ((0.488829, 0.117626, 0.393545), 8.550e-3), 1.0: ((0.477668, 0.135138, 0.387193), 16.034e-3)}
    for I, (xo, eta) in want.items():
        X = cf.anode_1d(np.array([2e-3]), (0.5, 0.1, 0.4), I, 1073.0, 101325.0, 1e-6, 1.0)[:, -1]
        assert np.allclose(X, xo, atol=0.5e-6)
        assert nernst_overpotential(1073.0, (0.5, 0.1, 0.4), X) == pytest.approx(eta, abs=0.0005e-3)
        o, _ = _run_1d(33, 2e-3, I, tol=1e-13)
        assert np.allclose(o.outlet_mean(), xo, atol=5e-6)
        assert o.overpotential() == pytest.approx(eta, rel=2e-4)


def test_table2_closed_form_eta_minus_eta0():
    """The homogenised Table 2 anode (1023.15 K, 1.013e5 Pa, eps/tau =
    0.46/4.5, d_p = 2.6 um, L = 2 mm, H2:H2O = 4:1 diluted by Ar; eta_0 at
    X_H2 = 0.8): eta - eta_0 (V) worked out by hand from Eqs. 19 and 39-43,
    to four decimals.  Rows 0.3, 0.7, 1.0 A/cm^2 (Figs. 2-4); columns
    X_H2,in = 0.6, 0.4, 0.3, 0.2."""
    table = {0.3: (0.0073, 0.0197, 0.0302, 0.0475),
             0.7: (0.0135, 0.0348, 0.0522, 0.0827),
             1.0: (0.0170, 0.0434, 0.0659, 0.1124)}
    g = cases.PAPER_TABLE2

    def eta(I, xh):
        x_in = (xh, xh / 4.0, 1.0 - 1.25 * xh)
        X = cf.anode_1d(np.array([2e-3]), x_in, I, g.T, g.p, g.pore_diameter, g.eps_over_tau)[:, -1]
        return nernst_overpotential(g.T, x_in, X)

    for I, row in table.items():
        e0 = eta(I, 0.8)
        for xh, v in zip((0.6, 0.4, 0.3, 0.2), row):
            assert eta(I, xh) - e0 == pytest.approx(v, abs=0.5e-4), (I, xh)


def test_eq24_tau_at_unequal_diffusivities():
    """Eq. 24 evaluated with the fluxes of the 1-D steady state, N_1 = -N_2 =
    I/2F and N_3 = 0 (Eq. 39, Section 3.1), at strongly unequal D_ij:
    1/D_1 = (X_1 + X_2)/D_12 + X_3/D_13 and 1/D_2 = (X_1 + X_2)/D_12 +
    X_3/D_23, so tau_i = D_i/c_s^2 + 1/2 (Eq. 25) in lattice units.  For Ar
    (N_3 = 0) Eq. 24 is singular and the mixture value
    (X_1 + X_2)/(X_1/D_13 + X_2/D_23) is taken.  An index or sign slip in
    the oracle's Eq. 24 coefficients moves tau_1 or tau_2 off these values."""
    Db = np.array([[0.0, 6e-4, 3e-4], [6e-4, 0.0, 1.5e-4], [3e-4, 1.5e-4, 0.0]])
    gas = cases.Gas(D_binary=Db, pore_diameter=0.0, eps_over_tau=1.0)
    c = cases.open_channel(17, 1, current_A_cm2=1.5, length_x=4e-3, gas=gas)
    o = Oracle(c)
    _, Ct = cf.gas_point(gas.T, gas.p, 0.0, 1.0)
    N = cf.outlet_flux(1.5)
    x = np.arange(17) * (4e-3 / 16)
    o.init(ternary_1d(x, c.x_in, N[0], Ct, Db[0, 1], Db[0, 2], Db[1, 2])[:, None, None, :])
    n, r = o.run_to_residual(1e-13, 400000, 100)
    assert r <= 1e-13
    X1, X2, X3 = (o.X[i, 0, 0] for i in range(3))
    lat = o.sc.dt / o.sc.dx ** 2           # m^2/s -> lattice units
    D = {}
    for i, (k, l) in ((0, (1, 2)), (1, (0, 2))):
        # 1/D_i = sum_j X_j / D_ij - X_i N_j / (D_ij N_i), j != i
        inv = sum(o.X[j, 0, 0] / Db[i, j] - o.X[i, 0, 0] * N[j] / (Db[i, j] * N[i]) for j in (k, l))
        D[i] = 1.0 / inv
    assert np.allclose(1.0 / D[0], (X1 + X2) / Db[0, 1] + X3 / Db[0, 2], rtol=1e-14)
    D[2] = (X1 + X2) / (X1 / Db[0, 2] + X2 / Db[1, 2])
    for i in range(3):
        tau = 3.0 * D[i] * lat + 0.5
        assert np.all((tau > 1.0) & (tau < 5.0)), i        # the clamp of Eq. 25 is inactive
        assert np.allclose(o.tau[i, 0, 0], tau, rtol=1e-12, atol=0), i
    assert np.abs(o.tau[0] - o.tau[1]).max() > 0.1           # the D_ij really differ


@pytest.mark.parametrize("kind", ["1d", "porous"])
def test_lagged_gradient_reaches_the_paper_order_steady_state(kind):
    """Section 3.2 computes Eq. 35 on the moments of the current step; the
    fused kernel (and the default oracle) can only use the previous step's
    field.  At steady state X no longer changes, so both orders must reach
    the same state."""
    if kind == "1d":
        c = cases.open_channel(17, 1, current_A_cm2=1.0, length_x=1e-2)
    else:
        c = cases.porous((12, 20), radius=2, porosity=0.6, seed=7, current_A_cm2=1.0)
    res = []
    for lag in (True, False):
        o = Oracle(c, lag=lag)
        n, r = o.run_to_residual(1e-13, 400000, 100)
        assert r <= 1e-13
        res.append(o.X.copy())
    assert np.abs(res[0] - res[1]).max() < 1e-10
    # and the two orders do differ on the way there
    a, b = Oracle(c, lag=True), Oracle(c, lag=False)
    a.step(50)
    b.step(50)
    assert np.abs(a.X - b.X).max() > 1e-8


@pytest.mark.slow
def test_eq21_closure_drifts():
    """Section 3.2 takes Ar's flux from Eq. 21, N_3 = -(N_1 + N_2).  With that
    closure nothing restores sum_i X_i = 1: on the 1-D anode the residual
    stalls near 1e-8, sum X - 1 keeps growing and Ar carries a net flux.
    With Ar's own row of Eq. 19 (the reading used) the same run converges
    to rounding, sum X - 1 settles at its O(dx^2) value and Ar's net flux
    vanishes."""
    out = {}
    for closure in ("row_n", "eq21"):
        c = cases.open_channel(17, 1, current_A_cm2=1.0, length_x=1e-2)
        o = Oracle(c, closure=closure)
        o.step(20000)
        o.residual(1)
        o.step(5000)
        r1 = o.residual(5000)
        s1 = np.abs(o.X.sum(axis=0) - 1.0).max()
        o.step(5000)
        r2 = o.residual(5000)
        s2 = np.abs(o.X.sum(axis=0) - 1.0).max()
        far = np.abs(o.plane_flux()[2]).max() / abs(o.sc.q_lat[0])
        out[closure] = (r1, r2, s1, s2, far)
    r1, r2, s1, s2, far = out["row_n"]
    assert r2 < 1e-13 and abs(s2 - s1) < 1e-12 and s2 < 1e-5 and far < 1e-9
    r1, r2, s1, s2, far = out["eq21"]
    assert r2 > 5e-9 and r2 > 0.5 * r1         # stalled
    assert s2 > s1 + 1e-5                      # sum X - 1 still growing
    assert far > 1e-5


# ------------------------------------------------------------- P4: I = 0
def test_zero_current_keeps_inlet_state():
    c = cases.porous((16, 24), radius=3, porosity=0.6, seed=5, current_A_cm2=0.0)
    o = Oracle(c)
    o.step(60)
    f = ~c.solid
    for i in range(3):
        assert np.abs(o.X[i][f] - c.x_in[i]).max() < 1e-15
    assert o.overpotential() == pytest.approx(0.0, abs=1e-15)


# ---------------------------------------- P1: 1-D ternary closed form
def _closed_form_1d(c):
    """The closed-form profile at the nodes x_j = j L / (nx - 1) of a 1-D
    case, with gas data computed by closed_forms (not by the oracle)."""
    g = c.gas
    nx = c.solid.shape[2]
    x = np.arange(nx) * (c.length_x / (nx - 1))
    return cf.anode_1d(x, c.x_in, c.current_A_cm2, g.T, g.p, g.pore_diameter, g.eps_over_tau)


def _run_1d(nx, L, current, x_in=(0.5, 0.1, 0.4), gas=None, tol=1e-13, **okw):
    c = cases.open_channel(nx, 1, current_A_cm2=current, length_x=L, x_in=x_in,
                           gas=gas or cases.Gas())
    o = Oracle(c, **okw)
    Xc = _closed_form_1d(c)
    o.init(Xc[:, None, None, :])
    n, r = o.run_to_residual(tol, 400000, 100)
    assert r <= tol
    return o, Xc


def test_ternary_1d_closed_form_second_order():
    """Eqs. 19, 24, 25, 28, 32-36, 39: the homogeneous 1-D anode converges to
    the ternary Maxwell-Stefan profile with Stefan flux at second order; the
    component velocities of Eq. 20 (from the fluxes of Eqs. 31-34) approach
    u_i = N_i / (C_t X_i) with the outlet fluxes of Eq. 39 (N_Ar = 0)."""
    errs, sums, uerr = [], [], []
    for nx in (9, 17, 33):
        o, Xc = _run_1d(nx, 1e-2, 1.0)
        X = o.X[:, 0, 0, :]
        k = (nx - 1) // 8
        errs.append(np.abs(X - Xc)[:, ::k].max())
        sums.append(np.abs(X.sum(axis=0) - 1.0).max())
        u = o.fields()[1][:, 0, 0, 0, 1:-1]             # x components, interior nodes
        want = o.sc.N_out[:2, None] / (o.sc.C_t * X[:2, 1:-1])
        uerr.append(max(np.abs(u[:2] / want - 1.0).max(), np.abs(u[2]).max() / np.abs(u[0]).max()))
        # inert species: zero net flux through every plane (Eq. 39, nu_3 = 0)
        F = o.plane_flux()
        assert np.abs(F[2]).max() < 1e-9 * abs(o.sc.q_lat[0])
        assert np.allclose(F[0], o.sc.q_lat[0], rtol=1e-9)
        assert np.allclose(F[1], o.sc.q_lat[1], rtol=1e-9)
    assert errs[-1] < 1e-6
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5
    assert sums[0] / sums[1] > 3.5 and sums[1] / sums[2] > 3.5
    assert uerr[-1] < 2e-4 and uerr[0] / uerr[1] > 1.7 and uerr[1] / uerr[2] > 1.7


def test_overpotential_matches_closed_form_and_table2_trend():
    """Eq. 43 on the homogenised Table 2 anode (eps/tau = 0.46/4.5,
    d_p = 2.6 um, 2 mm, H2:H2O = 4:1 diluted by Ar, Section 4.2): the LBM
    eta - eta_0 agrees with the closed-form profile, and grows as H2 is
    diluted (Figs. 2-4 trend)."""
    gas = cases.PAPER_TABLE2
    res = {}
    for xh in (0.8, 0.6, 0.3):
        x_in = (xh, xh / 4.0, 1.0 - 1.25 * xh)
        o, Xc = _run_1d(13, 2e-3, 1.0, x_in=x_in, gas=gas, tol=1e-12)
        eta = o.overpotential()
        eta_cf = nernst_overpotential(gas.T, x_in, Xc[:, -1])
        res[xh] = (eta, eta_cf)
        assert eta == pytest.approx(eta_cf, rel=2e-4)
    d06 = res[0.6][0] - res[0.8][0]
    d03 = res[0.3][0] - res[0.8][0]
    assert 0 < d06 < d03
    assert d03 == pytest.approx(res[0.3][1] - res[0.8][1], rel=2e-4)


# ------------------------------------------------ P2: exact binary limit
def test_binary_limit_is_exact_linear():
    """No Ar: Eq. 32 reduces to Fick with D12; the D2Q9 steady state is the
    exact linear profile with the Eq. 39 slope (wet-node Eq. 36 inlet)."""
    x_in = (0.7, 0.3, 0.0)
    c = cases.open_channel(12, 1, current_A_cm2=1.0, length_x=2e-3, x_in=x_in)
    o = Oracle(c)
    n, r = o.run_to_residual(1e-14, 200000, 100)
    j = np.arange(12)
    X1 = binary_linear(j, 0.7, o.sc.q_lat[0], o.sc.D_lat[0, 1])
    assert np.abs(o.X[0, 0, 0] - X1).max() < 1e-11
    assert np.abs(o.X[1, 0, 0] - (1.0 - X1)).max() < 1e-11
    assert np.all(o.X[2] == 0.0)


# -------------------------------------- P3: exact pulse variance law
@pytest.mark.parametrize("dim,axis", [(2, 0), (2, 1), (3, 0), (3, 1), (3, 2)])
def test_pulse_variance_exact(dim, axis):
    """Equal binary diffusivities: Eq. 32 gives B = I/D, every species
    relaxes with tau = D/c_s^2 + 1/2 (Eq. 25) and the pulse variance follows
    the exact lattice law (closed_forms.pulse_variance)."""
    n = 600
    shape = [1, 1, 1]
    shape[2 - axis] = n
    D = 2e-4
    gas = cases.Gas(D_binary=np.full((3, 3), D), pore_diameter=0.0, eps_over_tau=1.0)
    c = cases.Case(name="pulse", solid=np.zeros(shape, bool), dim=dim,
                   periodic_x=True, gas=gas, length_x=1e-3 * shape[2])
    o = Oracle(c)
    dt = 3.0 * o.sc.dt                      # D* = 1/2, tau = 2
    o = Oracle(c, dt=dt)
    assert o.sc.D_lat[0, 1] == pytest.approx(0.5, rel=1e-14)
    X0 = cases.gaussian_pulse(tuple(shape), axis, sigma0=3.0, amplitude=0.05)
    o.init(X0)
    steps = 1000
    o.step(steps)
    assert np.allclose(o.tau[0], 2.0, rtol=1e-12)
    pulse = (o.X[0] - 0.3).reshape(-1)
    s = np.arange(n) - (n - 1) / 2.0
    m0 = pulse.sum()
    var = (s * s * pulse).sum() / m0
    assert m0 == pytest.approx((X0[0] - 0.3).sum(), rel=1e-9)
    assert var == pytest.approx(pulse_variance(steps, 9.0, 2.0), rel=1e-9)


# ----------------------------------------------- P5: closed-box balance
@pytest.mark.parametrize("shape", [(24, 32), (10, 12, 16)])
def test_closed_box_conserves_each_species(shape):
    """Bounce-back on the mask (Section 3.3) and periodic sides: Eq. 28 with
    Eq. 29 conserves every species exactly."""
    c = cases.porous(shape, radius=3, porosity=0.55, seed=11)
    c = c.with_(periodic_x=True)
    o = Oracle(c)
    rng = np.random.Generator(np.random.PCG64(3))
    X = np.empty((3,) + c.solid.shape)
    X[0] = 0.4 + 0.05 * rng.random(c.solid.shape)
    X[2] = 0.3 + 0.05 * rng.random(c.solid.shape)
    X[1] = 1.0 - X[0] - X[2]
    o.init(X)
    tot0 = o.total()
    o.step(200)
    assert np.allclose(o.total(), tot0, rtol=1e-13)


# ---------------------------------------------- P6: steady flux balance
def test_porous_steady_flux_balance():
    """Section 4.2: at steady state the flux through every x-plane equals the
    Eq. 39 outlet flux (H2 in, H2O out), Ar carries none."""
    c = cases.porous((12, 20), radius=2, porosity=0.6, seed=7, current_A_cm2=1.0)
    o = Oracle(c)
    n, r = o.run_to_residual(1e-12, 300000, 100)
    assert r <= 1e-12
    F = o.plane_flux()
    n_out = c.solid.shape[0] * c.solid.shape[1]
    q = o.sc.q_lat
    assert np.allclose(F[0], q[0] * n_out, rtol=1e-7)
    assert np.allclose(F[1], q[1] * n_out, rtol=1e-7)
    assert np.abs(F[2]).max() < 1e-7 * abs(q[0]) * n_out


# ---------------------------------- P8: D2Q9 and D3Q19 on 1-D states
def test_d2q9_d3q19_agree_on_1d_states():
    """Both lattices project onto the same 1-D three-velocity lattice
    (weights 2/3, 1/6, 1/6), so x-only states evolve identically."""
    x_in = (0.5, 0.1, 0.4)
    c2 = cases.open_channel(20, 1, current_A_cm2=2.0, x_in=x_in)
    c3 = c2.with_(dim=3)
    o2, o3 = Oracle(c2), Oracle(c3)
    prof = np.linspace(0, 1, 20)
    X = np.empty((3, 1, 1, 20))
    X[0, 0, 0] = 0.5 - 0.1 * prof ** 2
    X[2, 0, 0] = 0.4 + 0.03 * prof
    X[1] = 1.0 - X[0] - X[2]
    o2.init(X)
    o3.init(X)
    for _ in range(5):
        o2.step(40)
        o3.step(40)
        assert np.abs(o2.X - o3.X).max() < 1e-14
        assert np.abs(o2.tau - o3.tau).max() < 1e-12


# --------------------------------------------------- P9: mirror symmetry
def test_mirror_symmetry_2d():
    c = cases.porous((16, 24), radius=3, porosity=0.55, seed=9, current_A_cm2=1.0)
    cm = c.with_(solid=c.solid[:, ::-1, :].copy())
    o, om = Oracle(c), Oracle(cm)
    o.step(150)
    om.step(150)
    assert np.abs(o.X - om.X[:, :, ::-1, :]).max() < 1e-13


def test_mirror_and_transpose_symmetry_3d():
    c = cases.porous((8, 8, 12), radius=2, porosity=0.6, seed=4, current_A_cm2=1.0)
    variants = [
        (c.solid[::-1, :, :], lambda X: X[:, ::-1, :, :]),
        (c.solid[:, ::-1, :], lambda X: X[:, :, ::-1, :]),
        (np.swapaxes(c.solid, 0, 1), lambda X: np.swapaxes(X, 1, 2)),
    ]
    o = Oracle(c)
    o.step(80)
    for solid, back in variants:
        om = Oracle(c.with_(solid=np.ascontiguousarray(solid)))
        om.step(80)
        assert np.abs(o.X - back(om.X)).max() < 1e-13


# ------------------------- the literal readings of Eqs. 35 and 37 (options)
def _order_1d(grad_stencil, outlet_bc):
    errs, flux = [], []
    for nx in (9, 17, 33):
        c = cases.open_channel(nx, 1, current_A_cm2=1.0, length_x=2e-3)
        o = Oracle(c, grad_stencil=grad_stencil, outlet_bc=outlet_bc)
        sc = o.sc
        Xc = _closed_form_1d(c)
        o.init(Xc[:, None, None, :])
        n, r = o.run_to_residual(1e-12, 400000, 100)
        assert r <= 1e-12
        k = (nx - 1) // 8
        errs.append(np.abs(o.X[:, 0, 0, :] - Xc)[:, ::k].max())
        flux.append(np.abs(o.plane_flux()[0] / sc.q_lat[0] - 1.0).max())
    return np.array(errs), np.array(flux)


@pytest.mark.slow
def test_forward_gradient_stencil_is_first_order():
    """Eq. 35 as printed (forward difference, x only): the 1-D anode still
    converges to the closed form, at first order, and the flux condition
    (Eq. 39) still holds exactly."""
    errs, flux = _order_1d("forward", "flux")
    ratios = errs[:-1] / errs[1:]
    assert np.all((ratios > 1.7) & (ratios < 2.3))
    assert flux.max() < 1e-8


@pytest.mark.slow
def test_extrapolated_outlet_is_first_order():
    """Eq. 37 read as a wet node: first-order convergence to the closed form,
    and the delivered outlet flux approaches Eq. 39's as dx halves."""
    errs, flux = _order_1d("central", "extrapolated")
    ratios = errs[:-1] / errs[1:]
    assert np.all((ratios > 1.7) & (ratios < 2.3))
    fr = flux[:-1] / flux[1:]
    assert np.all((fr > 1.7) & (fr < 2.3))
    assert flux[-1] < 1e-4
