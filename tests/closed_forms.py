"""Closed-form results derived from the paper's equations, used to pin the oracle.

Written independently of ``oracle/``: each function states the mathematics
it follows, and the gas data, constants and unit conversions are this
module's own (Table 1 is read from tests/golden/table1_gas_data.txt).
"""
from __future__ import annotations

import math
import os

import numpy as np

R_J_MOL_K = 8.3145     # gas constant, the paper's nomenclature
F_C_MOL = 96485.0      # Faraday constant, Section 4.1 (Eq. 39)
N_ELECTRONS = 2        # Eq. 38
_GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def table1():
    """Molar masses (kg/kmol), Fuller volumes and nu_i of Table 1 / Eq. 38."""
    rows = [l.split() for l in open(os.path.join(_GOLDEN, "table1_gas_data.txt"))
            if l.strip() and not l.startswith("#")]
    return ([float(r[1]) for r in rows], [float(r[2]) for r in rows], [int(r[3]) for r in rows])


def fuller_m2s(T, p_pa, Mi, Mj, Vi, Vj):
    """Eq. 40 as printed: 0.00143 T^1.75 sqrt(1/M_i + 1/M_j) over
    p (V_i^(1/3) + V_j^(1/3))^2, in cm^2/s with p in bar; returned in m^2/s."""
    p_bar = p_pa * 1e-5
    cm2_s = 0.00143 * T ** 1.75 * math.sqrt(1.0 / Mi + 1.0 / Mj) / (p_bar * (Vi ** (1 / 3) + Vj ** (1 / 3)) ** 2)
    return cm2_s / 1e4


def knudsen_m2s(T, M_kg_kmol, d_pore):
    """Eq. 42 in SI: (d_p / 3) sqrt(8 R T / (pi M)), M in kg/mol."""
    return d_pore / 3.0 * math.sqrt(8.0 * R_J_MOL_K * T / (math.pi * M_kg_kmol * 1e-3))


def effective_m2s(Dij, DKi, DKj, eps_over_tau):
    """Eq. 41: (eps/tau)/2 times the sum of the two molecular-Knudsen
    harmonic combinations (DK = inf drops the Knudsen term)."""
    a = 1.0 / (1.0 / Dij + (0.0 if math.isinf(DKi) else 1.0 / DKi))
    b = 1.0 / (1.0 / Dij + (0.0 if math.isinf(DKj) else 1.0 / DKj))
    return 0.5 * eps_over_tau * (a + b)


def gas_point(T, p_pa, d_pore, eps_over_tau):
    """D_ij,eff (3x3, m^2/s, zero diagonal) and C_t = p / RT (Section 4.1)
    from Table 1 and Eqs. 40-42."""
    M, V, _ = table1()
    DK = [knudsen_m2s(T, m, d_pore) if d_pore and d_pore > 0 else math.inf for m in M]
    D = np.zeros((3, 3))
    for i in range(3):
        for j in range(3):
            if i != j:
                D[i, j] = effective_m2s(fuller_m2s(T, p_pa, M[i], M[j], V[i], V[j]), DK[i], DK[j], eps_over_tau)
    return D, p_pa / (R_J_MOL_K * T)


def outlet_flux(I_A_cm2):
    """Eq. 39 with Eq. 38: N = I / (2F) mol/(m^2 s) for H2 (toward the A/E
    interface), -N for H2O, 0 for Ar; I in A/cm^2 (x 1e4 -> A/m^2)."""
    N = I_A_cm2 * 1e4 / (N_ELECTRONS * F_C_MOL)
    return np.array([N, -N, 0.0])


def anode_1d(x, x_in, I_A_cm2, T, p_pa, d_pore, eps_over_tau):
    """Steady 1-D homogeneous anode at positions x (m) from the inlet: the
    ternary profile of ``ternary_1d`` with this module's gas data."""
    D, Ct = gas_point(T, p_pa, d_pore, eps_over_tau)
    N = outlet_flux(I_A_cm2)[0]
    return ternary_1d(x, x_in, N, Ct, D[0, 1], D[0, 2], D[1, 2])


def ternary_1d(x, x_in, N, C_t, D12, D13, D23):
    """Steady 1-D ternary Maxwell-Stefan profile with Stefan flux.

    Eq. 19 with N_1 = N, N_2 = -N, N_3 = 0 (Eq. 39 fluxes of Eq. 38) and
    Gamma = I gives, for the inert species, dX_3/dx = a X_3 with
    a = (N/C_t)(1/D13 - 1/D23), and for H2
    dX_1/dx = -(N/C_t)[(1 - X_3)/D12 + X_3/D13]; X_2 = 1 - X_1 - X_3.
    """
    x = np.asarray(x, dtype=np.float64)
    a = (N / C_t) * (1.0 / D13 - 1.0 / D23)
    x3 = x_in[2] * np.exp(a * x)
    integ = x_in[2] * np.expm1(a * x) / a if a != 0 else x_in[2] * x
    x1 = x_in[0] - (N / C_t) * (x / D12 + (1.0 / D13 - 1.0 / D12) * integ)
    x2 = 1.0 - x1 - x3
    return np.stack([x1, x2, x3])


def binary_linear(j, x1_in, q, D12):
    """Binary limit (no Ar): Fick's law with constant D12 gives the exact
    linear lattice profile X_1(j) = X_1,in - q j / D12 (lattice units)."""
    return x1_in - q * np.asarray(j, dtype=np.float64) / D12


def pulse_variance(t, sigma0_sq, tau, cs2=1.0 / 3.0):
    """Variance per axis of a pulse diffusing under BGK streaming with
    f_eq = w X (Eqs. 28-29) and constant tau, started from equilibrium.

    Exact lattice moment recursion: with omega = 1/tau, the second moment
    grows by cs2 + 2(1-omega) G_t per step, G_{t+1} = (1-omega) G_t + cs2,
    G_0 = 0, which sums to
    sigma0^2 + 2 D t - 2 cs2 (1-omega)(1-(1-omega)^t)/omega^2,
    D = cs2 (tau - 1/2) (Eq. 25).
    """
    om = 1.0 / tau
    D = cs2 * (tau - 0.5)
    return sigma0_sq + 2.0 * D * t - 2.0 * cs2 * (1.0 - om) * (1.0 - (1.0 - om) ** t) / om ** 2


def nernst_overpotential(T, x_in, x_out, electrons=N_ELECTRONS, R=R_J_MOL_K, F=F_C_MOL):
    """Eq. 43."""
    return R * T / (electrons * F) * math.log(x_in[0] * x_out[1] / (x_out[0] * x_in[1]))
