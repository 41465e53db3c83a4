"""Closed-form results derived from the paper's equations, used to pin the oracle.

Written independently of ``oracle/``: each function states the mathematics
it follows.
"""
from __future__ import annotations

import math

import numpy as np


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


def nernst_overpotential(T, x_in, x_out, electrons=2, R=8.3145, F=96485.0):
    """Eq. 43."""
    return R * T / (electrons * F) * math.log(x_in[0] * x_out[1] / (x_out[0] * x_in[1]))
