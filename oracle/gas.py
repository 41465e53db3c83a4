"""Gas properties and lattice scaling for the oracle (FP64, plain Python).

TEST INFRASTRUCTURE: only tests/, the smoke check and the CPU-baseline leg of
the benchmark may use this package.  The CUDA solver computes its own
constants and shares nothing with this file.

* Eq. 40  Fuller binary diffusivity, paper form: 0.00143 T^1.75 sqrt(1/M_i +
  1/M_j) / (p_bar (V_i^(1/3) + V_j^(1/3))^2) in cm^2/s, p in bar.
* Eq. 42  Knudsen diffusivity D_iK = d_p/3 sqrt(8 R T / (pi M_i)), SI units.
* Eq. 41  effective binary diffusivity (eps/tau)/2 [1/(1/D_ij + 1/D_iK) +
  1/(1/D_ij + 1/D_jK)], symmetric in i, j.
* Section 4.1  total concentration C_t = p / (R T).
* Eq. 39  outlet molar flux N_i = -nu_i I / (n F).
* Eq. 25 with c_s^2 = 1/3: the time step makes the smallest effective binary
  diffusivity relax with tau = 1, i.e. dt = dx^2 / (6 min_ij D_ij,eff); the
  grid spacing is dx = L / (nx - 1) (inlet node at x = 0, outlet node at L;
  L / nx for a box periodic in x).
"""
from __future__ import annotations

import math

import numpy as np

R_GAS = 8.3145       # J/(mol K), nomenclature
FARADAY = 96485.0    # C/mol, Eq. 39
CS2 = 1.0 / 3.0


def fuller_binary(T, p_pa, M, V):
    """Eq. 40 -> 3x3 matrix in m^2/s (diagonal left at 0)."""
    n = len(M)
    D = np.zeros((n, n))
    p_bar = p_pa / 1.0e5
    for i in range(n):
        for j in range(n):
            if i == j:
                continue
            cm2 = (0.00143 * T ** 1.75 * math.sqrt(1.0 / M[i] + 1.0 / M[j])
                   / (p_bar * (V[i] ** (1.0 / 3.0) + V[j] ** (1.0 / 3.0)) ** 2))
            D[i, j] = cm2 * 1.0e-4
    return D


def knudsen(T, M, pore_diameter):
    """Eq. 42 -> per-species Knudsen diffusivity (inf when disabled)."""
    if pore_diameter is None or pore_diameter <= 0:
        return np.full(len(M), np.inf)
    return np.array([pore_diameter / 3.0 * math.sqrt(8.0 * R_GAS * T / (math.pi * m / 1000.0))
                     for m in M])


def effective_binary(D, DK, eps_over_tau):
    """Eq. 41 -> symmetric effective binary diffusivities (m^2/s)."""
    n = D.shape[0]
    E = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i == j:
                continue
            a = 1.0 / (1.0 / D[i, j] + 1.0 / DK[i])
            b = 1.0 / (1.0 / D[i, j] + 1.0 / DK[j])
            E[i, j] = eps_over_tau / 2.0 * (a + b)
    return E


def total_concentration(T, p_pa):
    return p_pa / (R_GAS * T)


class Scaling:
    """Physical constants of one case and their lattice-unit images."""

    def __init__(self, gas, nx, length_x, current_A_cm2, dt=None, periodic_x=False):
        self.T = gas.T
        self.p = gas.p
        if gas.D_binary is not None:
            D = np.array(gas.D_binary, dtype=np.float64)
        else:
            D = fuller_binary(gas.T, gas.p, gas.molar_mass, gas.fuller_volume)
        self.D_binary = D
        self.D_knudsen = knudsen(gas.T, gas.molar_mass, gas.pore_diameter)
        self.D_eff = effective_binary(D, self.D_knudsen, gas.eps_over_tau)
        self.C_t = total_concentration(gas.T, gas.p)
        # non-periodic: inlet node at 0, outlet node at L; periodic: period L
        self.dx = length_x / nx if periodic_x else length_x / (nx - 1)
        n = self.D_eff.shape[0]
        dmin = min(self.D_eff[i, j] for i in range(n) for j in range(n) if i != j)
        self.dt = dt if dt else CS2 * 0.5 * self.dx ** 2 / dmin
        self.D_lat = self.D_eff * self.dt / self.dx ** 2
        self.electrons = gas.electrons
        self.stoich = np.array(gas.stoich, dtype=np.float64)
        self.set_current(current_A_cm2)

    def set_current(self, current_A_cm2):
        self.current = current_A_cm2
        I = current_A_cm2 * 1.0e4                       # A/m^2
        self.N_out = -self.stoich * I / (self.electrons * FARADAY)   # Eq. 39
        self.q_lat = self.N_out * self.dt / (self.C_t * self.dx)

    def overpotential(self, x_in, x_out):
        """Eq. 43 (species 0 = H2, 1 = H2O)."""
        return (R_GAS * self.T / (self.electrons * FARADAY)
                * math.log(x_in[0] * x_out[1] / (x_out[0] * x_in[1])))
