// Host-side gas properties and lattice scaling of the solver (FP64).
//
//  Eq. 40  Fuller binary diffusivity as printed: 0.00143 T^1.75
//          sqrt(1/M_i + 1/M_j) / (p[bar] (V_i^1/3 + V_j^1/3)^2) cm^2/s
//  Eq. 42  Knudsen diffusivity D_iK = d_p/3 sqrt(8 R T / (pi M_i))
//  Eq. 41  D_ij,eff = (eps/tau)/2 [ (1/D_ij + 1/D_iK)^-1 + (1/D_ij + 1/D_jK)^-1 ]
//  Sec 4.1 C_t = p / (R T);  Eq. 39 N_i = -nu_i I / (n F)
//  Eq. 25  with c_s^2 = 1/3, the default time step relaxes the smallest
//          D_ij,eff with tau = 1: dt = dx^2 / (6 min D_ij,eff)
#pragma once

#include <cmath>

namespace lbms {

constexpr double kR = 8.3145;      // J/(mol K)
constexpr double kF = 96485.0;     // C/mol
constexpr double kPi = 3.14159265358979323846;

struct GasProps {
    double D_bin[3][3];   // m^2/s (Eq. 40 or user)
    double D_kn[3];       // m^2/s (Eq. 42), +inf when disabled
    double D_eff[3][3];   // m^2/s (Eq. 41)
    double C_t;           // mol/m^3
    double dx, dt;        // m, s
    double D_lat[3][3];   // D_eff dt / dx^2
    double T, p;
    int electrons;
    double stoich[3];
};

inline double fuller_cm2s(double T, double p_pa, double Mi, double Mj, double Vi, double Vj) {
    const double s = std::cbrt(Vi) + std::cbrt(Vj);
    return 0.00143 * std::pow(T, 1.75) * std::sqrt(1.0 / Mi + 1.0 / Mj) / ((p_pa * 1.0e-5) * s * s);
}

inline double knudsen_m2s(double T, double M_kg_kmol, double dp) {
    return dp / 3.0 * std::sqrt(8.0 * kR * T / (kPi * M_kg_kmol * 1.0e-3));
}

// Outlet flux per node per step in mole-fraction units (lattice image of Eq. 39).
inline void outlet_flux_lattice(const GasProps& g, double current_A_cm2, double q[3]) {
    const double I = current_A_cm2 * 1.0e4;
    for (int s = 0; s < 3; ++s) {
        const double N = -g.stoich[s] * I / (g.electrons * kF);
        q[s] = N * g.dt / (g.C_t * g.dx);
    }
}

}  // namespace lbms
