"""Plain FP64 CPU oracle of the advection-diffusion LBM coupled to the
Maxwell-Stefan equations (ternary H2-H2O-Ar).  TEST INFRASTRUCTURE.

Dense arrays over the whole box, indexed ``[species, direction, z, y, x]``;
two lattices (pull streaming); every step is written out in the order of the
method, vectorised over cells with numpy and nothing else.

One time step t (all quantities in lattice units, c_s^2 = 1/3):

1. Stream (Eq. 28 left-hand side, pull form): f_a(x) = f*_a(x - e_a) from the
   stored post-collision lattice.  A solid source gives half-way bounce-back
   f_a(x) = f*_abar(x) (Section 3.3, solid boundaries).
   Inlet x = 0, for e_ax = +1 (Eq. 36, read as the anti-bounce-back rule for
   every incoming link): f_a = (w_a + w_abar) X_in - f_abar, with f_abar the
   value just streamed into the same node.
   Outlet x = nx-1, for e_ax = -1 (Eq. 39 flux imposed link-wise):
   f_a = f*_abar - (w_abar / W) q, W = sum of w over e_x = +1 links, q the
   lattice image of N_i = -nu_i I/(nF); this removes exactly q per node per
   step (zero for Ar).  outlet_bc="extrapolated" instead reads Eq. 37 as a
   wet node: X_out = X^{t-1}(nx-2) + dX with dX from Eq. 19 over one
   spacing at the outlet fluxes, dX_i = sum_j (X_i q_j - X_j q_i) / D_ij
   (X at nx-2, or at the node itself where nx-2 is solid), applied with the
   Eq. 36 rule f_a = (w_a + w_abar) X_out - f_abar.
2. Moments: X_i = sum_a f_a (the zeroth moment of Eq. 29's distribution).
3. Gradient of the stored field of the previous step (Eq. 35, read as a
   central difference on every axis; a fused one-pass step can only see its
   neighbours' X of the step before).  lag=False follows the order of
   Section 3.2 instead: the gradient of the moments of step 2 of this very
   step, after every cell has taken them.  Either way the steady state is
   the same (X then no longer changes from step to step).  The stencil:
   (X(x+e) - X(x-e))/2; a solid neighbour takes the centre value (mirror
   about the half-way wall); at the x = 0 / x = nx-1 nodes the one-sided
   difference is used.
   grad_stencil="forward" takes Eq. 35 literally: X(x+1) - X(x) along x
   only (backward at x = nx-1), zero along y and z.
4. Maxwell-Stefan coupling with species 3 (Ar) as the reference n:
   B from Eq. 32, J = -B^-1 grad X per axis (Eqs. 31, 33, 34 with
   Gamma = I, Eq. 30 ideal gas); J_3 from the n-th row of Eq. 19 given
   J_1, J_2 (not from the closure of Eq. 21, which leaves sum X - 1 without
   a restoring term); N = J (Eq. 20, u_M = 0, Section 3.1).
   closure="eq21" takes Section 3.2 literally instead: J_3 = -J_1 - J_2.
5. Effective diffusivity, Eq. 24, with the paper's rule that each flux
   points as its stoichiometric coefficient says (Section 3.1) and its
   observation that the fluxes across the thin anode stay at their A/E values
   (Sections 4.1-4.2), so that N_j / N_i = nu_j / nu_i:
   1/D_i = sum_{j!=i} (X_j - X_i nu_j/nu_i) / D_ij.  For the inert species
   (nu_i = 0) Eq. 24 is singular and D_i is the mixture value
   sum_{j!=i} X_j / sum_{j!=i} X_j/D_ij.
6. Relaxation time, Eq. 25: tau_i = D_i / c_s^2 + 1/2, clamped to
   [tau_min, tau_max]; tau_min = 1 keeps omega <= 1 (Section 2.3 (2b)).
   The part of the Maxwell-Stefan flux of step 4 that the relaxation alone
   does not carry goes into a velocity in the slot of Eq. 26:
   v_i = (N_i + D_i^tau g_i) X_i / (X_i^2 + eps_x^2), |v_i| <= v_max,
   D_i^tau = c_s^2 (tau_i - 1/2).  For the reacting species of the 1-D anode
   at steady state v_i vanishes and the step is Eqs. 28-29 exactly; the inert
   species keeps the drift that carries its Stefan drag.
7. Collide (Eq. 28 with Eq. 29 / Eq. 26 equilibrium):
   f*_a = f_a - (f_a - w_a X_i (1 + e_a . v_i / c_s^2)) / tau_i.
8. The moments of step 2 become the stored field used by the next gradient.

Residual (the paper defines none): every K steps
r = max_i ||X_i(t) - X_i(t-K)||_2 / (K ||X_i(t)||_2) over fluid cells.
Overpotential: Eq. 43 with X_out the mean over the outlet column.
"""
from __future__ import annotations

import numpy as np

from . import lattice as _lattice
from .gas import CS2, Scaling

D_BIG = 1.0e30        # stands for an unbounded D_i (tau then sits at tau_max)
EPS_X = 1.0e-12       # guard of 1/X_i
MIX_DELTA = 1.0e-12   # guard of the mixture average when the others vanish
V_MAX = 0.1           # bound on |v_i| (lattice units)


class Oracle:
    def __init__(self, case, tau_min=1.0, tau_max=5.0, coupling="ms", dt=None,
                 grad_stencil="central", outlet_bc="flux", lag=True, closure="row_n"):
        self.case = case
        self.solid = np.asarray(case.solid, dtype=bool)
        self.fluid = ~self.solid
        self.dim = case.dim
        self.nz, self.ny, self.nx = self.solid.shape
        self.E, self.W, self.opp = _lattice.for_dim(case.dim)
        self.Q = len(self.W)
        self.periodic_x = bool(case.periodic_x)
        if not self.periodic_x and (self.solid[:, :, 0].any() or self.solid[:, :, -1].any()):
            raise ValueError("inlet/outlet columns must be fluid")
        self.sc = Scaling(case.gas, self.nx, case.length_x, case.current_A_cm2, dt,
                          periodic_x=self.periodic_x)
        self.x_in = np.array(case.x_in, dtype=np.float64)
        self.tau_min = tau_min
        self.tau_max = tau_max
        self.coupling = coupling
        if grad_stencil not in ("central", "forward") or outlet_bc not in ("flux", "extrapolated"):
            raise ValueError("grad_stencil: central | forward; outlet_bc: flux | extrapolated")
        if closure not in ("row_n", "eq21"):
            raise ValueError("closure: row_n | eq21")
        self.grad_stencil = grad_stencil
        self.outlet_bc = outlet_bc
        self.lag = bool(lag)
        self.closure = closure
        self.t = 0
        self.init()

    # ------------------------------------------------------------------ state
    def _w(self):
        return self.W.reshape(1, self.Q, 1, 1, 1)

    def init(self, X=None):
        """f = w_a X (Eq. 29 equilibrium); X defaults to the inlet values."""
        if X is None:
            X = self.x_in
        X = np.asarray(X, dtype=np.float64)
        if X.ndim == 1:
            X = X.reshape(3, 1, 1, 1) * np.ones((1,) + self.solid.shape)
        X = np.where(self.fluid, X, 0.0)
        self.A = self._w() * X[:, None]
        self.X = X.copy()
        self.Xprev = X.copy()
        self.snap = X.copy()
        self.tau = np.ones((3,) + self.solid.shape)
        self.u = np.zeros((3, self.dim) + self.solid.shape)
        self.t = 0

    def set_bc(self, x_in=None, current_A_cm2=None):
        if x_in is not None:
            self.x_in = np.array(x_in, dtype=np.float64)
        if current_A_cm2 is not None:
            self.sc.set_current(current_A_cm2)

    # ---------------------------------------------------------------- step 1
    def _shift(self, a):
        ex, ey, ez = self.E[a]
        return (int(ez), int(ey), int(ex))

    def _stream(self):
        A, E, W, opp = self.A, self.E, self.W, self.opp
        P = np.empty_like(A)
        for a in range(self.Q):
            sh = self._shift(a)
            P[:, a] = np.roll(A[:, a], sh, axis=(1, 2, 3))
            bounce = np.roll(self.solid, sh, axis=(0, 1, 2)) & self.fluid
            P[:, a][:, bounce] = A[:, opp[a]][:, bounce]
        if not self.periodic_x:
            nx = self.nx
            q = self.sc.q_lat
            w_out = sum(W[a] for a in range(self.Q) if E[a, 0] == 1)
            for a in range(self.Q):
                b = opp[a]
                if E[a, 0] == 1:
                    P[:, a, :, :, 0] = ((W[a] + W[b]) * self.x_in[:, None, None]
                                        - P[:, b, :, :, 0])
                elif E[a, 0] == -1 and self.outlet_bc == "flux":
                    P[:, a, :, :, nx - 1] = (A[:, b, :, :, nx - 1]
                                             - (W[b] / w_out) * q[:, None, None])
            if self.outlet_bc == "extrapolated":
                Dl = self.sc.D_lat
                Xn = np.where(self.solid[None, :, :, nx - 2], self.Xprev[:, :, :, nx - 1],
                              self.Xprev[:, :, :, nx - 2])
                dX = np.zeros_like(Xn)
                for i in range(3):
                    for j in range(3):
                        if j != i:
                            dX[i] += (Xn[i] * q[j] - Xn[j] * q[i]) / Dl[i, j]
                Xout = Xn + dX
                for a in range(self.Q):
                    if E[a, 0] == -1:
                        b = opp[a]
                        P[:, a, :, :, nx - 1] = (W[a] + W[b]) * Xout - P[:, b, :, :, nx - 1]
        P[:, :, self.solid] = 0.0
        return P

    # ---------------------------------------------------------------- step 3
    def _gradient(self, Xp):
        G = np.zeros((3, self.dim) + self.solid.shape)
        for a in range(self.dim):
            ax = 3 - a                       # x -> array axis 3, y -> 2, z -> 1
            p = np.roll(Xp, -1, axis=ax)     # value at x + e_a
            m = np.roll(Xp, 1, axis=ax)      # value at x - e_a
            p = np.where(np.roll(self.solid, -1, axis=ax - 1), Xp, p)
            m = np.where(np.roll(self.solid, 1, axis=ax - 1), Xp, m)
            if a == 0 and not self.periodic_x:
                xi = np.arange(self.nx)
                has_p = (xi < self.nx - 1).reshape(1, 1, -1)
                has_m = (xi > 0).reshape(1, 1, -1)
            else:
                has_p = np.ones((1, 1, 1), bool)
                has_m = np.ones((1, 1, 1), bool)
            if self.grad_stencil == "forward":
                if a == 0:
                    G[:, a] = np.where(has_p, p - Xp, np.where(has_m, Xp - m, 0.0))
                continue
            G[:, a] = np.where(has_p & has_m, 0.5 * (p - m),
                               np.where(has_p, p - Xp, np.where(has_m, Xp - m, 0.0)))
        return G

    # ------------------------------------------------------------ steps 4-6
    def _coupling(self, X, G):
        Dl = self.sc.D_lat
        D12, D13, D23 = Dl[0, 1], Dl[0, 2], Dl[1, 2]
        X1, X2, X3 = X[0], X[1], X[2]
        B11 = X1 / D13 + X2 / D12 + X3 / D13
        B12 = -X1 * (1.0 / D12 - 1.0 / D13)
        B21 = -X2 * (1.0 / D12 - 1.0 / D23)
        B22 = X2 / D23 + X1 / D12 + X3 / D23
        det = B11 * B22 - B12 * B21
        with np.errstate(divide="ignore", invalid="ignore"):
            inv_det = np.where(det > 0, 1.0 / np.where(det > 0, det, 1.0), 0.0)
        g1, g2, g3 = G[0], G[1], G[2]
        j1 = -(B22 * g1 - B12 * g2) * inv_det
        j2 = -(B11 * g2 - B21 * g1) * inv_det
        if self.closure == "eq21":
            # Section 3.2 literally: N_n = -(N_1 + N_2) (Eq. 21 with u_M = 0)
            j3 = -j1 - j2
        else:
            # species n from its own row of Eq. 19 given N_1, N_2
            d3 = X1 / D13 + X2 / D23
            with np.errstate(divide="ignore", invalid="ignore"):
                inv_d3 = np.where(d3 > 0, 1.0 / np.where(d3 > 0, d3, 1.0), 0.0)
            j3 = (-g3 + X3[None] * (j1 / D13 + j2 / D23)) * inv_d3
        J = np.stack([j1, j2, j3])

        nu = self.sc.stoich
        D = np.empty_like(X)
        for i in range(3):
            o = [k for k in range(3) if k != i]
            if nu[i] != 0:
                # Eq. 24 with N_j / N_i = nu_j / nu_i
                inv = sum((X[k] - X[i] * nu[k] / nu[i]) / Dl[i, k] for k in o)
                with np.errstate(divide="ignore", invalid="ignore"):
                    D[i] = np.where(inv > 0, 1.0 / np.where(inv > 0, inv, 1.0), D_BIG)
            else:
                num = X[o[0]] + X[o[1]] + MIX_DELTA
                den = (X[o[0]] / Dl[i, o[0]] + X[o[1]] / Dl[i, o[1]]
                       + MIX_DELTA * 0.5 * (1.0 / Dl[i, o[0]] + 1.0 / Dl[i, o[1]]))
                D[i] = num / den
        tau = np.clip(D / CS2 + 0.5, self.tau_min, self.tau_max)
        Dtau = CS2 * (tau - 0.5)
        xinv = X / (X * X + EPS_X * EPS_X)
        if self.coupling == "ms":
            v = (J + Dtau[:, None] * G) * xinv[:, None]
            vn2 = (v * v).sum(axis=1)
            with np.errstate(divide="ignore", invalid="ignore"):
                scale = np.where(vn2 > V_MAX * V_MAX, V_MAX / np.sqrt(np.maximum(vn2, 1e-300)), 1.0)
            v = v * scale[:, None]
        else:
            v = np.zeros_like(J)
        u = J * xinv[:, None]
        return tau, v, u

    # ------------------------------------------------------------------ step
    def step(self, n=1):
        for _ in range(int(n)):
            P = self._stream()
            X = P.sum(axis=1)
            X[:, self.solid] = 0.0
            G = self._gradient(self.Xprev if self.lag else X)
            tau, v, u = self._coupling(X, G)
            Anew = np.empty_like(P)
            for a in range(self.Q):
                ev = sum(self.E[a, d] * v[:, d] for d in range(self.dim))
                feq = self.W[a] * X * (1.0 + ev / CS2)
                Anew[:, a] = P[:, a] - (P[:, a] - feq) / tau
            Anew[:, :, self.solid] = 0.0
            tau = np.where(self.fluid, tau, 0.0)
            self.A = Anew
            self.X = X
            self.Xprev = X
            self.tau = tau
            self.u = np.where(self.fluid, u, 0.0)
            self.t += 1
        return self

    # -------------------------------------------------------------- outputs
    def residual(self, K):
        """K-step relative L2 change, max over species; refreshes the snapshot."""
        r = 0.0
        for i in range(3):
            nrm = np.sqrt((self.X[i] ** 2).sum())
            if nrm > 0:
                r = max(r, np.sqrt(((self.X[i] - self.snap[i]) ** 2).sum()) / (K * nrm))
        self.snap = self.X.copy()
        return r

    def run_to_residual(self, tol, max_steps, K=100):
        self.snap = self.X.copy()
        done = 0
        r = np.inf
        while done < max_steps:
            k = min(K, max_steps - done)
            self.step(k)
            done += k
            r = self.residual(k)
            if not np.isfinite(r) or r <= tol:
                break
        return done, r

    def outlet_mean(self):
        col = self.X[:, :, :, self.nx - 1]
        return col.reshape(3, -1).mean(axis=1)

    def overpotential(self):
        return self.sc.overpotential(self.x_in, self.outlet_mean())

    def plane_flux(self):
        """Net moles (mole-fraction units) per step crossing each plane
        x + 1/2, x = 0..nx-2, carried by the stored post-collision lattice."""
        F = np.zeros((3, self.nx - 1))
        for a in range(self.Q):
            ex = self.E[a, 0]
            if ex == 0:
                continue
            sh = self._shift(a)
            ok = self.fluid & ~np.roll(self.solid, tuple(-s for s in sh), axis=(0, 1, 2))
            col = (self.A[:, a] * ok).sum(axis=(1, 2))      # (3, nx)
            if ex == 1:
                F += col[:, :-1]
            else:
                F -= col[:, 1:]
        return F

    def total(self):
        return self.X.reshape(3, -1).sum(axis=1)

    def fields(self):
        """X, u (m/s, per axis) and tau of the last step, dense [z, y, x]."""
        return self.X.copy(), self.u * (self.sc.dx / self.sc.dt), self.tau.copy()
