"""1D radially symmetric Euler reference solver for the circular Sod problem (Sec. 3.3).
TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper compares its circular Sod profiles at t = 0.2 with "the exact result".  For a
cylindrically symmetric flow that result is the solution of the 1D Euler equations in the radius
with the geometric source of the divergence in polar coordinates,
    d(r U)/dt + d(r F)/dr = (0, p, 0),   U = (rho, rho u, E),  F = (rho u, rho u^2 + p, u (E + p)),
computed here at high resolution.  It is the standard reduction of a cylindrically symmetric
flow to one space dimension with a geometric source term, written as a finite-volume scheme on
cells [r_{i-1/2}, r_{i+1/2}]:
  * cell "volumes" V_i = (r_{i+1/2}^2 - r_{i-1/2}^2) / 2 and face "areas" A = r (per radian), so
    mass and energy are conserved exactly and a fluid at rest stays at rest (the pressure source
    p_i (A_{i+1/2} - A_{i-1/2}) balances the pressure flux);
  * piecewise-linear primitive variables with the minmod limiter (MUSCL);
  * the HLLC approximate Riemann solver with Davis wave-speed estimates (min / max of u -+ c);
  * SSP-RK3 in time at a CFL number below one half;
  * the axis r = 0 a mirror (no flux through a face of zero area), the outer radius transmissive.
alpha = 0 gives the planar (1D Cartesian) scheme on the same cells, for the pins against the
exact Riemann solution.
"""
import numpy as np


def _prim(U, g):
    rho = U[0]
    u = U[1] / rho
    p = (g - 1.0) * (U[2] - 0.5 * rho * u * u)
    return rho, u, p


def _cons(rho, u, p, g):
    return np.stack([rho, rho * u, p / (g - 1.0) + 0.5 * rho * u * u])


def _minmod(a, b):
    return np.where(a * b > 0.0, np.sign(a) * np.minimum(np.abs(a), np.abs(b)), 0.0)


def _hllc(rl, ul, pl, rr, ur, pr, g):
    """HLLC flux across faces with left / right primitive states (arrays)."""
    cl, cr = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    sl = np.minimum(ul - cl, ur - cr)
    sr = np.maximum(ul + cl, ur + cr)
    sm = (pr - pl + rl * ul * (sl - ul) - rr * ur * (sr - ur)) / (rl * (sl - ul) - rr * (sr - ur))
    El = pl / (g - 1.0) + 0.5 * rl * ul * ul
    Er = pr / (g - 1.0) + 0.5 * rr * ur * ur
    Fl = np.stack([rl * ul, rl * ul * ul + pl, ul * (El + pl)])
    Fr = np.stack([rr * ur, rr * ur * ur + pr, ur * (Er + pr)])
    Ul = np.stack([rl, rl * ul, El])
    Ur = np.stack([rr, rr * ur, Er])

    def star(r, u, p, E, s):
        f = r * (s - u) / (s - sm)
        return np.stack([f, f * sm, f * (E / r + (sm - u) * (sm + p / (r * (s - u))))])
    Fsl = Fl + sl * (star(rl, ul, pl, El, sl) - Ul)
    Fsr = Fr + sr * (star(rr, ur, pr, Er, sr) - Ur)
    return np.where(sl >= 0.0, Fl, np.where(sm >= 0.0, Fsl, np.where(sr > 0.0, Fsr, Fr)))


class Radial:
    """Cells of width dr on [0, R]; alpha = 1 cylindrical (the circular Sod problem), 0 planar."""

    def __init__(self, n, R, alpha=1, gamma=1.4):
        self.n, self.R, self.alpha, self.g = n, R, alpha, gamma
        self.dr = R / n
        self.rf = np.linspace(0.0, R, n + 1)             # faces
        self.rc = 0.5 * (self.rf[1:] + self.rf[:-1])     # centres
        if alpha == 1:
            self.A = self.rf.copy()
            self.V = 0.5 * (self.rf[1:] ** 2 - self.rf[:-1] ** 2)
        else:
            self.A = np.ones(n + 1)
            self.V = np.full(n, self.dr)

    def rhs(self, U):
        g = self.g
        rho, u, p = _prim(U, g)
        q = np.stack([rho, u, p])
        # ghost cells: a mirror at the axis (u odd) for the cylinder, transmissive elsewhere
        left = q[:, :2][:, ::-1].copy()
        if self.alpha == 1:
            left[1] = -left[1]
        qe = np.concatenate([left, q, q[:, -1:], q[:, -1:]], axis=1)
        d = _minmod(qe[:, 1:-1] - qe[:, :-2], qe[:, 2:] - qe[:, 1:-1])   # slopes of cells -1..n
        qL = qe[:, 1:-2] + 0.5 * d[:, :-1]       # left state at faces 0..n (cells -1..n-1)
        qR = qe[:, 2:-1] - 0.5 * d[:, 1:]        # right state at faces 0..n (cells 0..n)
        F = _hllc(qL[0], qL[1], qL[2], qR[0], qR[1], qR[2], g) * self.A
        out = -(F[:, 1:] - F[:, :-1])
        out[1] += p * (self.A[1:] - self.A[:-1])    # geometric source of the cylinder (0 planar)
        return out / self.V

    def dt(self, U, cfl=0.4):
        rho, u, p = _prim(U, self.g)
        return cfl * self.dr / np.max(np.abs(u) + np.sqrt(self.g * p / rho))

    def run(self, U, t_end, cfl=0.4):
        """SSP-RK3 from state U (3 x n conservative) to time t_end."""
        t = 0.0
        while t < t_end - 1e-15:
            dt = min(self.dt(U, cfl), t_end - t)
            U1 = U + dt * self.rhs(U)
            U2 = 0.75 * U + 0.25 * (U1 + dt * self.rhs(U1))
            U = U / 3.0 + 2.0 / 3.0 * (U2 + dt * self.rhs(U2))
            t += dt
        return U


def circular_sod(t_end, n=4000, R=2.0, r0=0.5, inside=(1.0, 0.0, 1.0), outside=(0.125, 0.0, 0.1),
                 gamma=1.4):
    """Reference density, velocity and pressure of the circular Sod problem (Sec. 3.3) at time
    t_end: cell centres r and the primitive profiles, n cells on [0, R]."""
    s = Radial(n, R, alpha=1, gamma=gamma)
    inner = s.rc < r0
    rho = np.where(inner, inside[0], outside[0])
    u = np.where(inner, inside[1], outside[1])
    p = np.where(inner, inside[2], outside[2])
    U = s.run(_cons(rho, u, p, gamma), t_end)
    return s.rc, _prim(U, gamma)
