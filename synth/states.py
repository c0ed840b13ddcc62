"""Initial and exact states of the test problems, as 12 x V float64 SoA arrays.

Row layout (the unknowns of Eq. (HWENO), Sec. 2.3): rows 0-3 hold w = (rho, rho*u, rho*v, E),
rows 4-7 its x derivatives w_x, rows 8-11 its y derivatives w_y.  Derivatives of smooth states
are exact: they are taken by the complex-step method (Im f(x + i*delta)/delta, delta = 1e-30),
which has no subtractive cancellation, so they are correct to rounding.
"""
import numpy as np

GAMMA = 1.4
_CS = 1e-30


def prim_to_cons(rho, u, v, p, gamma=GAMMA):
    """Conservative variables from primitives (works on complex input)."""
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


def _state_from_prim_fn(x, y, prim_fn, gamma):
    w = prim_to_cons(*prim_fn(x.astype(complex), y.astype(complex)), gamma=gamma).real
    wx = prim_to_cons(*prim_fn(x + 1j * _CS, y.astype(complex)), gamma=gamma).imag / _CS
    wy = prim_to_cons(*prim_fn(x.astype(complex), y + 1j * _CS), gamma=gamma).imag / _CS
    return np.ascontiguousarray(np.concatenate([w, wx, wy]))


def _min_image(d, L, periodic):
    if not periodic:
        return d
    return d - L * np.round(d.real / L)


def isentropic_vortex(mesh, beta=5.0, gamma=GAMMA, center=(5.0, 5.0), mean=(1.0, 1.0), t=0.0):
    """Isentropic vortex of Sec. 3.1 (strength beta, adiabatic p = rho^gamma) advected by the
    mean flow for time t; its centre is wrapped periodically.  Exact solution at time t."""
    xc = center[0] + mean[0] * t
    yc = center[1] + mean[1] * t
    a = (gamma - 1.0) * beta ** 2 / (8.0 * gamma * np.pi ** 2)

    def prim(x, y):
        xb = _min_image(x - xc, mesh["Lx"], mesh["periodic_x"])
        yb = _min_image(y - yc, mesh["Ly"], mesh["periodic_y"])
        r2 = xb * xb + yb * yb
        rho = (1.0 - a * np.exp(1.0 - r2)) ** (1.0 / (gamma - 1.0))
        s = beta / (2.0 * np.pi) * np.exp(0.5 * (1.0 - r2))
        return rho, mean[0] - s * yb, mean[1] + s * xb, rho ** gamma

    return _state_from_prim_fn(mesh["x"], mesh["y"], prim, gamma)


def uniform_state(mesh, rho=1.0, u=0.3, v=-0.2, p=1.0, gamma=GAMMA):
    V = len(mesh["x"])
    w = prim_to_cons(np.full(V, rho), np.full(V, u), np.full(V, v), np.full(V, p), gamma)
    return np.ascontiguousarray(np.concatenate([w, np.zeros((8, V))]))


def _piecewise(mesh, states, region, gamma):
    V = len(mesh["x"])
    U = np.zeros((12, V))
    for k, (rho, u, v, p) in enumerate(states):
        m = region == k
        U[:4, m] = prim_to_cons(rho, u, v, p, gamma)[:, None]
    return U


def four_quadrant(mesh, gamma=GAMMA, xm=0.5, ym=0.5):
    """Four-quadrant Riemann problem (shocks and contacts meeting at (xm, ym)); zero derivatives.
    Quadrants: (x>=xm,y>=ym) (1.5,0,0,1.5); (x<xm,y>=ym) (0.5323,1.206,0,0.3);
    (x<xm,y<ym) (0.138,1.206,1.206,0.029); (x>=xm,y<ym) (0.5323,0,1.206,0.3) as (rho,u,v,p)."""
    x, y = mesh["x"], mesh["y"]
    region = np.where(x >= xm, np.where(y >= ym, 0, 3), np.where(y >= ym, 1, 2))
    states = [(1.5, 0.0, 0.0, 1.5), (0.5323, 1.206, 0.0, 0.3),
              (0.138, 1.206, 1.206, 0.029), (0.5323, 0.0, 1.206, 0.3)]
    return _piecewise(mesh, states, region, gamma)


def planar_sod(mesh, gamma=GAMMA, x0=0.5, left=(1.0, 0.0, 0.0, 1.0), right=(0.125, 0.0, 0.0, 0.1)):
    """Sod's shock tube along x (discontinuity at x = x0); zero derivatives."""
    region = (mesh["x"] >= x0).astype(int)
    return _piecewise(mesh, [left, right], region, gamma)


def circular_sod(mesh, gamma=GAMMA, radius=0.5, inside=(1.0, 0.0, 0.0, 1.0),
                 outside=(0.125, 0.0, 0.0, 0.1)):
    """Circular Sod problem of Sec. 3.3: the inside state where |r| < radius, the outside state
    elsewhere; zero derivatives.  The circle's own vertices (mesh["on_circle"], placed exactly
    on it by `embedded_circle_box`) take the outside state, as the strict inequality says.  The
    outside velocity printed in the paper is garbled; it is read as 0 (at rest)."""
    r = np.hypot(mesh["x"], mesh["y"])
    region = (r >= radius).astype(int)
    if "on_circle" in mesh:
        region[mesh["on_circle"]] = 1
    return _piecewise(mesh, [inside, outside], region, gamma)


def taylor_green(mesh, mach=0.1, gamma=GAMMA):
    """Decaying Taylor-Green vortex initial state on [0, 2pi]^2: u = sin x cos y,
    v = -cos x sin y, rho = 1, p = p0 + (cos 2x + cos 2y)/4 with p0 = 1/(gamma M^2)."""
    p0 = 1.0 / (gamma * mach * mach)

    def prim(x, y):
        one = np.ones_like(x)
        return (one, np.sin(x) * np.cos(y), -np.cos(x) * np.sin(y),
                p0 + 0.25 * (np.cos(2 * x) + np.cos(2 * y)))

    return _state_from_prim_fn(mesh["x"], mesh["y"], prim, gamma)


def couette(mesh, u0=1.0, T_bottom=10.0, T_top=12.0, p=10.0, gamma=GAMMA, cp=10.0, kappa=0.01,
            mu=0.1, half=5.0):
    """Exact compressible Couette flow of Sec. 3.2 between walls at y = -half (moving at -u0)
    and y = +half (+u0): u = u0 y / half, v = 0, uniform p, and the temperature that balances
    conduction against viscous heating, kappa T'' + mu u'^2 = 0, with T = T_bottom / T_top at
    the walls; rho = gamma p / ((gamma - 1) cp T).  Extended unchanged into the ghost bands."""
    L = 2.0 * half

    def prim(x, y):
        u = 2.0 * y / L * u0
        T = (-2.0 * mu * u0 * u0 / (kappa * L * L) * y * y + (T_top - T_bottom) / L * y
             + 0.5 * (T_top + T_bottom) + 0.5 * mu * u0 * u0 / kappa)
        rho = gamma * p / ((gamma - 1.0) * cp * T)
        return rho, u, 0.0 * y, p + 0.0 * y

    return _state_from_prim_fn(mesh["x"], mesh["y"], prim, gamma)

