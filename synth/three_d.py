"""Seeded periodic tetrahedral meshes and 3D states for the three-dimensional extension.

The paper is two-dimensional and names the extension to three dimensions as future work
(Sec. 4); these inputs serve that extension.  The mesh stands in for an unstructured
tetrahedral mesh the way the 2D generator stands in for the paper's Delaunay meshes: an
n_x x n_y x n_z periodic vertex grid on [0, L_x) x [0, L_y) x [0, L_z), every vertex jittered by
U(-j h, j h) per axis, and every cell split into the six tetrahedra of the Kuhn (Freudenthal)
subdivision, which share the cell's main diagonal (000)-(111).  Neighbouring cells split the
same way, so the tetrahedra form a conforming mesh; each vertex has 14 edges.

Vertex ids are lexicographic, id = i + n_x (j + n_y k).  Random draws, in order from numpy's
PCG64(seed): x jitter, y jitter, z jitter for all vertices.

States are 20 x V float64 SoA arrays: rows 0-4 hold w = (rho, rho u, rho v, rho w, E), rows 5-9
its x derivatives, rows 10-14 its y derivatives and rows 15-19 its z derivatives.  Derivatives
of smooth states are taken by the complex-step method (correct to rounding).
"""
import numpy as np

GAMMA = 1.4
_CS = 1e-30

# the six Kuhn tetrahedra of the unit cell: vertex paths from corner 000 to 111 that add one
# unit vector at a time, one per permutation of the axes
_KUHN = []
for _perm in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
    _c = [0, 0, 0]
    _path = [tuple(_c)]
    for _ax in _perm:
        _c[_ax] = 1
        _path.append(tuple(_c))
    _KUHN.append(_path)


def periodic_tet_box(nx, ny, nz, Lx, Ly, Lz, seed, jitter=0.15):
    """Periodic jittered Kuhn-split tetrahedral mesh; returns a dict with x, y, z (V,), tet
    (T, 4) vertex ids with positive orientation (by minimum image), the box lengths and
    periodic flags, and the grid shape."""
    V = nx * ny * nz
    hx, hy, hz = Lx / nx, Ly / ny, Lz / nz
    rng = np.random.Generator(np.random.PCG64(seed))
    jx = rng.uniform(-1.0, 1.0, V) * (jitter * hx)
    jy = rng.uniform(-1.0, 1.0, V) * (jitter * hy)
    jz = rng.uniform(-1.0, 1.0, V) * (jitter * hz)
    K, J, I = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    I, J, K = I.ravel(), J.ravel(), K.ravel()
    x = I * hx + jx
    y = J * hy + jy
    z = K * hz + jz

    def vid(i, j, k):
        return (i % nx) + nx * ((j % ny) + ny * (k % nz))

    tets = []
    for path in _KUHN:
        tets.append(np.stack([vid(I + a, J + b, K + c) for (a, b, c) in path], 1))
    tet = np.concatenate(tets)
    mesh = {"x": x, "y": y, "z": z, "tet": tet, "Lx": float(Lx), "Ly": float(Ly),
            "Lz": float(Lz), "periodic": True, "shape": (nx, ny, nz)}
    # orient every tetrahedron positively (minimum-image edge vectors)
    d = [disp3(mesh, tet[:, 0], tet[:, k]) for k in (1, 2, 3)]
    vol = np.einsum("ij,ij->i", d[0], np.cross(d[1], d[2]))
    flip = vol < 0
    tet[flip, 1], tet[flip, 2] = tet[flip, 2].copy(), tet[flip, 1].copy()
    mesh["tet"] = tet
    return mesh


def disp3(mesh, a, b):
    """Vector(s) from vertex a to vertex b, minimum image on the periodic box; shape (..., 3)."""
    d = np.stack([mesh["x"][b] - mesh["x"][a], mesh["y"][b] - mesh["y"][a],
                  mesh["z"][b] - mesh["z"][a]], -1)
    L = np.array([mesh["Lx"], mesh["Ly"], mesh["Lz"]])
    return d - L * np.round(d / L)


def prim_to_cons3(rho, u, v, w, p, gamma=GAMMA):
    """Conservative variables from primitives (works on complex input)."""
    return np.stack([rho, rho * u, rho * v, rho * w,
                     p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)])


def _state(mesh, prim_fn, gamma):
    x, y, z = (mesh[k].astype(complex) for k in ("x", "y", "z"))
    w0 = prim_to_cons3(*prim_fn(x, y, z), gamma=gamma).real
    parts = [w0]
    for axis in range(3):
        c = [x, y, z]
        c[axis] = c[axis] + 1j * _CS
        parts.append(prim_to_cons3(*prim_fn(*c), gamma=gamma).imag / _CS)
    return np.ascontiguousarray(np.concatenate(parts))


def _wrap(d, L):
    return d - L * np.round(d.real / L)


def uniform_state3(mesh, rho=1.0, u=0.3, v=-0.2, w=0.1, p=1.0, gamma=GAMMA):
    """A constant state (zero derivatives): the freestream."""
    V = len(mesh["x"])
    out = np.zeros((20, V))
    out[0:5] = prim_to_cons3(rho, u, v, w, p, gamma)[:, None]
    return out


def vortex_tube(mesh, beta=5.0, gamma=GAMMA, center=None, mean=(1.0, 1.0, 0.5), t=0.0):
    """The isentropic vortex of Sec. 3.1 (strength beta, p = rho^gamma) as a straight tube
    along z, advected by the mean flow (u0, v0, w0) for time t: an exact solution of the 3D
    Euler equations (the axial velocity is uniform).  The centre line is wrapped periodically."""
    if center is None:
        center = (0.5 * mesh["Lx"], 0.5 * mesh["Ly"])
    xc = center[0] + mean[0] * t
    yc = center[1] + mean[1] * t
    a = (gamma - 1.0) * beta ** 2 / (8.0 * gamma * np.pi ** 2)

    def prim(x, y, z):
        xb = _wrap(x - xc, mesh["Lx"])
        yb = _wrap(y - yc, mesh["Ly"])
        r2 = xb * xb + yb * yb
        rho = (1.0 - a * np.exp(1.0 - r2)) ** (1.0 / (gamma - 1.0))
        s = beta / (2.0 * np.pi) * np.exp(0.5 * (1.0 - r2))
        return rho, mean[0] - s * yb, mean[1] + s * xb, mean[2] + 0.0 * z, rho ** gamma

    return _state(mesh, prim, gamma)


def density_wave(mesh, amp=0.2, vel=(0.5, -0.3, 0.4), p=1.0, gamma=GAMMA, t=0.0):
    """A smooth density wave rho = 1 + amp sin(2 pi (x/Lx + y/Ly + z/Lz)) carried by a uniform
    velocity at uniform pressure: an exact solution of the 3D Euler equations, whose exact time
    derivative is -(vel . grad) w."""
    Lx, Ly, Lz = mesh["Lx"], mesh["Ly"], mesh["Lz"]

    def prim(x, y, z):
        ph = 2.0 * np.pi * ((x - vel[0] * t) / Lx + (y - vel[1] * t) / Ly + (z - vel[2] * t) / Lz)
        rho = 1.0 + amp * np.sin(ph)
        one = 1.0 + 0.0 * x
        return rho, vel[0] * one, vel[1] * one, vel[2] * one, p * one

    return _state(mesh, prim, gamma)


def planar_sod3(mesh, gamma=GAMMA, left=(1.0, 0.0, 0.0, 0.0, 1.0), right=(0.125, 0.0, 0.0, 0.0, 0.1)):
    """Sod's shock-tube data along x in the periodic box: the left state on
    L_x/4 <= x < 3 L_x/4 and the right state elsewhere (two discontinuities), zero
    derivatives."""
    x = np.mod(mesh["x"], mesh["Lx"])
    inside = (x >= 0.25 * mesh["Lx"]) & (x < 0.75 * mesh["Lx"])
    V = len(x)
    out = np.zeros((20, V))
    wl = prim_to_cons3(*left, gamma=gamma)
    wr = prim_to_cons3(*right, gamma=gamma)
    out[0:5] = np.where(inside[None], wl[:, None], wr[:, None])
    return out
