"""Seeded jittered, randomly split structured triangle meshes.

The paper's tests run on Delaunay meshes of a square (Sec. 3.1: 3957-36408 nodes; Sec. 3.3:
3970-35458 nodes) that are not distributed with it.  These generators stand in for them: a
structured vertex grid whose vertices are jittered by U(-j*h, j*h) per axis and whose quads are
split along a Bernoulli(0.5) random diagonal.  Triangles are counter-clockwise.

Two kinds of axis are supported:
  * periodic: n vertices at a + i*L/n, i = 0..n-1, quads wrap around;
  * bounded:  n physical vertices at a + i*(b-a)/(n-1) (the boundary lines are not jittered),
              plus `ghost` layers of unjittered ghost vertices outside [a, b].  Each ghost vertex
              names a donor (the nearest physical vertex, by clamping the grid index) and flags
              which derivative components are zeroed when it is refreshed (bit 0: the x
              derivatives, bit 1: the y derivatives, i.e. the derivative normal to the boundary
              the ghost lies beyond).  A donor of -1 marks a fixed ghost, whose values the
              caller sets and nothing refreshes (`couette_channel`).

Vertex ids are row-major over the (possibly ghost-extended) grid.  Random draws, in order from
numpy's PCG64(seed): x jitter for all vertices, y jitter for all vertices, one diagonal bit
per quad.
"""
import numpy as np


def _axis(n, lo, hi, periodic, ghost):
    """Grid coordinates, physical mask and clamp index along one axis."""
    if periodic:
        h = (hi - lo) / n
        idx = np.arange(n)
        return lo + idx * h, np.ones(n, bool), idx, h, np.zeros(n, bool)
    h = (hi - lo) / (n - 1)
    idx = np.arange(-ghost, n + ghost)
    coord = lo + idx * h
    physical = (idx >= 0) & (idx <= n - 1)
    boundary = (idx == 0) | (idx == n - 1)
    return coord, physical, np.clip(idx, 0, n - 1) + ghost, h, boundary


def _grid(nx, ny, xr, yr, periodic_x, periodic_y, ghost, jitter, seed):
    cx, px, clx, hx, bx = _axis(nx, xr[0], xr[1], periodic_x, ghost)
    cy, py, cly, hy, by = _axis(ny, yr[0], yr[1], periodic_y, ghost)
    NX, NY = len(cx), len(cy)
    V = NX * NY
    rng = np.random.Generator(np.random.PCG64(seed))
    jx = rng.uniform(-1.0, 1.0, V) * (jitter * hx)
    jy = rng.uniform(-1.0, 1.0, V) * (jitter * hy)
    QX = NX if periodic_x else NX - 1
    QY = NY if periodic_y else NY - 1
    diag = rng.integers(0, 2, QX * QY)

    I, J = np.meshgrid(np.arange(NX), np.arange(NY), indexing="xy")
    I = I.ravel()
    J = J.ravel()
    phys = px[I] & py[J]
    on_bnd = bx[I] | by[J]
    jit = phys & ~on_bnd
    x = cx[I] + np.where(jit, jx, 0.0)
    y = cy[J] + np.where(jit, jy, 0.0)

    qI, qJ = np.meshgrid(np.arange(QX), np.arange(QY), indexing="xy")
    qI = qI.ravel()
    qJ = qJ.ravel()
    v00 = qJ * NX + qI
    v10 = qJ * NX + (qI + 1) % NX
    v01 = ((qJ + 1) % NY) * NX + qI
    v11 = ((qJ + 1) % NY) * NX + (qI + 1) % NX
    t0 = np.where(diag[:, None] == 0, np.stack([v00, v10, v11], 1), np.stack([v00, v10, v01], 1))
    t1 = np.where(diag[:, None] == 0, np.stack([v00, v11, v01], 1), np.stack([v10, v11, v01], 1))
    tri = np.concatenate([t0, t1]).astype(np.int32)

    ghost_ids = np.nonzero(~phys)[0].astype(np.int32)
    gI, gJ = I[ghost_ids], J[ghost_ids]
    donor = (cly[gJ] * NX + clx[gI]).astype(np.int32)
    flags = ((clx[gI] != gI).astype(np.int32) | ((cly[gJ] != gJ).astype(np.int32) << 1))
    return {
        "x": x, "y": y, "tri": tri,
        "Lx": float(xr[1] - xr[0]), "Ly": float(yr[1] - yr[0]),
        "periodic_x": bool(periodic_x), "periodic_y": bool(periodic_y),
        "ghost_ids": ghost_ids, "ghost_donor": donor, "ghost_flags": flags.astype(np.int32),
        "grid": (NX, NY), "h": (hx, hy), "seed": seed,
    }


def jittered_grid(nx, ny, Lx, Ly, seed, jitter=0.15, x0=0.0, y0=0.0):
    """Doubly periodic nx-by-ny vertex grid on [x0, x0+Lx) x [y0, y0+Ly), every vertex jittered."""
    return _grid(nx, ny, (x0, x0 + Lx), (y0, y0 + Ly), True, True, 0, jitter, seed)


def jittered_box_with_ghosts(nx, ny, xr, yr, ghost, seed, jitter=0.15, periodic_y=False):
    """nx-by-ny physical vertices on the closed box xr x yr with `ghost` ghost layers outside
    each bounded side (y may instead be periodic).  Boundary lines and ghosts are unjittered."""
    return _grid(nx, ny, xr, yr, False, periodic_y, ghost, jitter, seed)


def couette_channel(nx, ny, ghost, seed, jitter=0.15, half=5.0):
    """Channel of Sec. 3.2: x periodic on [-half, half), walls at y = -half and y = +half,
    `ghost` layers of fixed ghost vertices beyond each wall (donor -1: the caller's values are
    kept, here the exact solution).  nx-by-ny physical vertices."""
    m = _grid(nx, ny, (-half, half), (-half, half), True, False, ghost, jitter, seed)
    m["ghost_donor"] = np.full(len(m["ghost_ids"]), -1, dtype=np.int32)
    m["ghost_flags"] = np.zeros(len(m["ghost_ids"]), dtype=np.int32)
    return m


def mesh_summary(mesh):
    V = len(mesh["x"])
    return {"vertices": V, "triangles": len(mesh["tri"]), "ghosts": len(mesh["ghost_ids"]),
            "active": V - len(mesh["ghost_ids"])}


def embedded_circle_box(n, seed, radius=0.5, half=1.0, ghost=5, jitter=0.15, band=0.5):
    """Square [-half, half]^2 split into n segments per side with a circle of `radius` embedded
    at the centre (Sec. 3.3: the circle carries the initial discontinuity, so it is a line of
    mesh vertices).  Construction:
      * the (n+1)^2 physical grid vertices, interior ones jittered as in `jittered_box_with_ghosts`,
        plus `ghost` unjittered ghost layers outside each side (donors as there);
      * every jittered vertex within band*h of the circle is removed, and round(2 pi radius / h)
        vertices are placed on the circle at equal angles (the first at angle 0);
      * the vertices are triangulated by Delaunay (scipy's Qhull).  Exactly cocircular sets
        (unjittered grid cells) are broken by triangulating on coordinates moved by at most
        1e-6 h for every unjittered vertex off the outermost ring; the stored coordinates are
        the exact ones.
    Returns a mesh dict like the other generators plus "on_circle" (bool per vertex).  Random
    draws, in order from PCG64(seed): the grid's x and y jitter and diagonal bits (diagonals
    unused), then the tie-breaking moves (x then y)."""
    from scipy.spatial import Delaunay

    g = _grid(n + 1, n + 1, (-half, half), (-half, half), False, False, ghost, jitter, seed)
    h = g["h"][0]
    NX, NY = g["grid"]
    x, y = g["x"], g["y"]
    V = len(x)
    I = np.arange(V) % NX
    J = np.arange(V) // NX
    phys = np.ones(V, bool)
    phys[g["ghost_ids"]] = False
    on_bnd = phys & ((I == ghost) | (I == NX - 1 - ghost) | (J == ghost) | (J == NY - 1 - ghost))
    jittered = phys & ~on_bnd
    r = np.hypot(x, y)
    keep = ~(jittered & (np.abs(r - radius) < band * h))
    if not np.all(keep[~jittered]):
        raise ValueError("the circle must lie inside the jittered interior")
    nc = int(round(2.0 * np.pi * radius / h))
    th = 2.0 * np.pi * np.arange(nc) / nc
    old = np.nonzero(keep)[0]
    new_id = np.full(V, -1, np.int64)
    new_id[old] = np.arange(len(old))
    xs = np.concatenate([x[old], radius * np.cos(th)])
    ys = np.concatenate([y[old], radius * np.sin(th)])
    on_circle = np.concatenate([np.zeros(len(old), bool), np.ones(nc, bool)])
    fixed = np.concatenate([~jittered[old], np.zeros(nc, bool)])
    outer = np.concatenate([(I[old] == 0) | (I[old] == NX - 1) | (J[old] == 0) | (J[old] == NY - 1),
                            np.zeros(nc, bool)])
    rng = np.random.Generator(np.random.PCG64(seed))
    rng.uniform(size=2 * V)                      # the grid's jitter draws
    rng.integers(0, 2, (NX - 1) * (NY - 1))      # the grid's diagonal bits
    move = fixed & ~outer
    tx = xs + np.where(move, rng.uniform(-1.0, 1.0, len(xs)), 0.0) * 1e-6 * h
    ty = ys + np.where(move, rng.uniform(-1.0, 1.0, len(xs)), 0.0) * 1e-6 * h
    dl = Delaunay(np.stack([tx, ty], 1))
    if len(dl.coplanar):
        raise RuntimeError("Delaunay left vertices out of the triangulation")
    tri = dl.simplices.astype(np.int64)
    a = ((xs[tri[:, 1]] - xs[tri[:, 0]]) * (ys[tri[:, 2]] - ys[tri[:, 0]])
         - (xs[tri[:, 2]] - xs[tri[:, 0]]) * (ys[tri[:, 1]] - ys[tri[:, 0]]))
    tri[a < 0] = tri[a < 0][:, [0, 2, 1]]
    gid = new_id[g["ghost_ids"]]
    donor = new_id[g["ghost_donor"]]
    if np.any(gid < 0) or np.any(donor < 0):
        raise RuntimeError("a ghost or donor vertex was removed")
    return {
        "x": xs, "y": ys, "tri": tri.astype(np.int32),
        "Lx": 2.0 * half, "Ly": 2.0 * half, "periodic_x": False, "periodic_y": False,
        "ghost_ids": gid.astype(np.int32), "ghost_donor": donor.astype(np.int32),
        "ghost_flags": g["ghost_flags"], "grid": (NX, NY), "h": (h, h), "seed": seed,
        "on_circle": on_circle, "radius": radius,
    }


def vertex_areas(mesh):
    """Weights of an area-weighted objective over the vertices (the adjoint workload's
    J = sum_v A_v (rho - rho_exact)^2): one third of the area of every incident triangle, with
    triangle edges taken by the minimum image across periodic sides."""
    x, y = np.asarray(mesh["x"]), np.asarray(mesh["y"])
    t = np.asarray(mesh["tri"], dtype=np.int64)

    def d(a, b, c, L, per):
        v = c[b] - c[a]
        return v - L * np.round(v / L) if per else v
    ax, ay = d(t[:, 0], t[:, 1], x, mesh["Lx"], mesh["periodic_x"]), d(t[:, 0], t[:, 1], y, mesh["Ly"], mesh["periodic_y"])
    bx, by = d(t[:, 0], t[:, 2], x, mesh["Lx"], mesh["periodic_x"]), d(t[:, 0], t[:, 2], y, mesh["Ly"], mesh["periodic_y"])
    third = (0.5 * (ax * by - ay * bx)) / 3.0
    A = np.zeros(len(x))
    for k in range(3):
        np.add.at(A, t[:, k], third)
    return A
