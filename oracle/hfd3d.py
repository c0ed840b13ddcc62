"""FP64 oracle of the three-dimensional extension of the Hermite FD residual and SSP-RK3 step.

TEST INFRASTRUCTURE ONLY (see the package docstring): the product path never calls this.

The paper is two-dimensional and names three dimensions as future work (Sec. 4).  This module
carries each step of the 2D method over to tetrahedral meshes in the most direct way, and it
is the reference the 3D CUDA path is checked against.  The readings that three dimensions force
(T1-T6) are listed with the 3D design notes:
  * Sec. 2.1 and Fig. 1: curvilinear 6-node stencil per edge, extended twice from each end along
    the incident edge of smallest deflection (the same rule, with 3D cosines) -> `edge_stencil`.
  * Sec. 2.2: Hermite least squares on 5 nodes with data w, w_x, w_y, w_z: 20 equations.  T1: the
    basis is the complete degree-3 Taylor basis in 3D, whose 20 terms match the 20 data (the 2D
    method matches its 15 data with degree 4), so the interpolation is fourth order.  The same
    scaling, singular-value dropping (R3) and value-weight fix (R4) as in 2D  -> `five_node_weights`.
  * Sec. 2.3, Eq. (3nodes_intp): 3-node values-only systems, T2: with the degree-2 Taylor
    basis in 3D (10 terms), minimum-norm first row, exact rational arithmetic -> `three_node_weights`.
  * Sec. 2.3, Eq. (HWENO): unknowns w, w_x, w_y, w_z (20 per vertex).
  * Sec. 2.3, Alg. 1: Roe average of the edge ends, characteristic projection along the edge
    direction n with five waves (q_n - c, entropy, two shear waves, q_n + c).  T3: the shear
    waves use the tangents t1 = e_k x n / |e_k x n| (e_k the axis with the smallest |n_k|, lowest
    k on ties) and t2 = n x t1.  Uniform WENO5 weights as the sensor, 5-node or weighted 3-node
    value per component and side, back-projection, positivity fallback (R16) -> `edge_values`.
  * Riemann flux: Roe's flux with Harten's fix on all five waves (R9)    -> `roe_flux`.
  * Sec. 2.3, Eq. (flux_polynomials) and the d-rows: two-level least squares for the three flux
    vectors (f, g, k) from vertex values and edge projections; T4: degree 4 (35 terms per flux,
    105 unknowns), fixed (a stencil whose sigma_min/sigma_max falls below div_cond_min is an
    error); rows d_0, d_x, d_y, d_z                                      -> `div_rows`.
  * T5: periodic boxes only (no ghost layers); every vertex is active.
  * T6: the inviscid equations only (no viscous rows).
  * Sec. 2.3 (end): three-stage TVD (SSP) Runge-Kutta                   -> `step`.

State layout: U is a 20 x V float64 array; rows 0-4 are w = (rho, rho u, rho v, rho w, E), rows
5-9 w_x, rows 10-14 w_y and rows 15-19 w_z.  Vertex ids are the input's.
"""
from dataclasses import dataclass
from fractions import Fraction
from math import factorial

import numpy as np
import scipy.sparse as sp

from .hfd_oracle import weno_weights, ssp_rk3


@dataclass
class Options3:
    gamma: float = 1.4
    weno_eps: float = 1e-2        # R2, as in 2D
    sens_lo: float = 0.01         # Sec. 2.3 sensor band, as in 2D
    sens_hi: float = 0.79
    div_degree: int = 4           # T4
    sv_rtol: float = 1e-13        # R3
    div_cond_min: float = 1e-12   # T4: smaller sigma_min/sigma_max is an error
    harten: float = 0.1           # R9
    force_branch: str = "sensor"  # testing aid: "hermite" / "weno" everywhere
    cfl: float = 0.3              # R12


# --------------------------------------------------------------------------- topology

def build_topology(mesh):
    """Unique undirected edges of the tetrahedra, oriented tail < head and sorted; sorted
    neighbour lists; edge lookup."""
    tet = np.asarray(mesh["tet"], dtype=np.int64)
    V = len(mesh["x"])
    e = np.concatenate([tet[:, [a, b]] for a in range(4) for b in range(a + 1, 4)])
    e = np.unique(np.sort(e, axis=1), axis=0)
    nbrs = [[] for _ in range(V)]
    for a, b in e:
        nbrs[a].append(b)
        nbrs[b].append(a)
    nbrs = [np.array(sorted(n), dtype=np.int64) for n in nbrs]
    index = {(int(a), int(b)): k for k, (a, b) in enumerate(e)}
    return {"edges": e, "nbrs": nbrs, "index": index, "V": V}


def disp(mesh, a, b):
    """Vector from vertex a to vertex b, minimum image on the periodic box."""
    d = np.array([mesh["x"][b] - mesh["x"][a], mesh["y"][b] - mesh["y"][a],
                  mesh["z"][b] - mesh["z"][a]])
    L = np.array([mesh["Lx"], mesh["Ly"], mesh["Lz"]])
    return d - L * np.round(d / L)


def _extend(mesh, topo, cur, t, used):
    """One extension step (Sec. 2.1): the unused neighbour of `cur` whose edge has the largest
    cosine with the travel direction t; ties within 1e-12 keep the lower id (R11)."""
    best, best_cos, best_d = -1, -np.inf, None
    tn = np.sqrt(t @ t)
    for c in topo["nbrs"][cur]:
        if c in used:
            continue
        d = disp(mesh, cur, c)
        cs = (t @ d) / (tn * np.sqrt(d @ d))
        if cs > best_cos + 1e-12:
            best, best_cos, best_d = int(c), cs, d
    if best < 0:
        raise ValueError(f"stencil cannot be extended from vertex {cur}")
    return best, best_d


def edge_stencil(mesh, topo, e):
    """6-node stencil [i-2, i-1, i, i+1, i+2, i+3] of edge e = (i, i+1) (Sec. 2.1): two
    extensions backwards from the tail, two forwards from the head; positions relative to the
    tail, accumulated along the path."""
    a, b = (int(v) for v in topo["edges"][e])
    used = {a, b}
    dab = disp(mesh, a, b)
    b1, d1 = _extend(mesh, topo, a, -dab, used)
    used.add(b1)
    b2, d2 = _extend(mesh, topo, b1, d1, used)
    used.add(b2)
    f1, d3 = _extend(mesh, topo, b, dab, used)
    used.add(f1)
    f2, d4 = _extend(mesh, topo, f1, d3, used)
    ids = np.array([b2, b1, a, b, f1, f2], dtype=np.int64)
    pos = np.zeros((6, 3))
    pos[1] = d1
    pos[0] = pos[1] + d2
    pos[3] = dab
    pos[4] = pos[3] + d3
    pos[5] = pos[4] + d4
    return ids, pos


def tangents(n):
    """T3: t1 = e_k x n / |e_k x n| with e_k the axis of smallest |n_k| (lowest k on ties),
    t2 = n x t1; (n, t1, t2) is a right-handed orthonormal frame."""
    k = int(np.argmin(np.abs(n)))
    e = np.zeros(3)
    e[k] = 1.0
    t1 = np.cross(e, n)
    t1 = t1 / np.sqrt(t1 @ t1)
    return t1, np.cross(n, t1)


def edge_geometry(mesh, topo, e):
    """Stencil ids, node positions relative to the edge midpoint, length and unit direction."""
    ids, pos = edge_stencil(mesh, topo, e)
    d = pos[3].copy()
    ell = np.sqrt(d @ d)
    return ids, pos - 0.5 * pos[3], ell, d / ell


# --------------------------------------------------------------------------- bases and weights

def taylor_basis(x, y, z, deg):
    """Complete 3D Taylor basis x^a y^b z^c / (a! b! c!), ordered by degree, then by decreasing
    a, then by decreasing b.  Degree 1 is (x, y, z) at indices 1-3; degree 2 is (xx, xy, xz, yy,
    yz, zz) at indices 4-9.  Returns p, p_x, p_y, p_z, each of length C(deg + 3, 3)."""
    out = [[], [], [], []]
    for d in range(deg + 1):
        for a in range(d, -1, -1):
            for b in range(d - a, -1, -1):
                c = d - a - b
                f = 1.0 / (factorial(a) * factorial(b) * factorial(c))
                out[0].append(f * x ** a * y ** b * z ** c)
                out[1].append(f * a * x ** (a - 1) * y ** b * z ** c if a > 0 else 0.0 * x)
                out[2].append(f * b * x ** a * y ** (b - 1) * z ** c if b > 0 else 0.0 * x)
                out[3].append(f * c * x ** a * y ** b * z ** (c - 1) if c > 0 else 0.0 * x)
    return tuple(np.array(o) for o in out)


def five_node_weights(rel5, ell, near, sv_rtol=1e-13):
    """First row of the pseudo-inverse of the 20 x 20 Hermite system on 5 nodes (Sec. 2.2 with
    T1), in coordinates scaled by the edge length: data (c, ell c_x, ell c_y, ell c_z) per node.
    Singular values are dropped smallest first while any entry of the scaled row is >= 1 (R3);
    derivative weights are unscaled and the value weights made to sum to one at the near node
    (R4).  Returns (w[20] as (v, x, y, z) per node, rank kept)."""
    X = rel5 / ell
    p, px, py, pz = taylor_basis(X[:, 0], X[:, 1], X[:, 2], 3)        # each (20, 5)
    P = np.zeros((20, 20))
    P[0::4], P[1::4], P[2::4], P[3::4] = p.T, px.T, py.T, pz.T
    U, S, Vt = np.linalg.svd(P)
    r = int(np.sum(S > sv_rtol * S[0]))
    while True:
        w = np.zeros(20)
        for i in range(r):
            w += Vt[i, 0] * U[:, i] / S[i]
        if np.max(np.abs(w)) < 1.0:
            break
        r -= 1
        if r == 0:
            raise ValueError("no singular value left")
    for k in (1, 2, 3):
        w[k::4] *= ell
    w[4 * near] += 1.0 - np.sum(w[0::4])
    return w, r


def three_node_weights(rel3, near):
    """First row of the minimum-norm pseudo-inverse of the 3 x 10 values-only system with the
    degree-2 3D Taylor basis (Eq. (3nodes_intp) with T2), unscaled coordinates relative to the
    edge midpoint, value weights made to sum to one at node `near` (R4).  Returns w[3].

    As in 2D, A has full row rank for distinct nodes and its first column is all ones, so the
    row is w = (A A^T)^-1 1; A A^T is nearly singular for short edges, so w is formed in exact
    rational arithmetic from the binary coordinates and rounded once."""
    S = max(float(c).as_integer_ratio()[1] for k in range(3) for c in rel3[k])
    rows = []
    for x, y, z in rel3:
        X, Y, Z = (int(Fraction(float(c)) * S) for c in (x, y, z))
        # 2 S^2 [1, x, y, z, x^2/2, xy, xz, y^2/2, yz, z^2/2] with x = X / S
        rows.append([2 * S * S, 2 * S * X, 2 * S * Y, 2 * S * Z, X * X, 2 * X * Y, 2 * X * Z,
                     Y * Y, 2 * Y * Z, Z * Z])
    G = [[sum(rows[i][k] * rows[j][k] for k in range(10)) for j in range(3)] for i in range(3)]

    def det3(M):
        return (M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1])
                - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0])
                + M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]))

    den = det3(G)
    b = 4 * S ** 4                 # (2 S^2 A)(2 S^2 A)^T = 4 S^4 A A^T
    num = [det3([[b if j == c else G[i][j] for j in range(3)] for i in range(3)])
           for c in range(3)]
    num[near] += den - sum(num)
    return np.array([float(Fraction(v, den)) for v in num])


# sub-stencils of the 6-node stencil, as in 2D (R2 / Alg. 1)
LEFT5, RIGHT5 = [0, 1, 2, 3, 4], [1, 2, 3, 4, 5]
LEFT_ORDER, RIGHT_ORDER = [0, 1, 2, 3, 4], [5, 4, 3, 2, 1]
LEFT3 = [[0, 1, 2], [1, 2, 3], [2, 3, 4]]
RIGHT3 = [[5, 4, 3], [4, 3, 2], [3, 2, 1]]


def edge_prep(mesh, topo, e, opts):
    """Geometry-only data of one edge: stencil, frame (n, t1, t2) and the 2 x (20 + 9) weights."""
    ids, rel, ell, n = edge_geometry(mesh, topo, e)
    t1, t2 = tangents(n)
    w5L, rL = five_node_weights(rel[LEFT5], ell, near=2, sv_rtol=opts.sv_rtol)
    w5R, rR = five_node_weights(rel[RIGHT5], ell, near=2, sv_rtol=opts.sv_rtol)
    w3 = np.zeros((2, 3, 3))
    for j in range(3):
        w3[0, j] = three_node_weights(rel[LEFT3[j]], near=LEFT3[j].index(2))
        w3[1, j] = three_node_weights(rel[RIGHT3[j]], near=RIGHT3[j].index(3))
    return {"ids": ids, "ell": ell, "n": n, "t1": t1, "t2": t2, "w5": np.stack([w5L, w5R]),
            "w3": w3, "rank": (rL, rR)}


# --------------------------------------------------------------------------- physics

def pressure(w, gamma):
    return (gamma - 1.0) * (w[4] - 0.5 * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]) / w[0])


def euler_flux(w, gamma):
    """Analytic inviscid flux vectors F, G, K of 3D Euler along x, y, z (vertex fluxes)."""
    rho, mx, my, mz, E = w
    p = pressure(w, gamma)
    u, v, ww = mx / rho, my / rho, mz / rho
    F = np.stack([mx, mx * u + p, my * u, mz * u, (E + p) * u])
    G = np.stack([my, mx * v, my * v + p, mz * v, (E + p) * v])
    K = np.stack([mz, mx * ww, my * ww, mz * ww + p, (E + p) * ww])
    return F, G, K


def normal_flux(w, n, gamma):
    F, G, K = euler_flux(w, gamma)
    return F * n[..., 0] + G * n[..., 1] + K * n[..., 2]


def roe_average(wl, wr, gamma):
    """Roe-averaged velocity (3,...), total enthalpy and sound speed of two states (5, ...)."""
    rl, rr = np.sqrt(wl[0]), np.sqrt(wr[0])
    pl, pr = pressure(wl, gamma), pressure(wr, gamma)
    s = rl + rr
    vel = np.stack([(wl[k] / rl + wr[k] / rr) / s for k in (1, 2, 3)])
    H = ((wl[4] + pl) / rl + (wr[4] + pr) / rr) / s
    c = np.sqrt((gamma - 1.0) * (H - 0.5 * np.sum(vel * vel, axis=0)))
    return vel, H, c


def eigenvectors(vel, H, c, n, t1, t2, gamma):
    """Right (columns of R) and left (rows of L = R^-1) eigenvectors of the 3D Euler flux
    Jacobian along n at the state (vel, H, c).  Waves: q_n - c, entropy, shear along t1, shear
    along t2, q_n + c.  vel (3, E); n, t1, t2 (E, 3).  Returns L, R of shape (E, 5, 5)."""
    u = vel.T                                            # (E, 3)
    qn = np.sum(u * n, -1)
    q1 = np.sum(u * t1, -1)
    q2 = np.sum(u * t2, -1)
    K = np.sum(u * u, -1)
    b1 = (gamma - 1.0) / (c * c)
    b2 = 0.5 * b1 * K
    one, zero = np.ones_like(qn), np.zeros_like(qn)
    cols = [np.concatenate([one[:, None], u - c[:, None] * n, (H - c * qn)[:, None]], 1),
            np.concatenate([one[:, None], u, (0.5 * K)[:, None]], 1),
            np.concatenate([zero[:, None], t1, q1[:, None]], 1),
            np.concatenate([zero[:, None], t2, q2[:, None]], 1),
            np.concatenate([one[:, None], u + c[:, None] * n, (H + c * qn)[:, None]], 1)]
    R = np.stack(cols, -1)
    rows = [np.concatenate([(0.5 * (b2 + qn / c))[:, None],
                            -0.5 * (b1[:, None] * u + n / c[:, None]), (0.5 * b1)[:, None]], 1),
            np.concatenate([(1.0 - b2)[:, None], b1[:, None] * u, -b1[:, None]], 1),
            np.concatenate([-q1[:, None], t1, zero[:, None]], 1),
            np.concatenate([-q2[:, None], t2, zero[:, None]], 1),
            np.concatenate([(0.5 * (b2 - qn / c))[:, None],
                            -0.5 * (b1[:, None] * u - n / c[:, None]), (0.5 * b1)[:, None]], 1)]
    L = np.stack(rows, -2)
    return L, R


def roe_flux(wl, wr, n, t1, t2, gamma, harten=0.1):
    """Roe's flux along n with Harten's entropy fix of width harten * c on all five waves
    (R9): h = (F_n(wl) + F_n(wr)) / 2 - R |Lambda| L (wr - wl) / 2.  wl, wr (5, E)."""
    vel, H, c = roe_average(wl, wr, gamma)
    L, R = eigenvectors(vel, H, c, n, t1, t2, gamma)
    qn = np.sum(vel.T * n, -1)
    lam = np.stack([qn - c, qn, qn, qn, qn + c], -1)
    delta = (harten * c)[:, None]
    a = np.abs(lam)
    a = np.where(a < delta, (lam * lam + delta * delta) / (2.0 * delta), a)
    alpha = np.einsum("eij,je->ei", L, wr - wl)
    diss = np.einsum("eij,ej->ie", R, a * alpha)
    return 0.5 * (normal_flux(wl, n, gamma) + normal_flux(wr, n, gamma)) - 0.5 * diss


# --------------------------------------------------------------------------- edge states

def edge_values(P, U, opts):
    """Left/right midpoint states of every edge by Alg. 1 in 3D: Roe average of the edge ends,
    characteristic values c = L w of the values and the three derivatives of all 6 nodes, the
    5-node value or the WENO-weighted 3-node value per component and side (sensor band of
    Eq. (2d_hweno_intp)), back-projection w = R c, positivity fallback to the end state (R16)."""
    g = opts.gamma
    W = U[:, P.stencil]                                     # (20, E, 6)
    wi, wj = W[0:5, :, 2], W[0:5, :, 3]
    vel, H, c = roe_average(wi, wj, g)
    L, R = eigenvectors(vel, H, c, P.normal, P.t1, P.t2, g)
    C = [np.einsum("eij,jek->eik", L, W[5 * k:5 * k + 5]) for k in range(4)]   # (E, 5, 6)
    out = []
    for side, (five, order, three) in enumerate([(LEFT5, LEFT_ORDER, LEFT3),
                                                 (RIGHT5, RIGHT_ORDER, RIGHT3)]):
        w5 = P.w5[:, side]
        c5 = sum(np.einsum("en,eqn->eq", w5[:, k::4], C[k][:, :, five]) for k in range(4))
        o1, o2, o3 = weno_weights(*[C[0][:, :, k] for k in order], opts.weno_eps)
        c3 = [np.einsum("en,eqn->eq", P.w3[:, side, j], C[0][:, :, three[j]]) for j in range(3)]
        weighted = o1 * c3[0] + o2 * c3[1] + o3 * c3[2]
        smooth = (o1 > opts.sens_lo) & (o1 < opts.sens_hi)
        if opts.force_branch != "sensor":
            smooth = np.full(smooth.shape, {"hermite": True, "weno": False}[opts.force_branch])
        cs = np.where(smooth, c5, weighted)
        out.append(np.einsum("eij,ej->ie", R, cs))
    wl, wr = out
    bad_l = (wl[0] <= 0) | (pressure(wl, g) <= 0)
    bad_r = (wr[0] <= 0) | (pressure(wr, g) <= 0)
    wl = np.where(bad_l[None], wi, wl)
    wr = np.where(bad_r[None], wj, wr)
    return wl, wr


# --------------------------------------------------------------------------- divergence rows

def vertex_stencil(topo, v):
    """Two-level stencil of vertex v (as in 2D, R7): every vertex within graph distance 2 (sorted
    by id) and every edge with both ends in that set (sorted by edge index)."""
    s = {v}
    for u in topo["nbrs"][v]:
        s.add(int(u))
        for w in topo["nbrs"][u]:
            s.add(int(w))
    verts = np.array(sorted(s), dtype=np.int64)
    edges = []
    for u in verts:
        for w in topo["nbrs"][u]:
            if w > u and int(w) in s:
                edges.append(topo["index"][(int(u), int(w))])
    return verts, np.array(sorted(edges), dtype=np.int64)


def div_rows(mesh, topo, v, opts):
    """Rows d_0, d_x, d_y, d_z of the two-level least-squares divergence at vertex v (Eq.
    flux_polynomials and the d-rows of Sec. 2.3, in 3D with T4).

    Unknowns (a, b, c): Taylor coefficients of f, g, k about v, degree opts.div_degree, in
    coordinates scaled by the mean incident edge length l_v.  Rows: (p^T, 0, 0), (0, p^T, 0),
    (0, 0, p^T) at each stencil vertex and (p^T n_x, p^T n_y, p^T n_z) at each stencil edge
    midpoint.  Data [f_1, g_1, k_1, ..., f_N, g_N, k_N, h_1, ..., h_M].  d_0 = a_x + b_y + c_z,
    d_x = a_xx + b_xy + c_xz, d_y = a_xy + b_yy + c_yz, d_z = a_xz + b_yz + c_zz (rows of A^+),
    unscaled by 1/l_v and 1/l_v^2."""
    verts, edges = vertex_stencil(topo, v)
    ell = float(np.mean([np.sqrt(d @ d) for d in (disp(mesh, v, u) for u in topo["nbrs"][v])]))
    xv = np.array([disp(mesh, v, u) for u in verts]) / ell
    te = topo["edges"][edges]
    xm = np.zeros((len(edges), 3))
    nm = np.zeros((len(edges), 3))
    for k, (a, b) in enumerate(te):
        d = disp(mesh, a, b)
        xm[k] = (disp(mesh, v, a) + 0.5 * d) / ell
        nm[k] = d / np.sqrt(d @ d)
    deg = opts.div_degree
    K = (deg + 1) * (deg + 2) * (deg + 3) // 6
    N, M = len(verts), len(edges)
    A = np.zeros((3 * N + M, 3 * K))
    pv = taylor_basis(xv[:, 0], xv[:, 1], xv[:, 2], deg)[0].T          # (N, K)
    pm = taylor_basis(xm[:, 0], xm[:, 1], xm[:, 2], deg)[0].T          # (M, K)
    for f in range(3):
        A[f:3 * N:3, f * K:(f + 1) * K] = pv
        A[3 * N:, f * K:(f + 1) * K] = pm * nm[:, f:f + 1]
    U, S, Vt = np.linalg.svd(A, full_matrices=False)
    if S[-1] / S[0] < opts.div_cond_min:
        raise ValueError(f"divergence stencil of vertex {v} is ill-conditioned")
    Ap = (Vt.T / S) @ U.T
    d0 = (Ap[1] + Ap[K + 2] + Ap[2 * K + 3]) / ell
    dx = (Ap[4] + Ap[K + 5] + Ap[2 * K + 6]) / ell ** 2
    dy = (Ap[5] + Ap[K + 7] + Ap[2 * K + 8]) / ell ** 2
    dz = (Ap[6] + Ap[K + 8] + Ap[2 * K + 9]) / ell ** 2
    return verts, edges, np.stack([d0, dx, dy, dz])


class Prep3:
    """Geometry-only data of the 3D residual."""


def prepare(mesh, opts=None, topo=None):
    """Divergence rows of every vertex and stencils, frames and weights of every edge."""
    opts = opts or Options3()
    topo = topo or build_topology(mesh)
    V, E = topo["V"], len(topo["edges"])
    rows, cols, vals = [[] for _ in range(4)], [[] for _ in range(4)], [[] for _ in range(4)]
    for v in range(V):
        verts, edges, d = div_rows(mesh, topo, v, opts)
        col = np.concatenate([np.stack([3 * verts, 3 * verts + 1, 3 * verts + 2], 1).ravel(),
                              3 * V + edges])
        for k in range(4):
            rows[k].append(np.full(len(col), v))
            cols[k].append(col)
            vals[k].append(d[k])
    P = Prep3()
    P.topo, P.opts = topo, opts
    P.D = [sp.csr_matrix((np.concatenate(vals[k]), (np.concatenate(rows[k]),
                                                     np.concatenate(cols[k]))), shape=(V, 3 * V + E))
           for k in range(4)]
    ep = [edge_prep(mesh, topo, e, opts) for e in range(E)]
    P.stencil = np.array([q["ids"] for q in ep], dtype=np.int64).reshape(-1, 6)
    P.normal = np.array([q["n"] for q in ep]).reshape(-1, 3)
    P.t1 = np.array([q["t1"] for q in ep]).reshape(-1, 3)
    P.t2 = np.array([q["t2"] for q in ep]).reshape(-1, 3)
    P.w5 = np.array([q["w5"] for q in ep]).reshape(-1, 2, 20)
    P.w3 = np.array([q["w3"] for q in ep]).reshape(-1, 2, 3, 3)
    P.rank = np.array([q["rank"] for q in ep]).reshape(-1, 2)
    P.ell_edge = np.array([q["ell"] for q in ep])
    return P


# --------------------------------------------------------------------------- residual and step

def residual(mesh, P, U, opts=None):
    """R(U) = -div f(w), -div f_x, -div f_y, -div f_z (Eq. HWENO in 3D): 20 x V."""
    opts = opts or P.opts
    g = opts.gamma
    V = U.shape[1]
    F, G, Kf = euler_flux(U[0:5], g)
    wl, wr = edge_values(P, U, opts)
    h = roe_flux(wl, wr, P.normal, P.t1, P.t2, g, opts.harten)        # (5, E)
    E = h.shape[1]
    R = np.zeros((20, V))
    for q in range(5):
        z = np.zeros(3 * V + E)
        z[0:3 * V:3], z[1:3 * V:3], z[2:3 * V:3] = F[q], G[q], Kf[q]
        z[3 * V:] = h[q]
        for k in range(4):
            R[5 * k + q] = -(P.D[k] @ z)
    return R


def step(mesh, P, U, dt, opts=None):
    """One SSP-RK3 step of the semi-discrete 3D system.  Returns a new array."""
    opts = opts or P.opts
    return ssp_rk3(U.copy(), dt, lambda u: residual(mesh, P, u, opts))


def cfl_dt(mesh, P, U, opts=None):
    """Time step (R12): cfl * min over vertices of l_min / (|u| + c), l_min the shortest
    incident edge."""
    opts = opts or P.opts
    g = opts.gamma
    topo = P.topo
    lmin = np.array([min(np.sqrt(d @ d) for d in (disp(mesh, v, u) for u in topo["nbrs"][v]))
                     for v in range(topo["V"])])
    w = U[0:5]
    speed = np.sqrt(np.sum((w[1:4] / w[0]) ** 2, axis=0)) + np.sqrt(g * pressure(w, g) / w[0])
    return opts.cfl * float(np.min(lmin / speed))
