"""FP64 oracle of the per-stage residual and SSP-RK3 step of the Hermite FD method.

TEST INFRASTRUCTURE ONLY (see the package docstring): the product path never calls this.

Paper map (arXiv 2109.01286):
  * Sec. 2.1 and Fig. 1: curvilinear 5-edge / 6-node stencil assembled per edge by extending it
    twice from each end along the incident edge of smallest deflection  -> `edge_stencil`.
  * Sec. 2.2, Eq. (hintp_5): 15x15 Hermite least-squares system on 5 nodes with the complete
    degree-4 Taylor basis p, p_x, p_y; solved by SVD with trial dropping of the smallest
    singular values; only the first row of P^+ is kept               -> `five_node_weights`.
  * Sec. 2.3, Eq. (3nodes_intp): 3-node 3x6 Lagrangian systems with p_3, solved by SVD (min-norm)
                                                                        -> `three_node_weights`.
  * Sec. 2.3, Eq. (HWENO): unknowns w, w_x, w_y (12 per vertex).
  * Sec. 2.3, Alg. 1 and Eq. (2d_hweno_intp): Roe average of the edge's end states, characteristic
    projection, uniform WENO5 weights as a discontinuity sensor, 5-node or weighted 3-node value,
    back-projection                                                     -> `edge_values`.
  * Sec. 2.3 (after Alg. 1): Riemann flux along the edge direction, analytic flux at vertices
                                                                        -> `roe_flux`, `euler_flux`.
  * Sec. 2.3, Eq. (flux_polynomials) and the d_0, d_x, d_y rows: two-level least-squares
    divergence of (f, g) from vertex values and edge projections       -> `div_rows`.
  * Sec. 2.3 "Computing Viscous Flux": vertex viscous flux, vertex-only LS divergence
                                                                        -> `viscous_flux`, `visc_rows`.
  * Sec. 2.3 (end): three-stage TVD (SSP) Runge-Kutta                   -> `ssp_rk3`, `step`.

State layout: U is a 12 x V float64 array; rows 0-3 are w = (rho, rho u, rho v, E), rows 4-7
are w_x and rows 8-11 are w_y.  All arithmetic is float64.  Entities are processed with numpy
array operations where each entity's arithmetic is exactly the per-entity definition.
"""
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


@dataclass
class Options:
    gamma: float = 1.4
    weno_eps: float = 1e-2        # R2: epsilon of the WENO weights (not given in the paper)
    sens_lo: float = 0.01         # Sec. 2.3: omega_1 in (0.01, 0.79) in smooth regions
    sens_hi: float = 0.79
    div_degree: int = 5           # R6: degree of the LS divergence polynomials
    visc_degree: int = 4          # R6: viscous LS degree ("fourth order")
    sv_rtol: float = 1e-13        # R3: singular values below rtol*sigma_max count as zero
    div_cond_min: float = 1e-12   # R6: fall back to degree-1 below this sigma_min/sigma_max
    visc_coef_max: float = 8.0    # R6b: viscous LS degree drops while a scaled weight exceeds this
    harten: float = 0.1           # R9: entropy-fix width delta = harten * c_roe
    flux: str = "roe"             # R9: Riemann solver, "roe" or "rusanov"
    conservative: bool = False    # value equations as median-dual finite volumes (not in the paper)
    force_branch: str = "sensor"  # testing aid: "hermite" / "weno" take that branch of Alg. 1 everywhere
    viscous: bool = False
    mu: float = 0.0
    prandtl: float = 0.72
    R_gas: float = 1.0
    cfl: float = 0.3              # R12


# --------------------------------------------------------------------------- topology (Sec. 2.1)

def build_topology(mesh):
    """Unique undirected edges of the triangulation, oriented tail < head (input ids, R8) and
    sorted lexicographically; sorted neighbour lists; edge lookup."""
    tri = np.asarray(mesh["tri"], dtype=np.int64)
    V = len(mesh["x"])
    e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]])
    e = np.sort(e, axis=1)
    e = np.unique(e, axis=0)
    nbrs = [[] for _ in range(V)]
    for a, b in e:
        nbrs[a].append(b)
        nbrs[b].append(a)
    nbrs = [np.array(sorted(n), dtype=np.int64) for n in nbrs]
    index = {(int(a), int(b)): k for k, (a, b) in enumerate(e)}
    ghost = np.zeros(V, bool)
    ghost[np.asarray(mesh["ghost_ids"], dtype=np.int64)] = True
    return {"edges": e, "nbrs": nbrs, "index": index, "V": V, "ghost": ghost}


def disp(mesh, a, b):
    """Vector from vertex a to vertex b; minimum image on periodic axes."""
    dx = mesh["x"][b] - mesh["x"][a]
    dy = mesh["y"][b] - mesh["y"][a]
    if mesh["periodic_x"]:
        dx = dx - mesh["Lx"] * np.round(dx / mesh["Lx"])
    if mesh["periodic_y"]:
        dy = dy - mesh["Ly"] * np.round(dy / mesh["Ly"])
    return np.array([dx, dy])


def _extend(mesh, topo, cur, t, used):
    """One extension step (Sec. 2.1): among the neighbours of `cur` not yet in the stencil,
    pick the one whose edge deviates least from the travel direction t (largest cosine).
    Ties (cosines within 1e-12) go to the lower vertex id (R11): candidates are scanned in
    ascending id order and replace the current best only when larger by more than 1e-12."""
    best, best_cos, best_d = -1, -np.inf, None
    tn = np.sqrt(t[0] * t[0] + t[1] * t[1])
    for c in topo["nbrs"][cur]:
        if c in used:
            continue
        d = disp(mesh, cur, c)
        cs = (t[0] * d[0] + t[1] * d[1]) / (tn * np.sqrt(d[0] * d[0] + d[1] * d[1]))
        if cs > best_cos + 1e-12:
            best, best_cos, best_d = int(c), cs, d
    if best < 0:
        raise ValueError(f"stencil cannot be extended from vertex {cur}")
    return best, best_d


def edge_stencil(mesh, topo, e):
    """6-node curvilinear stencil [i-2, i-1, i, i+1, i+2, i+3] of edge e = (i, i+1) (Sec. 2.1,
    Fig. 1 and Fig. 4): two extensions backwards from the tail, then two forwards from the head.
    Returns the node ids and their positions relative to the tail (accumulated along the path)."""
    a, b = (int(v) for v in topo["edges"][e])
    used = {a, b}
    dab = disp(mesh, a, b)
    # backwards from the tail: travel direction b -> a
    b1, d1 = _extend(mesh, topo, a, -dab, used)
    used.add(b1)
    b2, d2 = _extend(mesh, topo, b1, d1, used)
    used.add(b2)
    f1, d3 = _extend(mesh, topo, b, dab, used)
    used.add(f1)
    f2, d4 = _extend(mesh, topo, f1, d3, used)
    ids = np.array([b2, b1, a, b, f1, f2], dtype=np.int64)
    pos = np.zeros((6, 2))
    pos[1] = d1
    pos[0] = pos[1] + d2
    pos[3] = dab
    pos[4] = pos[3] + d3
    pos[5] = pos[4] + d4
    return ids, pos


def edge_geometry(mesh, topo, e):
    """Stencil ids, node positions relative to the edge midpoint, length and unit direction."""
    ids, pos = edge_stencil(mesh, topo, e)
    d = pos[3].copy()
    ell = np.sqrt(d[0] * d[0] + d[1] * d[1])
    rel = pos - 0.5 * pos[3]
    return ids, rel, ell, d / ell


# --------------------------------------------------------------------------- bases (Sec. 2.2)

def taylor_basis(x, y, deg):
    """Complete Taylor basis of the given degree, ordered by degree then by decreasing power of
    x: x^a y^b / (a! b!).  Degree 4 gives the 15-term p of Sec. 2.2; degree 2 gives p_3.
    Returns p, p_x, p_y (each of length (deg+1)(deg+2)/2)."""
    from math import factorial
    p, px, py = [], [], []
    for d in range(deg + 1):
        for b in range(d + 1):
            a = d - b
            c = 1.0 / (factorial(a) * factorial(b))
            p.append(c * x ** a * y ** b)
            px.append(c * a * x ** (a - 1) * y ** b if a > 0 else 0.0 * x)
            py.append(c * b * x ** a * y ** (b - 1) if b > 0 else 0.0 * x)
    return np.array(p), np.array(px), np.array(py)


# --------------------------------------------------------------------------- weights

def five_node_weights(rel5, ell, near, sv_rtol=1e-13):
    """First row of the pseudo-inverse of the 15x15 Hermite system P (Eq. hintp_5, Sec. 2.2).

    rel5: (5, 2) node positions relative to the edge midpoint; near: index (0..4) of the edge
    end on this side.  The system is built in coordinates scaled by the edge length ell (R3), so
    the data are (c, ell c_x, ell c_y).  Singular values are dropped smallest first while any
    entry of the stored (scaled) row is >= 1 in magnitude (R3, the weight-row reading of the
    paper's dropping rule).  Derivative weights are then unscaled (times ell) and the value
    weights are made to sum to one by adjusting the weight of the near end node (R4).
    Returns (w[15] as (v, x, y) per node, rank kept)."""
    X = rel5 / ell
    p, px, py = taylor_basis(X[:, 0], X[:, 1], 4)              # each (15, 5)
    P = np.zeros((15, 15))
    P[0::3], P[1::3], P[2::3] = p.T, px.T, py.T
    U, S, Vt = np.linalg.svd(P)
    r = int(np.sum(S > sv_rtol * S[0]))
    while True:
        w = np.zeros(15)
        for i in range(r):
            w += Vt[i, 0] * U[:, i] / S[i]
        if np.max(np.abs(w)) < 1.0:
            break
        r -= 1
        if r == 0:
            raise ValueError("no singular value left")
    w[1::3] *= ell
    w[2::3] *= ell
    w[3 * near] += 1.0 - np.sum(w[0::3])
    return w, r


def three_node_weights(rel3, near):
    """First row of the min-norm pseudo-inverse of the 3x6 Lagrangian system of Eq. (3nodes_intp)
    with p_3 = [1, x, y, x^2/2, xy, y^2/2], in unscaled coordinates relative to the edge midpoint
    (R5), then the value weights made to sum to one at node `near` (R4).  Returns w[3].

    Three distinct nodes always give A full row rank, so A^+ = A^T (A A^T)^-1 and, because the
    first column of A is all ones, its first row is w = (A A^T)^-1 1.  In unscaled coordinates
    A A^T = 1 1^T + O(h^2) is nearly singular for small h, so w is computed in exact rational
    arithmetic from the (exact) binary coordinates and rounded once at the end."""
    # exact integers: with S a power of two making every coordinate an integer, 2 S^2 A is an
    # integer matrix; G' = (2 S^2 A)(2 S^2 A)^T = 4 S^4 A A^T and G' w = 4 S^4 1.
    S = max(max(float(c).as_integer_ratio()[1] for c in rel3[k]) for k in range(3))
    A = []
    for x, y in rel3:
        X = float(x).as_integer_ratio()
        Y = float(y).as_integer_ratio()
        X = X[0] * (S // X[1])
        Y = Y[0] * (S // Y[1])
        A.append([2 * S * S, 2 * S * X, 2 * S * Y, X * X, 2 * X * Y, Y * Y])
    G = [[sum(A[i][k] * A[j][k] for k in range(6)) for j in range(3)] for i in range(3)]

    def det3(M):
        return (M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1])
                - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0])
                + M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]))

    den = det3(G)
    b = 4 * S ** 4
    num = [det3([[b if j == c else G[i][j] for j in range(3)] for i in range(3)])
           for c in range(3)]                # Cramer's rule: w_c = num_c / den
    num[near] += den - sum(num)              # R4, exactly
    from fractions import Fraction
    return np.array([float(Fraction(v, den)) for v in num])


# sub-stencils (indices into the 6-node stencil) and near-end positions, R2/Alg. 1:
# left side uses nodes 0..4 (i-2..i+2), right side mirrors: 5,4,3,2,1 (i+3..i-1)
LEFT5, RIGHT5 = [0, 1, 2, 3, 4], [1, 2, 3, 4, 5]
LEFT_ORDER, RIGHT_ORDER = [0, 1, 2, 3, 4], [5, 4, 3, 2, 1]
def dual_faces(mesh, topo):
    """Median-dual geometry of the conservative variant (the paper names conservation as open,
    Sec. 4): for every edge (a, b), tail a < b, the dual-face area vector S_e = sum over the
    triangles holding the edge of the segment from the edge midpoint to the triangle centroid,
    turned by 90 degrees and oriented so that S_e . (x_b - x_a) > 0; and the median-dual cell
    areas (R17).  Cached in topo."""
    if "dual_S" in topo:
        return topo["dual_S"], topo["dual_A"]
    S = np.zeros((len(topo["edges"]), 2))
    for t in np.asarray(mesh["tri"], dtype=np.int64):
        x = [np.zeros(2), disp(mesh, t[0], t[1]), disp(mesh, t[0], t[2])]
        g = (x[0] + x[1] + x[2]) / 3.0
        for i, j in ((0, 1), (1, 2), (2, 0)):
            a, b = (i, j) if t[i] < t[j] else (j, i)
            seg = g - 0.5 * (x[i] + x[j])
            nrm = np.array([seg[1], -seg[0]])
            if nrm @ (x[b] - x[a]) < 0:
                nrm = -nrm
            S[topo["index"][(int(t[a]), int(t[b]))]] += nrm
    topo["dual_S"], topo["dual_A"] = S, vertex_areas(mesh)
    return topo["dual_S"], topo["dual_A"]


LEFT3 = [[0, 1, 2], [1, 2, 3], [2, 3, 4]]
RIGHT3 = [[5, 4, 3], [4, 3, 2], [3, 2, 1]]


def edge_prep(mesh, topo, e, opts):
    """All geometry-only data of one edge: stencil, direction and the 48 interpolation weights."""
    ids, rel, ell, n = edge_geometry(mesh, topo, e)
    if opts.conservative:            # projection and Riemann flux along the dual-face normal
        S = dual_faces(mesh, topo)[0][e]
        n = S / np.sqrt(S[0] * S[0] + S[1] * S[1])
    w5L, rL = five_node_weights(rel[LEFT5], ell, near=2, sv_rtol=opts.sv_rtol)
    w5R, rR = five_node_weights(rel[RIGHT5], ell, near=2, sv_rtol=opts.sv_rtol)
    w3 = np.zeros((2, 3, 3))
    for j in range(3):
        w3[0, j] = three_node_weights(rel[LEFT3[j]], near=LEFT3[j].index(2))
        w3[1, j] = three_node_weights(rel[RIGHT3[j]], near=RIGHT3[j].index(3))
    return {"ids": ids, "rel": rel, "ell": ell, "n": n, "w5": np.stack([w5L, w5R]),
            "w3": w3, "rank": (rL, rR)}


# --------------------------------------------------------------------------- divergence rows

def vertex_stencil(topo, v):
    """Two-level stencil of vertex v (Fig. 6, R7): every vertex within graph distance 2 (sorted
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


def _vertex_scale(mesh, topo, v):
    return float(np.mean([np.linalg.norm(disp(mesh, v, u)) for u in topo["nbrs"][v]]))


def div_rows(mesh, topo, v, opts):
    """Rows d_0, d_x, d_y of the two-level least-squares divergence at vertex v (Eq.
    flux_polynomials and the d-row definitions, Sec. 2.3).

    Unknowns (a, b): Taylor coefficients of f and g about v, degree opts.div_degree (R6), in
    coordinates scaled by the mean incident edge length l_v.  Rows: (p^T, 0) and (0, p^T) at each
    stencil vertex, (p^T n_x, p^T n_y) at each stencil edge midpoint.  The data vector is
    [f_1, g_1, ..., f_N, g_N, h_1, ..., h_M].  d_0 = row(a_2)+row(b_3) (divergence of f),
    d_x = row(a_4)+row(b_5) (divergence of f_x), d_y = row(a_5)+row(b_6) (divergence of f_y),
    unscaled by 1/l_v and 1/l_v^2.  If sigma_min/sigma_max < div_cond_min the degree drops by one."""
    verts, edges = vertex_stencil(topo, v)
    ell = _vertex_scale(mesh, topo, v)
    xv = np.array([disp(mesh, v, u) for u in verts]) / ell
    te = topo["edges"][edges]
    xm = np.zeros((len(edges), 2))
    nm = np.zeros((len(edges), 2))
    if opts.conservative:
        Sd, Ad = dual_faces(mesh, topo)
    for k, (a, b) in enumerate(te):
        d = disp(mesh, a, b)
        xm[k] = (disp(mesh, v, a) + 0.5 * d) / ell
        if opts.conservative:        # h is the flux along the dual-face normal
            d = Sd[edges[k]]
        nm[k] = d / np.sqrt(d[0] * d[0] + d[1] * d[1])
    deg = opts.div_degree
    while True:
        K = (deg + 1) * (deg + 2) // 2
        N, M = len(verts), len(edges)
        A = np.zeros((2 * N + M, 2 * K))
        pv = taylor_basis(xv[:, 0], xv[:, 1], deg)[0].T          # (N, K)
        pm = taylor_basis(xm[:, 0], xm[:, 1], deg)[0].T          # (M, K)
        A[0:2 * N:2, :K] = pv
        A[1:2 * N:2, K:] = pv
        A[2 * N:, :K] = pm * nm[:, 0:1]
        A[2 * N:, K:] = pm * nm[:, 1:2]
        U, S, Vt = np.linalg.svd(A, full_matrices=False)
        if S[-1] / S[0] >= opts.div_cond_min or deg <= 2:
            break
        deg -= 1
    Ap = (Vt.T / S) @ U.T
    d0 = (Ap[1] + Ap[K + 2]) / ell
    dx = (Ap[3] + Ap[K + 4]) / ell ** 2
    dy = (Ap[4] + Ap[K + 5]) / ell ** 2
    if opts.conservative:
        # divergence of the value flux as the median-dual cell's boundary integral: the flux
        # through face e is |S_e| h_e, leaving the tail's cell and entering the head's
        d0 = np.zeros_like(d0)
        N = len(verts)
        for k, (a, b) in enumerate(te):
            if v in (a, b):
                sgn = 1.0 if v == a else -1.0
                d0[2 * N + k] = sgn * np.linalg.norm(Sd[edges[k]]) / Ad[v]
    return verts, edges, np.stack([d0, dx, dy]), deg


def visc_rows(mesh, topo, v, opts):
    """Vertex-only least-squares divergence rows of the viscous flux (Sec. 2.3, "Computing
    Viscous Flux"): f_vis and g_vis are fitted separately on the two-level vertex set with the
    Taylor basis of degree opts.visc_degree, in coordinates scaled by l_v.  Rows over the
    interleaved data [f_1, g_1, ...]: e_0 (divergence), e_x, e_y (divergence of the x/y
    derivative fluxes).  With only about as many stencil vertices as basis terms some vertex
    sets are nearly unisolvent and the fitted weights explode; the degree then drops by one
    while any scaled weight of the rows used (first and second derivatives) exceeds
    opts.visc_coef_max (R6b), down to degree 2."""
    verts, _ = vertex_stencil(topo, v)
    ell = _vertex_scale(mesh, topo, v)
    xv = np.array([disp(mesh, v, u) for u in verts]) / ell
    deg = opts.visc_degree
    while True:
        B = taylor_basis(xv[:, 0], xv[:, 1], deg)[0].T
        Q = np.linalg.pinv(B)
        if np.abs(Q[1:6]).max() <= opts.visc_coef_max or deg <= 2:
            break
        deg -= 1
    N = len(verts)
    rows = np.zeros((3, 2 * N))
    rows[0, 0::2], rows[0, 1::2] = Q[1] / ell, Q[2] / ell
    rows[1, 0::2], rows[1, 1::2] = Q[3] / ell ** 2, Q[4] / ell ** 2
    rows[2, 0::2], rows[2, 1::2] = Q[4] / ell ** 2, Q[5] / ell ** 2
    return verts, rows, deg


class Prep:
    """Geometry-only data for the residual at a set of active vertices."""


def prepare(mesh, opts=None, active=None, topo=None):
    """Precompute everything geometry-only: divergence rows at the active vertices (default: all
    non-ghost vertices) and edge stencils/weights of every edge those rows reference."""
    opts = opts or Options()
    topo = topo or build_topology(mesh)
    V = topo["V"]
    E = len(topo["edges"])
    if active is None:
        active = np.nonzero(~topo["ghost"])[0]
    active = np.asarray(active, dtype=np.int64)
    rows, cols, vals = [[], [], []], [[], [], []], [[], [], []]
    need = set()
    degs, vdegs = [], []
    vrows, vcols, vvals = [[], [], []], [[], [], []], [[], [], []]
    for r, v in enumerate(active):
        verts, edges, d, deg = div_rows(mesh, topo, int(v), opts)
        degs.append(deg)
        need.update(int(e) for e in edges)
        col = np.concatenate([np.stack([2 * verts, 2 * verts + 1], 1).ravel(), 2 * V + edges])
        for k in range(3):
            rows[k].append(np.full(len(col), r))
            cols[k].append(col)
            vals[k].append(d[k])
        if opts.viscous:
            vv, vr, vdeg = visc_rows(mesh, topo, int(v), opts)
            vdegs.append(vdeg)
            vcol = np.stack([2 * vv, 2 * vv + 1], 1).ravel()
            for k in range(3):
                vrows[k].append(np.full(len(vcol), r))
                vcols[k].append(vcol)
                vvals[k].append(vr[k])
    P = Prep()
    P.topo, P.active, P.opts = topo, active, opts
    P.div_degree = np.array(degs)
    P.visc_degree = np.array(vdegs, dtype=np.int64)
    shape = (len(active), 2 * V + E)
    P.D = [sp.csr_matrix((np.concatenate(vals[k]), (np.concatenate(rows[k]),
                                                     np.concatenate(cols[k]))), shape=shape)
           for k in range(3)]
    if opts.viscous:
        P.Dv = [sp.csr_matrix((np.concatenate(vvals[k]), (np.concatenate(vrows[k]),
                                                           np.concatenate(vcols[k]))),
                              shape=(len(active), 2 * V)) for k in range(3)]
    P.edges = np.array(sorted(need), dtype=np.int64)
    ep = [edge_prep(mesh, topo, int(e), opts) for e in P.edges]
    P.stencil = np.array([q["ids"] for q in ep], dtype=np.int64).reshape(-1, 6)
    P.normal = np.array([q["n"] for q in ep]).reshape(-1, 2)
    P.w5 = np.array([q["w5"] for q in ep]).reshape(-1, 2, 15)
    P.w3 = np.array([q["w3"] for q in ep]).reshape(-1, 2, 3, 3)
    P.rank = np.array([q["rank"] for q in ep]).reshape(-1, 2)
    P.ell_edge = np.array([q["ell"] for q in ep])
    return P


# --------------------------------------------------------------------------- physics

def pressure(w, gamma):
    return (gamma - 1.0) * (w[3] - 0.5 * (w[1] * w[1] + w[2] * w[2]) / w[0])


def euler_flux(w, gamma):
    """Analytic inviscid flux vectors F(w), G(w) of 2D Euler (Sec. 2.3, vertex fluxes)."""
    rho, m, n, E = w
    p = pressure(w, gamma)
    u, v = m / rho, n / rho
    F = np.stack([m, m * u + p, n * u, (E + p) * u])
    G = np.stack([n, m * v, n * v + p, (E + p) * v])
    return F, G


def viscous_flux(U, opts):
    """Viscous flux at vertices from w, w_x, w_y (Sec. 2.3, "Computing Viscous Flux"; model R13:
    constant mu, Stokes hypothesis, Fourier heat flux with kappa = mu c_p / Pr, p = rho R T)."""
    g, mu = opts.gamma, opts.mu
    rho, m, n, E = U[0:4]
    wx, wy = U[4:8], U[8:12]
    u, v = m / rho, n / rho
    ux, vx = (wx[1] - u * wx[0]) / rho, (wx[2] - v * wx[0]) / rho
    uy, vy = (wy[1] - u * wy[0]) / rho, (wy[2] - v * wy[0]) / rho
    q2 = u * u + v * v
    p = (g - 1.0) * (E - 0.5 * rho * q2)
    px = (g - 1.0) * (wx[3] - 0.5 * wx[0] * q2 - rho * (u * ux + v * vx))
    py = (g - 1.0) * (wy[3] - 0.5 * wy[0] * q2 - rho * (u * uy + v * vy))
    R = opts.R_gas
    Tx = (px / rho - p * wx[0] / (rho * rho)) / R
    Ty = (py / rho - p * wy[0] / (rho * rho)) / R
    kappa = mu * (g * R / (g - 1.0)) / opts.prandtl
    txx = mu * (4.0 / 3.0 * ux - 2.0 / 3.0 * vy)
    tyy = mu * (4.0 / 3.0 * vy - 2.0 / 3.0 * ux)
    txy = mu * (uy + vx)
    z = np.zeros_like(rho)
    Fv = np.stack([z, txx, txy, u * txx + v * txy + kappa * Tx])
    Gv = np.stack([z, txy, tyy, u * txy + v * tyy + kappa * Ty])
    return Fv, Gv


def roe_average(wl, wr, gamma):
    """Roe-averaged velocity, total enthalpy and sound speed of two states (Alg. 1, first step;
    also the Riemann flux, R9).  Arrays of shape (4, ...)."""
    rl, rr = np.sqrt(wl[0]), np.sqrt(wr[0])
    pl, pr = pressure(wl, gamma), pressure(wr, gamma)
    s = rl + rr
    u = (wl[1] / rl + wr[1] / rr) / s
    v = (wl[2] / rl + wr[2] / rr) / s
    H = ((wl[3] + pl) / rl + (wr[3] + pr) / rr) / s
    c = np.sqrt((gamma - 1.0) * (H - 0.5 * (u * u + v * v)))
    return u, v, H, c


def eigenvectors(u, v, H, c, nx, ny, gamma):
    """Right (columns of R) and left (rows of L = R^-1) eigenvectors of the 2D Euler flux
    Jacobian along direction n (Alg. 1, second step; R10).  Waves: q_n - c, entropy, shear,
    q_n + c.  Returns L, R with shape (..., 4, 4)."""
    qn = u * nx + v * ny
    qt = -u * ny + v * nx
    K = u * u + v * v
    b1 = (gamma - 1.0) / (c * c)
    b2 = 0.5 * b1 * K
    one = np.ones_like(u)
    zero = np.zeros_like(u)
    R = np.stack([
        np.stack([one, one, zero, one], -1),
        np.stack([u - c * nx, u, -ny * one, u + c * nx], -1),
        np.stack([v - c * ny, v, nx * one, v + c * ny], -1),
        np.stack([H - c * qn, 0.5 * K, qt, H + c * qn], -1)], -2)
    L = np.stack([
        np.stack([0.5 * (b2 + qn / c), -0.5 * (b1 * u + nx / c), -0.5 * (b1 * v + ny / c), 0.5 * b1], -1),
        np.stack([1.0 - b2, b1 * u, b1 * v, -b1 * one], -1),
        np.stack([-qt, -ny * one, nx * one, zero], -1),
        np.stack([0.5 * (b2 - qn / c), -0.5 * (b1 * u - nx / c), -0.5 * (b1 * v - ny / c), 0.5 * b1], -1)], -2)
    return L, R


def weno_weights(u0, u1, u2, u3, u4, eps):
    """Nonlinear weights of uniform-grid WENO5 interpolation (Sec. 2.1 and Sec. 2.3, R2):
    Jiang-Shu smoothness indicators of the three 3-point sub-stencils, linear weights
    (1/16, 10/16, 5/16) of the WCNS-E5 interpolation, alpha = d/(eps+beta)^2, omega = alpha/sum."""
    b1 = 13.0 / 12.0 * (u0 - 2.0 * u1 + u2) ** 2 + 0.25 * (u0 - 4.0 * u1 + 3.0 * u2) ** 2
    b2 = 13.0 / 12.0 * (u1 - 2.0 * u2 + u3) ** 2 + 0.25 * (u1 - u3) ** 2
    b3 = 13.0 / 12.0 * (u2 - 2.0 * u3 + u4) ** 2 + 0.25 * (3.0 * u2 - 4.0 * u3 + u4) ** 2
    a1 = (1.0 / 16.0) / (eps + b1) ** 2
    a2 = (10.0 / 16.0) / (eps + b2) ** 2
    a3 = (5.0 / 16.0) / (eps + b3) ** 2
    s = a1 + a2 + a3
    return a1 / s, a2 / s, a3 / s


def normal_flux(w, nx, ny, gamma):
    F, G = euler_flux(w, gamma)
    return F * nx + G * ny


def roe_flux(wl, wr, nx, ny, gamma, harten=0.1):
    """Numerical flux h along direction n at the edge midpoint (Sec. 2.3, after Alg. 1; solver
    not named in the paper, R9): Roe's flux with Harten's entropy fix of width harten*c on all
    four waves.  wl, wr have shape (4, ...)."""
    u, v, H, c = roe_average(wl, wr, gamma)
    L, R = eigenvectors(u, v, H, c, nx, ny, gamma)
    qn = u * nx + v * ny
    lam = np.stack([qn - c, qn, qn, qn + c], -1)
    delta = harten * c
    a = np.where(np.real(lam) < 0, -lam, lam)          # |lambda| (real-part sign: complex-step safe)
    a = np.where(np.real(a) < np.real(delta[..., None]),
                 (lam * lam + delta[..., None] ** 2) / (2.0 * delta[..., None]), a)
    dw = np.moveaxis(wr - wl, 0, -1)
    alpha = np.einsum("...ij,...j->...i", L, dw)
    diss = np.einsum("...ij,...j->...i", R, a * alpha)
    return 0.5 * (normal_flux(wl, nx, ny, gamma) + normal_flux(wr, nx, ny, gamma)) \
        - 0.5 * np.moveaxis(diss, -1, 0)


def rusanov_flux(wl, wr, nx, ny, gamma):
    """Rusanov's (local Lax-Friedrichs) flux along n, the alternative Riemann solver of R9:
    h = (F_n(wl) + F_n(wr)) / 2 - s (wr - wl) / 2, with s the larger of |u_n| + c over the
    two states.  Complex-step safe (comparisons on real parts)."""
    def speed(w):
        un = (w[1] * nx + w[2] * ny) / w[0]
        c = np.sqrt(gamma * pressure(w, gamma) / w[0])
        return np.where(np.real(un) < 0, -un, un) + c
    sl, sr = speed(wl), speed(wr)
    s = np.where(np.real(sl) >= np.real(sr), sl, sr)
    return 0.5 * (normal_flux(wl, nx, ny, gamma) + normal_flux(wr, nx, ny, gamma)) \
        - 0.5 * s * (wr - wl)


def riemann_flux(wl, wr, nx, ny, opts):
    """The edge's numerical flux h (Sec. 2.3, after Alg. 1) with the solver of opts.flux."""
    if opts.flux == "rusanov":
        return rusanov_flux(wl, wr, nx, ny, opts.gamma)
    if opts.flux != "roe":
        raise ValueError(f"unknown Riemann solver {opts.flux!r}")
    return roe_flux(wl, wr, nx, ny, opts.gamma, opts.harten)


# --------------------------------------------------------------------------- residual

def ghost_fill(mesh, U):
    """Transmissive ghost refresh (R14): copy the donor's 12 values, zero the derivative normal
    to the boundary (flag bit 0: x, bit 1: y).  Ghosts with donor -1 are fixed (R22: wall bands
    holding given values) and keep theirs.  In place; returns U."""
    g = np.asarray(mesh["ghost_ids"], dtype=np.int64)
    d = np.asarray(mesh["ghost_donor"], dtype=np.int64)
    f = np.asarray(mesh["ghost_flags"])
    keep = d >= 0
    g, d, f = g[keep], d[keep], f[keep]
    if len(g) == 0:
        return U
    U[:, g] = U[:, d]
    U[4:8, g[(f & 1) != 0]] = 0.0
    U[8:12, g[(f & 2) != 0]] = 0.0
    return U


def edge_values(P, U, opts, diag=None):
    """Left/right midpoint states of every needed edge by Alg. 1 (Sec. 2.3) with the branch
    sense of Eq. (2d_hweno_intp) (R1: 5-node value when sens_lo < omega_1 < sens_hi, else the
    omega-weighted 3-node values), per characteristic component and side; then R16 positivity."""
    return edge_values_from_stencil(P, U[:, P.stencil], opts, diag)


def edge_values_from_stencil(P, W, opts, diag=None):
    """edge_values on the gathered stencil states W (12, Ee, 6); works on complex input
    (branch and positivity decisions use real parts) for complex-step derivatives."""
    g = opts.gamma
    wi, wj = W[0:4, :, 2], W[0:4, :, 3]
    u, v, H, c = roe_average(wi, wj, g)
    L, R = eigenvectors(u, v, H, c, P.normal[:, 0], P.normal[:, 1], g)
    # characteristic values c = L w for the values and both derivatives of all 6 nodes
    C = [np.einsum("eij,jek->eik", L, W[4 * k:4 * k + 4]) for k in range(3)]   # (Ee, 4, 6)
    out = []
    for side, (five, order, three) in enumerate([(LEFT5, LEFT_ORDER, LEFT3),
                                                 (RIGHT5, RIGHT_ORDER, RIGHT3)]):
        w5 = P.w5[:, side]
        c5 = (np.einsum("en,eqn->eq", w5[:, 0::3], C[0][:, :, five])
              + np.einsum("en,eqn->eq", w5[:, 1::3], C[1][:, :, five])
              + np.einsum("en,eqn->eq", w5[:, 2::3], C[2][:, :, five]))
        o1, o2, o3 = weno_weights(*[C[0][:, :, k] for k in order], opts.weno_eps)
        c3 = [np.einsum("en,eqn->eq", P.w3[:, side, j], C[0][:, :, three[j]]) for j in range(3)]
        weighted = o1 * c3[0] + o2 * c3[1] + o3 * c3[2]
        smooth = (np.real(o1) > opts.sens_lo) & (np.real(o1) < opts.sens_hi)
        if opts.force_branch != "sensor":
            smooth = np.full(smooth.shape, {"hermite": True, "weno": False}[opts.force_branch])
        cs = np.where(smooth, c5, weighted)
        ws = np.einsum("eij,ej->ie", R, cs)          # back-projection w = R c
        if diag is not None:
            diag.setdefault("omega1", []).append(o1)
            diag.setdefault("smooth", []).append(smooth)
        out.append(ws)
    wl, wr = out
    bad_l = (np.real(wl[0]) <= 0) | (np.real(pressure(wl, g)) <= 0)
    bad_r = (np.real(wr[0]) <= 0) | (np.real(pressure(wr, g)) <= 0)
    wl = np.where(bad_l[None], wi, wl)
    wr = np.where(bad_r[None], wj, wr)
    if diag is not None:
        diag["positivity_fallbacks"] = int(bad_l.sum() + bad_r.sum())
    return wl, wr


def edge_flux_from_stencil(P, W, opts):
    """Numerical flux h (4, Ee) of every needed edge from its gathered stencil states."""
    wl, wr = edge_values_from_stencil(P, W, opts)
    return riemann_flux(wl, wr, P.normal[:, 0], P.normal[:, 1], opts)


def residual(mesh, P, U, opts=None, diag=None):
    """R(U) = -div f (w), -div f_x, -div f_y (+ viscous divergences) at the active vertices
    (Eq. HWENO).  Ghost rows of U are refreshed first (in place).  Returns a 12 x V array that
    is zero at non-active vertices."""
    opts = opts or P.opts
    g = opts.gamma
    U = ghost_fill(mesh, U)
    V = U.shape[1]
    F, G = euler_flux(U[0:4], g)
    wl, wr = edge_values(P, U, opts, diag)
    h = riemann_flux(wl, wr, P.normal[:, 0], P.normal[:, 1], opts)   # (4, Ee)
    E = len(P.topo["edges"])
    Rm = np.zeros((12, V), dtype=U.dtype)
    for q in range(4):
        z = np.zeros(2 * V + E, dtype=U.dtype)
        z[0:2 * V:2] = F[q]
        z[1:2 * V:2] = G[q]
        z[2 * V + P.edges] = h[q]
        for k in range(3):
            Rm[4 * k + q, P.active] = -(P.D[k] @ z)
    if opts.viscous:
        Fv, Gv = viscous_flux(U, opts)
        for q in range(4):
            z = np.zeros(2 * V, dtype=U.dtype)
            z[0::2] = Fv[q]
            z[1::2] = Gv[q]
            for k in range(3):
                Rm[4 * k + q, P.active] += P.Dv[k] @ z
    if diag is not None:
        diag["h"] = h
    return Rm


def ssp_rk3(u, dt, rhs):
    """Three-stage TVD (SSP) Runge-Kutta of Shu and Osher (Sec. 2.3, end):
    u1 = u + dt L(u); u2 = 3/4 u + 1/4 (u1 + dt L(u1)); u+ = 1/3 u + 2/3 (u2 + dt L(u2))."""
    u1 = u + dt * rhs(u)
    u2 = 0.75 * u + 0.25 * (u1 + dt * rhs(u1))
    return u / 3.0 + 2.0 / 3.0 * (u2 + dt * rhs(u2))


def step(mesh, P, U, dt, opts=None):
    """One SSP-RK3 step of the semi-discrete system; only active vertices are advanced and the
    ghost rows of the result are refreshed (R14).  Returns a new array."""
    opts = opts or P.opts
    act = P.active

    def rhs(u):
        return residual(mesh, P, u, opts)

    u = ghost_fill(mesh, U.copy())
    out = ssp_rk3(u, dt, rhs)
    res = u.copy()
    res[:, act] = out[:, act]
    return ghost_fill(mesh, res)


def cfl_dt(mesh, P, U, opts=None):
    """Time step (R12): cfl * min over active vertices of l_min / (|u| + c), l_min the shortest
    incident edge."""
    opts = opts or P.opts
    g = opts.gamma
    topo = P.topo
    act = P.active
    lmin = np.array([min(np.linalg.norm(disp(mesh, v, u)) for u in topo["nbrs"][v]) for v in act])
    w = U[0:4, act]
    p = pressure(w, g)
    speed = np.sqrt((w[1] / w[0]) ** 2 + (w[2] / w[0]) ** 2) + np.sqrt(g * p / w[0])
    return opts.cfl * float(np.min(lmin / speed))


def vertex_areas(mesh):
    """Median-dual vertex areas (R17): one third of the area of every incident triangle."""
    tri = np.asarray(mesh["tri"], dtype=np.int64)
    A = np.zeros(len(mesh["x"]))
    for t in tri:
        d1 = disp(mesh, t[0], t[1])
        d2 = disp(mesh, t[0], t[2])
        area = 0.5 * (d1[0] * d2[1] - d1[1] * d2[0])
        A[t] += area / 3.0
    return A
