"""Alternative readings of the paper's open points, and the linear stability sweep over them.

TEST INFRASTRUCTURE ONLY, like the rest of `oracle/`: the product path never imports it.

The method as read (`hfd_oracle`) is linearly unstable about a uniform state.  This module
re-derives the residual under each reading the paper's text leaves open and measures, for each:

  * the growth rate max Re(lambda) * h / (|u| + c) of the residual's Jacobian about a uniform
    flow on small jittered periodic meshes (complex-step linearisation, exact to rounding), and
    the largest amplification |G(lambda dt)| of one SSP-RK3 step at CFL 0.3;
  * the Monte Carlo order of the 5-node interpolation (Sec. 2.2, Fig. 5) under its rule;
  * the truncation orders of all 12 residual rows on the exact isentropic vortex (Sec. 3.1).

Readings (each names the passage it reads):
  sv_rule   "row": R3, drop singular values while an entry of the stored first row of the
            scaled P^+ is >= 1 (the weights must be data independent, Sec. 2.2);
            "all": drop while any entry of the whole scaled P^+ is >= 1 -- "each component of
            k" for every unit datum (Sec. 2.2).
  div_degree  degree of the least-squares flux polynomials, "up to specified degree" (Sec. 2.3).
  deriv     how the derivative equations of Eq. (HWENO) get div f_x and div f_y:
            "fit2": the second derivatives a_4+b_5, a_5+b_6 of the two-level fit of f, g
            (Sec. 2.3, the d_x, d_y rows; the method as read);
            "vertex": first derivatives of a vertex-only fit of the flux derivatives
            f_x = A w_x, g_x = B w_x (and f_y, g_y) -- the "fluxes and their derivatives"
            evaluated at vertices, fitted like the viscous fluxes (Sec. 2.3, viscous flux);
            "hermite": the two-level fit of f, g takes the vertex flux derivatives as extra
            Hermite data rows beside the values and the edge projections (the Hermite idea of
            Sec. 2.2 carried over to Eq. (flux_polynomials)); every row comes from that fit.
  deriv_degree  degree of the vertex-only fit for deriv = "vertex".
  flux      the Riemann solver, which the paper does not name (Sec. 2.3 after Alg. 1).
  ls_weight edge-row weight relative to the vertex rows in Eq. (flux_polynomials) (the paper
            weights none).
The sensor's linear weights (R2) do not enter: about a uniform state every side takes the
5-node branch.
"""
from dataclasses import dataclass, replace

import numpy as np
import scipy.sparse as sp

from . import hfd_oracle as H

_CS = 1e-30


@dataclass(frozen=True)
class Reading:
    sv_rule: str = "row"
    div_degree: int = 5
    deriv: str = "fit2"
    deriv_degree: int = 3
    flux: str = "roe"
    ls_weight: float = 1.0

    def label(self):
        s = f"R3 {self.sv_rule}, LS degree {self.div_degree}, derivative rows {self.deriv}"
        if self.deriv == "vertex":
            s += f" (degree {self.deriv_degree})"
        if self.flux != "roe":
            s += f", {self.flux} flux"
        if self.ls_weight != 1.0:
            s += f", edge rows weighted {self.ls_weight:g}"
        return s


# ------------------------------------------------------------------ 5-node weights (Sec. 2.2)

def five_node_weights(rel5, ell, near, sv_rule="row", sv_rtol=1e-13):
    """First row of the scaled pseudo-inverse of the 15x15 Hermite system (Eq. hintp_5), with
    the smallest singular values dropped while the test of `sv_rule` finds an entry >= 1:
    "row" tests the stored row (R3), "all" every entry of the scaled P^+ (each Taylor
    coefficient for each unit datum).  Unscaled and made constant-consistent as in R3/R4."""
    X = rel5 / ell
    p, px, py = H.taylor_basis(X[:, 0], X[:, 1], 4)
    P = np.zeros((15, 15))
    P[0::3], P[1::3], P[2::3] = p.T, px.T, py.T
    U, S, Vt = np.linalg.svd(P)
    r = int(np.sum(S > sv_rtol * S[0]))
    while True:
        Pi = (Vt[:r].T / S[:r]) @ U[:, :r].T
        test = Pi[0] if sv_rule == "row" else Pi
        if np.max(np.abs(test)) < 1.0:
            break
        r -= 1
        if r == 0:
            raise ValueError("no singular value left")
    w = Pi[0].copy()
    w[1::3] *= ell
    w[2::3] *= ell
    w[3 * near] += 1.0 - np.sum(w[0::3])
    return w, r


# ------------------------------------------------------------------ divergence rows (Sec. 2.3)

def _local(mesh, topo, v):
    verts, edges = H.vertex_stencil(topo, v)
    ell = H._vertex_scale(mesh, topo, v)
    xv = np.array([H.disp(mesh, v, u) for u in verts]) / ell
    te = topo["edges"][edges]
    xm = np.zeros((len(edges), 2))
    nm = np.zeros((len(edges), 2))
    for k, (a, b) in enumerate(te):
        d = H.disp(mesh, a, b)
        xm[k] = (H.disp(mesh, v, a) + 0.5 * d) / ell
        nm[k] = d / np.sqrt(d[0] * d[0] + d[1] * d[1])
    return verts, edges, ell, xv, xm, nm


def div_rows(mesh, topo, v, rd):
    """Rows d_0, d_x, d_y over the extended data of vertex v under reading rd.  The extended
    data of one flux component q, for the whole mesh, is
        z = [f_1, g_1, ..., f_V, g_V | h_1 ... h_E | fx_1, fy_1, gx_1, gy_1, ..., gy_V],
    vertex fluxes (Sec. 2.3 after Alg. 1), edge projections h (Eq. flux_polynomials) and the
    vertex flux derivatives f_x = A w_x, f_y = A w_y, g_x = B w_x, g_y = B w_y.  Returns
    (column ids into z, 3 x ncol rows)."""
    verts, edges, ell, xv, xm, nm = _local(mesh, topo, v)
    V = topo["V"]
    E = len(topo["edges"])
    N, M = len(verts), len(edges)
    deg = rd.div_degree
    K = (deg + 1) * (deg + 2) // 2
    pv, pxv, pyv = [t.T for t in H.taylor_basis(xv[:, 0], xv[:, 1], deg)]
    pm = H.taylor_basis(xm[:, 0], xm[:, 1], deg)[0].T
    nrow = 2 * N + M + (4 * N if rd.deriv == "hermite" else 0)
    A = np.zeros((nrow, 2 * K))
    A[0:2 * N:2, :K] = pv                                  # (p^T, 0): f at a vertex
    A[1:2 * N:2, K:] = pv                                  # (0, p^T): g at a vertex
    A[2 * N:2 * N + M, :K] = pm * nm[:, 0:1]               # (p^T n_x, p^T n_y): h at an edge
    A[2 * N:2 * N + M, K:] = pm * nm[:, 1:2]
    o = 2 * N + M
    if rd.deriv == "hermite":                              # (p_x^T, 0) ... : flux derivatives
        A[o + 0::4, :K] = pxv
        A[o + 1::4, :K] = pyv
        A[o + 2::4, K:] = pxv
        A[o + 3::4, K:] = pyv
    W = np.ones(nrow)
    W[2 * N:2 * N + M] = rd.ls_weight
    Ap = np.linalg.pinv(A * W[:, None]) * W[None, :]
    if rd.deriv == "hermite":
        Ap[:, o:] *= ell                                   # derivative data in scaled coordinates
    d0 = (Ap[1] + Ap[K + 2]) / ell
    dx = (Ap[3] + Ap[K + 4]) / ell ** 2
    dy = (Ap[4] + Ap[K + 5]) / ell ** 2
    cols = [np.stack([2 * verts, 2 * verts + 1], 1).ravel(), 2 * V + edges]
    if rd.deriv == "hermite":
        cols.append((2 * V + E + 4 * verts[:, None] + np.arange(4)[None]).ravel())
        return np.concatenate(cols), np.stack([d0, dx, dy])
    cols = np.concatenate(cols)
    if rd.deriv == "fit2":
        return cols, np.stack([d0, dx, dy])
    # "vertex": div f_x = d/dx f_x + d/dy g_x from a vertex-only fit of degree deriv_degree
    B = H.taylor_basis(xv[:, 0], xv[:, 1], rd.deriv_degree)[0].T
    Q = np.linalg.pinv(B)
    base = 2 * V + E + 4 * verts
    cols = np.concatenate([cols, base + 0, base + 2, base + 1, base + 3])
    z = np.zeros(2 * N + M)
    rows = np.zeros((3, len(cols)))
    rows[0, :2 * N + M] = d0
    rows[1] = np.concatenate([z, Q[1] / ell, Q[2] / ell, 0 * Q[1], 0 * Q[2]])   # fx, gx
    rows[2] = np.concatenate([z, 0 * Q[1], 0 * Q[2], Q[1] / ell, Q[2] / ell])   # fy, gy
    return cols, rows


class Prep:
    """Geometry-only data of one reading (all vertices active, periodic meshes)."""


def prepare(mesh, rd):
    """Edge stencils and weights (Sec. 2.2-2.3) and the extended divergence operators D_k of
    reading rd at every vertex of a periodic mesh."""
    opts = H.Options(div_degree=rd.div_degree, flux=rd.flux)
    P = H.prepare(mesh, opts)
    if rd.sv_rule != "row":
        for i, e in enumerate(P.edges):
            ids, rel, ell, n = H.edge_geometry(mesh, P.topo, int(e))
            P.w5[i, 0], P.rank[i, 0] = five_node_weights(rel[H.LEFT5], ell, 2, rd.sv_rule)
            P.w5[i, 1], P.rank[i, 1] = five_node_weights(rel[H.RIGHT5], ell, 2, rd.sv_rule)
    V = P.topo["V"]
    E = len(P.topo["edges"])
    r_, c_, v_ = [[], [], []], [[], [], []], [[], [], []]
    for r, v in enumerate(P.active):
        cols, rows = div_rows(mesh, P.topo, int(v), rd)
        for k in range(3):
            r_[k].append(np.full(len(cols), r))
            c_[k].append(cols)
            v_[k].append(rows[k])
    P.Dx = [sp.csr_matrix((np.concatenate(v_[k]), (np.concatenate(r_[k]), np.concatenate(c_[k]))),
                          shape=(len(P.active), 6 * V + E)) for k in range(3)]
    P.reading = rd
    return P


def flux_derivatives(U, gamma):
    """A(w) w_x, B(w) w_x, A(w) w_y, B(w) w_y at every vertex, by the complex-step derivative
    of the analytic flux along w_x and w_y (exact to rounding)."""
    w = U[0:4].astype(complex)
    Fx, Gx = H.euler_flux(w + 1j * _CS * U[4:8], gamma)
    Fy, Gy = H.euler_flux(w + 1j * _CS * U[8:12], gamma)
    return Fx.imag / _CS, Gx.imag / _CS, Fy.imag / _CS, Gy.imag / _CS


def residual(mesh, P, U):
    """R(U) of Eq. (HWENO) under the reading of P (inviscid, periodic): rows 0-3 -div f,
    rows 4-7 -div f_x, rows 8-11 -div f_y, each -D_k z_q."""
    g = P.opts.gamma
    V = U.shape[1]
    E = len(P.topo["edges"])
    F, G = H.euler_flux(U[0:4], g)
    wl, wr = H.edge_values(P, U, P.opts)
    h = H.riemann_flux(wl, wr, P.normal[:, 0], P.normal[:, 1], P.opts)
    Fx, Gx, Fy, Gy = flux_derivatives(U, g)
    Rm = np.zeros((12, V))
    for q in range(4):
        z = np.zeros(6 * V + E)
        z[0:2 * V:2], z[1:2 * V:2] = F[q], G[q]
        z[2 * V + P.edges] = h[q]
        o = 2 * V + E
        z[o + 0::4], z[o + 1::4], z[o + 2::4], z[o + 3::4] = Fx[q], Fy[q], Gx[q], Gy[q]
        for k in range(3):
            Rm[4 * k + q, P.active] = -(P.Dx[k] @ z)
    return Rm


# ------------------------------------------------------------------ linear stability

def jacobian(mesh, P, U0):
    """dR/dU (12V x 12V) about the uniform state U0, assembled from complex-step derivatives:
    the analytic flux Jacobians A, B at the state and, per edge, the derivative of its Riemann
    flux with respect to each of the 72 stencil values (Alg. 1 is smooth there: every side
    takes the 5-node branch)."""
    V = U0.shape[1]
    E = len(P.topo["edges"])
    N = 12 * V
    w0 = U0[:4, 0].astype(complex)
    A = np.zeros((4, 4))
    B = np.zeros((4, 4))
    for j in range(4):
        dw = np.zeros(4, complex)
        dw[j] = 1j * _CS
        F, G = H.euler_flux((w0 + dw)[:, None], P.opts.gamma)
        A[:, j], B[:, j] = F[:, 0].imag / _CS, G[:, 0].imag / _CS
    W0 = U0[:, P.stencil].astype(complex)
    Jh = np.zeros((4, len(P.edges), 12, 6))
    for r in range(12):
        for k in range(6):
            W = W0.copy()
            W[r, :, k] += 1j * _CS
            Jh[:, :, r, k] = H.edge_flux_from_stencil(P, W, P.opts).imag / _CS
    ar = np.arange(V)
    o = 2 * V + E
    J = np.zeros((N, N))
    for q in range(4):
        r_, c_, v_ = [], [], []
        for j in range(4):
            for M_, slot_v, slots_d in ((A, 0, (0, 1)), (B, 1, (2, 3))):
                if M_[q, j] == 0.0:
                    continue
                r_.append(2 * ar + slot_v)
                c_.append(j * V + ar)
                v_.append(np.full(V, M_[q, j]))
                for slot, off in zip(slots_d, (4, 8)):         # d(M w_x)/d w_x = M at w_x = 0
                    r_.append(o + 4 * ar + slot)
                    c_.append((off + j) * V + ar)
                    v_.append(np.full(V, M_[q, j]))
        for rr in range(12):
            for k in range(6):
                r_.append(2 * V + P.edges)
                c_.append(rr * V + P.stencil[:, k])
                v_.append(Jh[q, :, rr, k])
        Z = sp.csr_matrix((np.concatenate(v_), (np.concatenate(r_), np.concatenate(c_))),
                          shape=(6 * V + E, N))
        for k in range(3):
            J[(4 * k + q) * V + P.active] = -(P.Dx[k] @ Z).toarray()
    return J


def rk3_gain(z):
    """|G(z)| of the three-stage SSP Runge-Kutta scheme, G(z) = 1 + z + z^2/2 + z^3/6."""
    return np.abs(1.0 + z + z * z / 2.0 + z ** 3 / 6.0)


def linear_growth(n, rd, jitter=0.15, seed=3, u=0.5, v=0.2):
    """Growth of the linearised method about the uniform flow (rho, u, v, p) = (1, u, v, 1) on
    the n x n jittered periodic unit square: (max Re lambda * h / (|u| + c), max RK3 gain at
    the CFL-0.3 step of R12, the Jacobian's eigenvalues)."""
    from synth import jittered_grid, uniform_state
    m = jittered_grid(n, n, 1.0, 1.0, seed=seed, jitter=jitter)
    P = prepare(m, rd)
    U0 = uniform_state(m, rho=1.0, u=u, v=v, p=1.0)
    lam = np.linalg.eigvals(jacobian(m, P, U0))
    speed = np.hypot(u, v) + np.sqrt(1.4)
    lmin = min(min(np.linalg.norm(H.disp(m, a, b)) for b in P.topo["nbrs"][a])
               for a in range(len(m["x"])))
    dt = 0.3 * lmin / speed
    return lam.real.max() / n / speed, rk3_gain(lam * dt).max(), lam


def fourier_1d(herm_degree=4, div_degree=5, levels=2, upwind=True, nth=181):
    """Largest Re(lambda) h / a over the Fourier modes of the 1D analogue of the method for
    u_t + a u_x = 0 on a uniform grid: unknowns u_j and v_j (the derivative), the edge value at
    j+1/2 from a 1D Hermite least-squares fit of degree herm_degree to (u, v) at j-2..j+2 (the
    upwind side; upwind=False averages it with the other side's j-1..j+3), and u_t, v_t minus
    the first and second derivatives of a least-squares polynomial of degree div_degree fitted
    to the vertex values at j-levels..j+levels and the edge values between them (the 1D form of
    Eq. flux_polynomials and of the d_0, d_x rows)."""
    from math import factorial

    def basis(x, deg):
        return (np.array([x ** k / factorial(k) for k in range(deg + 1)]),
                np.array([k * x ** (k - 1) / factorial(k) if k else 0.0 * x
                          for k in range(deg + 1)]))

    def herm(nodes):
        A = np.zeros((2 * len(nodes), herm_degree + 1))
        for i, x in enumerate(nodes):
            A[2 * i], A[2 * i + 1] = basis(x - 0.5, herm_degree)
        w = np.linalg.pinv(A)[0]
        return w[0::2], w[1::2]

    xv = np.arange(-levels, levels + 1.0)
    xm = np.arange(-levels + 0.5, levels, 1.0)
    Ap = np.linalg.pinv(np.array([basis(x, div_degree)[0] for x in np.concatenate([xv, xm])]))
    d1, d2 = Ap[1], Ap[2]
    nv = len(xv)
    kl, kr = np.arange(-2, 3), np.arange(-1, 4)
    al, bl = herm(kl.astype(float))
    ar, br = herm(kr.astype(float))
    worst = -np.inf
    for th in np.linspace(0.0, np.pi, nth):
        Ha = np.sum(al * np.exp(1j * th * (kl - 0.5)))
        Hb = np.sum(bl * np.exp(1j * th * (kl - 0.5)))
        if not upwind:
            Ha = 0.5 * (Ha + np.sum(ar * np.exp(1j * th * (kr - 0.5))))
            Hb = 0.5 * (Hb + np.sum(br * np.exp(1j * th * (kr - 0.5))))
        ev, em = np.exp(1j * th * xv), np.exp(1j * th * xm)
        C1v, C1e, C2v, C2e = d1[:nv] @ ev, d1[nv:] @ em, d2[:nv] @ ev, d2[nv:] @ em
        Msym = -np.array([[C1v + C1e * Ha, C1e * Hb], [C2v + C2e * Ha, C2e * Hb]])
        worst = max(worst, np.linalg.eigvals(Msym).real.max())
    return worst


# ------------------------------------------------------------------ accuracy under a reading

def monte_carlo_order(sv_rule, samples=150, seed=5):
    """Median observed order of the 5-node interpolation on the random stencils of the paper's
    Monte Carlo test (Sec. 2.2: edge lengths with 15 % spread, deflections N(0, pi/12), random
    orientation), halving the stencil size once."""
    rng = np.random.default_rng(seed)

    def f(x, y):
        v = np.sin(1.3 * x + 0.7) * np.cos(0.9 * y - 0.4) + 0.5 * np.exp(0.3 * x * y)
        fx = 1.3 * np.cos(1.3 * x + 0.7) * np.cos(0.9 * y - 0.4) + 0.15 * y * np.exp(0.3 * x * y)
        fy = -0.9 * np.sin(1.3 * x + 0.7) * np.sin(0.9 * y - 0.4) + 0.15 * x * np.exp(0.3 * x * y)
        return v, fx, fy

    orders = []
    for _ in range(samples):
        L = 1.0 + 0.15 * rng.standard_normal(3)
        th = rng.normal(0.0, np.pi / 12, 3)
        pts = {2: np.array([-0.5, 0.0]), 3: np.array([0.5, 0.0])}
        a, p = 0.0, pts[2]
        for k, node in enumerate([1, 0]):
            a += th[k]
            p = p + L[k] * np.array([-np.cos(a), -np.sin(a)])
            pts[node] = p
        pts[4] = pts[3] + L[2] * np.array([np.cos(th[2]), np.sin(th[2])])
        X = np.array([pts[k] for k in range(5)])
        phi = rng.uniform(0, 2 * np.pi)
        X = X @ np.array([[np.cos(phi), np.sin(phi)], [-np.sin(phi), np.cos(phi)]])
        x0 = rng.uniform(-1, 1, 2)
        errs = []
        for hh in (0.05, 0.025):
            rel = X * hh
            w, _ = five_node_weights(rel, hh, 2, sv_rule)
            Q = x0[None] + rel
            v, fx, fy = f(Q[:, 0], Q[:, 1])
            errs.append(abs(w @ np.stack([v, fx, fy], 1).ravel() - f(*x0)[0]))
        orders.append(np.log2(errs[0] / errs[1]))
    return float(np.median(orders))


def vortex_row_orders(rd, ns=(20, 40, 80), nsample=60):
    """Truncation orders of the value rows and of the two derivative-row groups: the residual
    of the exact isentropic vortex (Sec. 3.1, beta = 5, mean flow (1, 1)) against its exact
    time derivative, mean absolute error over about nsample vertices near the vortex centre.
    The exact derivative of all 12 unknowns is a fourth-order central difference in time of
    the translated exact solution (step 1e-3: error ~1e-11, far below the residual errors)."""
    from synth import jittered_grid, isentropic_vortex
    errs = []
    for n in ns:
        m = jittered_grid(n, n, 10.0, 10.0, seed=1)
        U = isentropic_vortex(m)
        d = 1e-3
        dUdt = (-isentropic_vortex(m, t=2 * d) + 8 * isentropic_vortex(m, t=d)
                - 8 * isentropic_vortex(m, t=-d) + isentropic_vortex(m, t=-2 * d)) / (12 * d)
        act = np.nonzero((np.abs(m["x"] - 5) < 2.0) & (np.abs(m["y"] - 5) < 2.0))[0]
        act = act[:: max(1, len(act) // nsample)]
        opts = H.Options(div_degree=rd.div_degree, flux=rd.flux)
        P = H.prepare(m, opts, active=act)
        if rd.sv_rule != "row":
            for i, e in enumerate(P.edges):
                ids, rel, ell, nn = H.edge_geometry(m, P.topo, int(e))
                P.w5[i, 0], _ = five_node_weights(rel[H.LEFT5], ell, 2, rd.sv_rule)
                P.w5[i, 1], _ = five_node_weights(rel[H.RIGHT5], ell, 2, rd.sv_rule)
        V = len(m["x"])
        E = len(P.topo["edges"])
        r_, c_, v_ = [[], [], []], [[], [], []], [[], [], []]
        for r, v in enumerate(act):
            cols, rows = div_rows(m, P.topo, int(v), rd)
            for k in range(3):
                r_[k].append(np.full(len(cols), r))
                c_[k].append(cols)
                v_[k].append(rows[k])
        P.Dx = [sp.csr_matrix((np.concatenate(v_[k]), (np.concatenate(r_[k]),
                                                        np.concatenate(c_[k]))),
                              shape=(len(act), 6 * V + E)) for k in range(3)]
        R = residual(m, P, U)
        e = np.abs(R[:, act] - dUdt[:, act])
        errs.append([e[0:4].mean(), e[4:8].mean(), e[8:12].mean()])
    errs = np.array(errs)
    return np.log2(errs[:-1] / errs[1:]), errs


READINGS = [
    Reading(),
    Reading(sv_rule="all"),
    Reading(div_degree=4), Reading(div_degree=3),
    Reading(sv_rule="all", div_degree=4), Reading(sv_rule="all", div_degree=3),
    Reading(deriv="vertex", deriv_degree=4), Reading(deriv="vertex", deriv_degree=3),
    Reading(deriv="vertex", deriv_degree=2),
    Reading(sv_rule="all", deriv="vertex", deriv_degree=2),
    Reading(deriv="hermite"), Reading(deriv="hermite", div_degree=4),
    Reading(deriv="hermite", div_degree=6),
    Reading(flux="rusanov"),
    Reading(ls_weight=3.0), Reading(ls_weight=0.3),
]


def sweep(readings=READINGS, sizes=(8, 10, 12), accuracy=True, out=print):
    """Prints one table row per reading: the worst growth and RK3 gain over the meshes (jitter
    0 and 0.15), the Monte Carlo order and the vortex truncation orders of the three row
    groups from 40 to 80 vertices per side."""
    out("| reading | max Re(lambda) h/(|u|+c), jitter 0 / 0.15 | max RK3 gain | MC order | "
        "vortex orders 40->80 (w, w_x, w_y) |")
    out("|---|---|---|---|---|")
    for rd in readings:
        g0 = max(linear_growth(n, rd, jitter=0.0)[0] for n in sizes)
        gains, g1 = [], -np.inf
        for n in sizes:
            gr, gain, _ = linear_growth(n, rd)
            g1 = max(g1, gr)
            gains.append(gain)
        mc = vor = "-"
        if accuracy:
            mc = f"{monte_carlo_order(rd.sv_rule):.2f}"
            o, _ = vortex_row_orders(rd)
            vor = ", ".join(f"{x:.1f}" for x in o[-1])
        out(f"| {rd.label()} | {g0:.3f} / {g1:.3f} | {max(gains):.3f} | {mc} | {vor} |")


if __name__ == "__main__":
    sweep()
