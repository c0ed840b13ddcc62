"""FP64 oracle of the discrete adjoint (vector-Jacobian product) of the residual and of one
SSP-RK3 step.  TEST INFRASTRUCTURE ONLY (see the package docstring).

The residual is R(U) = -D [F(U), G(U), h(U)] (+ the viscous divergence), with D the fixed
least-squares divergence rows of Eq. (flux_polynomials).  Its transpose product is therefore
  (dR/dU)^T mu = -sum_vertices J_(F,G)^T (D^T mu)_vertex - sum_edges J_h^T (D^T mu)_edge,
where J_(F,G) are the 4x4 Jacobians of the analytic vertex fluxes and J_h the 4x72 Jacobian of
an edge's numerical flux with respect to the 12 values of its 6 stencil nodes (Alg. 1 + Roe
flux, branch decisions held fixed).  Both Jacobians are taken by the complex-step method on the
oracle's own flux functions (exact to rounding: no subtractive cancellation), vectorised over
all vertices / edges at once.  The ghost refresh is linear and enters transposed.
"""
import numpy as np

from .hfd_oracle import (edge_flux_from_stencil, euler_flux, ghost_fill, residual,
                         viscous_flux)

_H = 1e-30


def _ghost_transpose(mesh, g):
    """Adjoint of the ghost refresh: transmissive ghost columns pass their (masked) sensitivities
    to their donors and become zero; fixed ghosts (donor -1) keep theirs."""
    gid = np.asarray(mesh["ghost_ids"], dtype=np.int64)
    dn = np.asarray(mesh["ghost_donor"], dtype=np.int64)
    fl = np.asarray(mesh["ghost_flags"])
    # fixed ghosts (R22) are not overwritten by the refresh: their values are inputs of the
    # residual like any other column and keep their sensitivities
    gid, dn, fl = gid[dn >= 0], dn[dn >= 0], fl[dn >= 0]
    if len(gid) == 0:
        return g
    gg = g[:, gid].copy()
    gg[4:8, (fl & 1) != 0] = 0.0
    gg[8:12, (fl & 2) != 0] = 0.0
    np.add.at(g.T, dn, gg.T)
    g[:, gid] = 0.0
    return g


def residual_vjp(mesh, P, U, mu, opts=None):
    """(dR/dU)^T mu for mu of shape 12 x V (its ghost columns are ignored)."""
    opts = opts or P.opts
    Ug = ghost_fill(mesh, np.array(U, dtype=float, copy=True))
    V = Ug.shape[1]
    E = len(P.topo["edges"])
    act = P.active
    z = np.zeros((4, 2 * V + E))
    for q in range(4):
        z[q] = -(P.D[0].T @ mu[q, act] + P.D[1].T @ mu[4 + q, act] + P.D[2].T @ mu[8 + q, act])
    zF, zG, zh = z[:, 0:2 * V:2], z[:, 1:2 * V:2], z[:, 2 * V + P.edges]
    g = np.zeros((12, V))
    for k in range(4):                         # analytic vertex fluxes
        w = Ug[:4].astype(complex)
        w[k] += 1j * _H
        F, G = euler_flux(w, opts.gamma)
        g[k] += np.sum(zF * (F.imag / _H) + zG * (G.imag / _H), axis=0)
    W = Ug[:, P.stencil]                       # (12, Ee, 6)
    for node in range(6):                      # edge numerical fluxes
        for r in range(12):
            Wc = W.astype(complex)
            Wc[r, :, node] += 1j * _H
            dh = edge_flux_from_stencil(P, Wc, opts).imag / _H          # (4, Ee)
            np.add.at(g[r], P.stencil[:, node], np.sum(zh * dh, axis=0))
    if opts.viscous:                           # + div(f_vis): rows Dv, all 12 state values
        zv = np.zeros((4, 2 * V))
        for q in range(4):
            zv[q] = P.Dv[0].T @ mu[q, act] + P.Dv[1].T @ mu[4 + q, act] + P.Dv[2].T @ mu[8 + q, act]
        for r in range(12):
            Uc = Ug.astype(complex)
            Uc[r] += 1j * _H
            Fv, Gv = viscous_flux(Uc, opts)
            g[r] += np.sum(zv[:, 0::2] * (Fv.imag / _H) + zv[:, 1::2] * (Gv.imag / _H), axis=0)
    return _ghost_transpose(mesh, g)


def step_vjp(mesh, P, U, dt, lam, opts=None):
    """(d step(U) / dU)^T lam for one SSP-RK3 step with a fixed dt (the oracle's `step`)."""
    opts = opts or P.opts
    act = P.active
    u = ghost_fill(mesh, np.array(U, dtype=float, copy=True))
    u1 = u + dt * residual(mesh, P, u.copy(), opts)
    u1g = ghost_fill(mesh, u1.copy())
    u2 = 0.75 * u + 0.25 * (u1g + dt * residual(mesh, P, u1g.copy(), opts))
    # reverse: the step's result is G(active columns of the last stage, ghosts from u)
    lr = _ghost_transpose(mesh, np.array(lam, dtype=float, copy=True))
    mu3 = np.zeros_like(lr)
    mu3[:, act] = lr[:, act]
    lu = lr - mu3                                  # ghost columns of the result come from u
    lu += mu3 / 3.0
    # fixed ghost columns (R22) of the stage states are those of u (the residual is zero there)
    fx = np.asarray(mesh["ghost_ids"], dtype=np.int64)[np.asarray(mesh["ghost_donor"]) < 0]
    lu2 = 2.0 / 3.0 * (mu3 + dt * residual_vjp(mesh, P, u2, mu3, opts))
    m2 = np.zeros_like(lu2)
    m2[:, act] = lu2[:, act]
    lu += 0.75 * m2
    lu[:, fx] += lu2[:, fx]
    lu1 = 0.25 * (m2 + dt * residual_vjp(mesh, P, u1, m2, opts))
    m1 = np.zeros_like(lu1)
    m1[:, act] = lu1[:, act]
    lu += m1 + dt * residual_vjp(mesh, P, u, m1, opts)
    lu[:, fx] += lu1[:, fx]
    return _ghost_transpose(mesh, lu)
