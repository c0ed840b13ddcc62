"""Pins of the 3D extension's oracle (oracle/hfd3d.py) against closed forms and invariants:
mesh conformity, the Taylor basis, polynomial exactness of the 5-node and 3-node weights and
of the divergence rows, the eigenstructure and Roe's property, freestream preservation,
covariance under a rotation of the axes, and the truncation order on an exact solution."""
import itertools
import os

import numpy as np
import pytest

from oracle import hfd3d as O
from synth import three_d as T


@pytest.fixture(scope="module")
def box6():
    m = T.periodic_tet_box(6, 6, 6, 1.0, 1.2, 0.9, seed=5)
    return m, O.prepare(m)


def _faces(tet):
    f = np.concatenate([np.sort(tet[:, list(c)], 1) for c in itertools.combinations(range(4), 3)])
    _, counts = np.unique(f, axis=0, return_counts=True)
    return counts


def test_kuhn_box_is_conforming_and_tiles():
    m = T.periodic_tet_box(5, 4, 6, 2.0, 1.0, 3.0, seed=2)
    tet = m["tet"]
    d = [T.disp3(m, tet[:, 0], tet[:, k]) for k in (1, 2, 3)]
    vol = np.einsum("ij,ij->i", d[0], np.cross(d[1], d[2])) / 6.0
    assert vol.min() > 0
    assert abs(vol.sum() - 6.0) < 1e-12
    assert np.all(_faces(tet) == 2)                 # every face shared by exactly two tetrahedra
    topo = O.build_topology(m)
    assert all(len(n) == 14 for n in topo["nbrs"])


def test_taylor_basis_order_and_derivatives_by_complex_step():
    x, y, z = 0.3, -0.7, 0.45
    p = O.taylor_basis(x, y, z, 2)[0]
    np.testing.assert_allclose(p, [1, x, y, z, x * x / 2, x * y, x * z, y * y / 2, y * z, z * z / 2])
    h = 1e-30
    for deg in (3, 4):
        p, px, py, pz = O.taylor_basis(x, y, z, deg)
        assert len(p) == (deg + 1) * (deg + 2) * (deg + 3) // 6
        np.testing.assert_allclose(px, O.taylor_basis(x + 1j * h, y, z, deg)[0].imag / h, atol=1e-14)
        np.testing.assert_allclose(py, O.taylor_basis(x, y + 1j * h, z, deg)[0].imag / h, atol=1e-14)
        np.testing.assert_allclose(pz, O.taylor_basis(x, y, z + 1j * h, deg)[0].imag / h, atol=1e-14)


def _cubic(rng):
    """A random cubic in 3D by its monomial coefficients, evaluated with its gradient
    independently of the oracle's basis."""
    mons = [(a, b, c) for a in range(4) for b in range(4) for c in range(4) if a + b + c <= 3]
    coef = rng.normal(size=len(mons))

    def ev(P):
        v = np.zeros(len(P)); g = np.zeros((len(P), 3))
        for k, (a, b, c) in enumerate(mons):
            x, y, z = P[:, 0], P[:, 1], P[:, 2]
            v += coef[k] * x ** a * y ** b * z ** c
            if a: g[:, 0] += coef[k] * a * x ** (a - 1) * y ** b * z ** c
            if b: g[:, 1] += coef[k] * b * x ** a * y ** (b - 1) * z ** c
            if c: g[:, 2] += coef[k] * c * x ** a * y ** b * z ** (c - 1)
        return v, g
    return ev, coef[mons.index((0, 0, 0))]


def test_five_node_weights_exact_for_cubics_at_full_rank(box6):
    """T1: with the 20 x 20 system at full rank the 5-node weights reproduce every cubic at the
    edge midpoint (value and gradient data at the five nodes)."""
    m, P = box6
    topo = P.topo
    rng = np.random.default_rng(7)
    checked = 0
    for e in rng.choice(len(topo["edges"]), 60, replace=False):
        ids, rel, ell, n = O.edge_geometry(m, topo, int(e))
        for side, five in enumerate((O.LEFT5, O.RIGHT5)):
            w, r = O.five_node_weights(rel[five], ell, near=2)
            assert abs(w[0::4].sum() - 1.0) < 1e-14          # constants exact (R4)
            if r < 20:
                continue
            ev, p0 = _cubic(rng)
            v, g = ev(rel[five])
            data = np.stack([v, g[:, 0], g[:, 1], g[:, 2]], 1).ravel()
            assert abs(w @ data - p0) < 1e-10 * (1 + np.abs(data).max())
            checked += 1
    assert checked > 60


def test_three_node_weights_match_pinv_and_are_exact_along_lines():
    """T2: the minimum-norm first row of the 3 x 10 system (checked against numpy's pinv with
    an independently written basis), constants exact, and quadratics along a straight line of
    nodes through the evaluation point exact."""
    rng = np.random.default_rng(3)

    def basis2(x, y, z):
        return np.array([1, x, y, z, x * x / 2, x * y, x * z, y * y / 2, y * z, z * z / 2])
    for _ in range(20):
        rel = rng.uniform(-1.5, 1.5, (3, 3))
        w = O.three_node_weights(rel, 1)
        ref = np.linalg.pinv(np.array([basis2(*r) for r in rel]))[0]
        ref[1] += 1.0 - ref.sum()
        np.testing.assert_allclose(w, ref, atol=1e-12)
        assert abs(w.sum() - 1.0) < 1e-14
    d = np.array([0.48, -0.6, 0.64])
    t = np.array([-2.3, -1.1, -0.4]) * 0.2
    w = O.three_node_weights(t[:, None] * d[None], 2)
    assert abs(w @ (0.7 - 1.3 * t + 2.1 * t * t) - 0.7) < 1e-12


def _random_states(rng, k):
    rho = rng.uniform(0.5, 2.0, k)
    vel = rng.uniform(-1.0, 1.0, (3, k))
    p = rng.uniform(0.5, 2.0, k)
    from synth.three_d import prim_to_cons3
    return prim_to_cons3(rho, vel[0], vel[1], vel[2], p)


def _unit(rng, k):
    n = rng.normal(size=(k, 3))
    return n / np.linalg.norm(n, axis=1)[:, None]


def test_tangent_frame_is_right_handed_orthonormal():
    rng = np.random.default_rng(4)
    for n in list(_unit(rng, 50)) + [np.array([1.0, 0, 0]), np.array([0, 0, -1.0]),
                                     np.array([1, 1, 1]) / np.sqrt(3)]:
        t1, t2 = O.tangents(n)
        F = np.stack([n, t1, t2])
        np.testing.assert_allclose(F @ F.T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(F) - 1.0) < 1e-14


def test_eigenvectors_inverse_and_diagonalise_flux_jacobian():
    """L R = I, and R diag(lambda) L is the flux Jacobian along n (by complex step of the
    normal flux, an independent route)."""
    rng = np.random.default_rng(5)
    k = 40
    w = _random_states(rng, k)
    n = _unit(rng, k)
    t1, t2 = np.array([O.tangents(x) for x in n]).transpose(1, 0, 2)
    vel, H, c = O.roe_average(w, w, 1.4)
    L, R = O.eigenvectors(vel, H, c, n, t1, t2, 1.4)
    np.testing.assert_allclose(np.einsum("eij,ejk->eik", L, R), np.broadcast_to(np.eye(5), (k, 5, 5)),
                               atol=1e-12)
    qn = np.sum(vel.T * n, 1)
    lam = np.stack([qn - c, qn, qn, qn, qn + c], 1)
    A = np.einsum("eij,ej,ejk->eik", R, lam, L)
    J = np.zeros((k, 5, 5))
    for j in range(5):
        wc = w.astype(complex)
        wc[j] += 1j * 1e-30
        J[:, :, j] = (O.normal_flux(wc, n, 1.4).imag / 1e-30).T
    np.testing.assert_allclose(A, J, atol=1e-11)


def test_roe_property_consistency_and_supersonic_upwinding():
    rng = np.random.default_rng(6)
    k = 40
    wl, wr = _random_states(rng, k), _random_states(rng, k)
    n = _unit(rng, k)
    t1, t2 = np.array([O.tangents(x) for x in n]).transpose(1, 0, 2)
    # Roe's property: F_n(wr) - F_n(wl) = R Lambda L (wr - wl) at the Roe average
    vel, H, c = O.roe_average(wl, wr, 1.4)
    L, R = O.eigenvectors(vel, H, c, n, t1, t2, 1.4)
    qn = np.sum(vel.T * n, 1)
    lam = np.stack([qn - c, qn, qn, qn, qn + c], 1)
    jump = np.einsum("eij,ej,ejk,ke->ie", R, lam, L, wr - wl)
    np.testing.assert_allclose(jump, O.normal_flux(wr, n, 1.4) - O.normal_flux(wl, n, 1.4),
                               atol=1e-12)
    # consistency h(w, w) = F_n(w)
    np.testing.assert_allclose(O.roe_flux(wl, wl, n, t1, t2, 1.4), O.normal_flux(wl, n, 1.4),
                               atol=1e-13)
    # supersonic along n: the flux is the upwind state's
    from synth.three_d import prim_to_cons3
    nn = np.tile([[0.6, 0.0, 0.8]], (3, 1))
    s1, s2 = np.array([O.tangents(x) for x in nn]).transpose(1, 0, 2)
    a = prim_to_cons3(np.ones(3), 3.0 * 0.6 * np.ones(3), 0.2 * np.ones(3), 3.0 * 0.8 * np.ones(3), np.ones(3))
    b = prim_to_cons3(1.2 * np.ones(3), 2.9 * 0.6 * np.ones(3), -0.1 * np.ones(3), 2.9 * 0.8 * np.ones(3), 1.1 * np.ones(3))
    np.testing.assert_allclose(O.roe_flux(a, b, nn, s1, s2, 1.4), O.normal_flux(a, nn, 1.4), atol=1e-12)


def _quartic_field(rng):
    mons = [(a, b, c) for a in range(5) for b in range(5) for c in range(5) if a + b + c <= 4]
    coef = rng.normal(size=(3, len(mons)))

    def ev(P, f, dx=(0, 0, 0)):
        """component f of the field (or its partial derivative of multi-index dx) at points P"""
        out = np.zeros(len(P))
        for k, (a, b, c) in enumerate(mons):
            e = (a - dx[0], b - dx[1], c - dx[2])
            if min(e) < 0:
                continue
            fac = 1.0
            for n_, d_ in zip((a, b, c), dx):
                for j in range(d_):
                    fac *= n_ - j
            out += coef[f, k] * fac * P[:, 0] ** e[0] * P[:, 1] ** e[1] * P[:, 2] ** e[2]
        return out
    return ev


def test_divergence_rows_exact_for_quartic_flux_fields(box6):
    """T4: for polynomial flux vectors (f, g, k) of degree 4, with vertex data f, g, k and edge
    data (f, g, k) . n at the midpoints, d_0 gives div at the vertex and d_x, d_y, d_z give the
    divergences of the x, y and z derivative fluxes exactly."""
    m, P = box6
    topo = P.topo
    rng = np.random.default_rng(8)
    V = topo["V"]
    for v in rng.choice(V, 6, replace=False):
        v = int(v)
        verts, edges, d = O.div_rows(m, topo, v, P.opts)
        ev = _quartic_field(rng)
        xv = np.array([O.disp(m, v, u) for u in verts])
        te = topo["edges"][edges]
        xm = np.array([O.disp(m, v, a) + 0.5 * O.disp(m, a, b) for a, b in te])
        nm = np.array([O.disp(m, a, b) / np.linalg.norm(O.disp(m, a, b)) for a, b in te])
        z = np.concatenate([np.stack([ev(xv, 0), ev(xv, 1), ev(xv, 2)], 1).ravel(),
                            sum(ev(xm, f) * nm[:, f] for f in range(3))])
        o = np.zeros((1, 3))
        div = lambda extra: sum(ev(o, f, tuple(int(i == f) + extra[i] for i in range(3)))[0]
                                for f in range(3))
        exact = [div((0, 0, 0)), div((1, 0, 0)), div((0, 1, 0)), div((0, 0, 1))]
        scale = np.abs(z).max()
        for k in range(4):
            assert abs(d[k] @ z - exact[k]) < 1e-9 * scale * (1 + np.abs(d[k]).sum())


def test_freestream_preserved(box6):
    m, P = box6
    U = T.uniform_state3(m)
    R = O.residual(m, P, U)
    assert np.abs(R).max() < 1e-12 * np.abs(U).max() / 0.2


def _cycle_axes(m, U):
    """The same mesh and state with the axes relabelled x' = y, y' = z, z' = x (a rotation)."""
    m2 = dict(m)
    m2["x"], m2["y"], m2["z"] = m["y"], m["z"], m["x"]
    m2["Lx"], m2["Ly"], m2["Lz"] = m["Ly"], m["Lz"], m["Lx"]
    comp = [0, 2, 3, 1, 4]                      # (rho, m_y, m_z, m_x, E)
    groups = [0, 2, 3, 1]                       # (w, w_y, w_z, w_x)
    out = np.concatenate([U[5 * g + np.array(comp)] for g in groups])
    return m2, out


def test_residual_is_rotation_covariant(box6):
    """Relabelling the axes cyclically maps the residual to the relabelled residual (5-node
    branch: its values are independent of the choice of the shear tangents)."""
    m, _ = box6
    opts = O.Options3(force_branch="hermite")
    P = O.prepare(m, opts)
    U = T.vortex_tube(m, beta=2.0, mean=(0.4, -0.3, 0.6))
    R = O.residual(m, P, U)
    m2, U2 = _cycle_axes(m, U)
    P2 = O.prepare(m2, opts)
    assert np.array_equal(P2.stencil, P.stencil)
    R2 = O.residual(m2, P2, U2)
    _, Rc = _cycle_axes(m, R)
    # the 20 x 20 Hermite systems are ill-conditioned (sigma_min / sigma_max has a median of about
    # 4e-7 and reaches 1e-11), so reordering the basis moves the weights by rounding amplified
    # that much; an index or sign mistake moves the residual by O(1)
    assert np.abs(R2 - Rc).max() < 1e-8 * np.abs(R).max()


def test_cfl_step_closed_form(box6):
    m, P = box6
    U = T.uniform_state3(m, rho=1.3, u=0.2, v=-0.4, w=0.1, p=0.9)
    lmin = min(np.linalg.norm(O.disp(m, a, b)) for a, b in P.topo["edges"])
    speed = np.sqrt(0.2 ** 2 + 0.4 ** 2 + 0.1 ** 2) + np.sqrt(1.4 * 0.9 / 1.3)
    assert abs(O.cfl_dt(m, P, U) - 0.3 * lmin / speed) < 1e-15


@pytest.mark.skipif(os.environ.get("HFD_SKIP_SLOW") == "1", reason="slow oracle refinement")
def test_residual_truncation_error_converges_on_an_exact_solution():
    """A density wave along x carried by a uniform flow: the exact time derivative of every row
    is -(u . grad) of it.  From 6^3 to 8^3 the error falls at order >= 3 in the value rows
    (fourth-order interpolation, degree-4 divergence; measured 4.2) and >= 1.5 in the derivative
    rows (measured 3.3-4.0)."""
    errs = []
    for n in (6, 8):
        m = T.periodic_tet_box(n, n, n, 1.0, 1.0, 1.0, seed=1)
        P = O.prepare(m)
        vel = (0.5, -0.3, 0.4)
        wave = lambda t: T.density_wave(dict(m, Ly=1e30, Lz=1e30), vel=vel, t=t)
        U = wave(0.0)
        dUdt = (wave(1e-6) - wave(-1e-6)) / 2e-6
        R = O.residual(m, P, U)
        errs.append([np.abs(R[5 * g:5 * g + 5] - dUdt[5 * g:5 * g + 5]).max() for g in range(4)])
    order = np.log(np.array(errs[0]) / np.array(errs[1])) / np.log(8 / 6)
    assert order[0] >= 3.0
    assert order[1:].min() >= 1.5
