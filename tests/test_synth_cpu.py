"""CPU checks of the synthetic inputs that the parity tests and the bench rely on: the
embedded-circle Delaunay mesh of the circular Sod problem (Sec. 3.3) and its initial state."""
import numpy as np
import pytest

import synth


@pytest.fixture(scope="module", params=[16, 50])
def circ(request):
    return synth.embedded_circle_box(request.param, seed=8)


def _edges(tri):
    e = np.sort(np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]]), axis=1)
    u, c = np.unique(e, axis=0, return_counts=True)
    return u, c


def test_embedded_circle_mesh_is_a_conforming_triangulation_of_the_box(circ):
    m = circ
    x, y, t = m["x"], m["y"], m["tri"].astype(np.int64)
    a = 0.5 * ((x[t[:, 1]] - x[t[:, 0]]) * (y[t[:, 2]] - y[t[:, 0]])
               - (x[t[:, 2]] - x[t[:, 0]]) * (y[t[:, 1]] - y[t[:, 0]]))
    h = m["h"][0]
    assert np.all(a > 0.1 * h * h)                          # counter-clockwise, no slivers
    side = (x.max() - x.min(), y.max() - y.min())
    assert abs(a.sum() - side[0] * side[1]) < 1e-12 * side[0] * side[1]   # tiles the box
    assert len(np.unique(t)) == len(x)                      # every vertex used
    u, c = _edges(t)
    assert set(c.tolist()) <= {1, 2}                        # conforming
    b = u[c == 1]                                           # boundary edges lie on the box sides
    xb, yb = x[b], y[b]
    on = lambda v, s: np.all(np.isclose(v, s), axis=1)
    assert np.all(on(xb, x.min()) | on(xb, x.max()) | on(yb, y.min()) | on(yb, y.max()))
    # Euler characteristic of a disc
    assert len(x) - len(u) + len(t) == 1


def test_embedded_circle_vertices_lie_on_the_circle_and_form_a_mesh_line(circ):
    m = circ
    x, y = m["x"], m["y"]
    on = np.nonzero(m["on_circle"])[0]
    assert np.abs(np.hypot(x[on], y[on]) - m["radius"]).max() < 2e-16
    # consecutive circle vertices (by angle) are joined by an edge: the circle is a mesh line
    order = on[np.argsort(np.arctan2(y[on], x[on]))]
    u, _ = _edges(m["tri"].astype(np.int64))
    E = set(map(tuple, u.tolist()))
    for i in range(len(order)):
        a, b = order[i], order[(i + 1) % len(order)]
        assert (min(a, b), max(a, b)) in E
    # no other vertex within half a spacing of the circle
    r = np.hypot(x, y)
    others = ~m["on_circle"]
    assert np.abs(r[others] - m["radius"]).min() >= 0.5 * m["h"][0] - 1e-15


def test_embedded_circle_ghosts_copy_physical_boundary_vertices(circ):
    m = circ
    x, y = m["x"], m["y"]
    g, d = m["ghost_ids"], m["ghost_donor"]
    assert len(np.intersect1d(g, d)) == 0
    assert np.all((np.abs(x[g]) > 1.0 + 1e-12) | (np.abs(y[g]) > 1.0 + 1e-12))
    assert np.all(np.isclose(np.maximum(np.abs(x[d]), np.abs(y[d])), 1.0))
    # the donor is the ghost clamped onto the box
    np.testing.assert_allclose(x[d], np.clip(x[g], -1.0, 1.0), atol=1e-14)
    np.testing.assert_allclose(y[d], np.clip(y[g], -1.0, 1.0), atol=1e-14)


def test_embedded_circle_mesh_is_seeded():
    a = synth.embedded_circle_box(16, seed=8)
    b = synth.embedded_circle_box(16, seed=8)
    c = synth.embedded_circle_box(16, seed=9)
    np.testing.assert_array_equal(a["tri"], b["tri"])
    np.testing.assert_array_equal(a["x"], b["x"])
    assert not np.array_equal(a["x"], c["x"])


def test_circular_sod_state(circ):
    m = circ
    U = synth.circular_sod(m)
    r = np.hypot(m["x"], m["y"])
    inside = (r < 0.5) & ~m["on_circle"]
    np.testing.assert_array_equal(U[0, inside], 1.0)
    np.testing.assert_allclose(U[3, inside], 2.5, rtol=1e-15)         # p / (gamma - 1)
    np.testing.assert_array_equal(U[0, ~inside], 0.125)
    np.testing.assert_allclose(U[3, ~inside], 0.25, rtol=1e-15)
    assert np.all(U[1:3] == 0.0) and np.all(U[4:] == 0.0)


@pytest.mark.parametrize("kind", ["periodic", "box", "circle"])
def test_vertex_areas_tile_the_domain(kind):
    """The objective weights: one third of each incident triangle; they sum to the domain area
    (periodic triangles by the minimum image) and are positive."""
    if kind == "periodic":
        m, area = synth.jittered_grid(12, 9, 10.0, 7.0, seed=4), 70.0
    elif kind == "box":
        m, area = synth.jittered_box_with_ghosts(10, 10, (0.0, 1.0), (0.0, 2.0), 2, seed=4), None
    else:
        m, area = synth.embedded_circle_box(16, seed=8), None
    A = synth.vertex_areas(m)
    assert np.all(A > 0)
    if area is None:
        area = (m["x"].max() - m["x"].min()) * (m["y"].max() - m["y"].min())
    assert abs(A.sum() - area) < 1e-12 * area
