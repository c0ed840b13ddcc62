"""CPU tests of the native library: it loads, exports every entry point of include/hfd.h, and
its host preprocessing agrees with the oracle (no GPU is used)."""
import os
import re

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2109_01286_gb300 as p
    return p


def test_library_exports_every_declared_entry_point(pkg):
    hdr = open(os.path.join(ROOT, "include", "hfd.h")).read()
    declared = set(re.findall(r"\b(hfd_[a-z0-9_]+)\s*\(", hdr))
    assert len(declared) >= 20
    lib = pkg.hfd._lib
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert declared == set(pkg.hfd.EXPORTED)


def test_library_exports_every_3d_entry_point(pkg):
    """The three-dimensional extension's header (include/hfd3d.h): every declared entry point
    is exported and bound."""
    from paper_2109_01286_gb300 import hfd3d
    hdr = open(os.path.join(ROOT, "include", "hfd3d.h")).read()
    declared = set(re.findall(r"\b(hfd3_[a-z0-9_]+)\s*\(", hdr))
    assert len(declared) >= 10
    for name in sorted(declared):
        assert hasattr(pkg.hfd._lib, name), name
    assert declared == set(hfd3d.EXPORTED)


def test_3d_host_preprocessing_matches_the_oracle(pkg):
    """The 3D preprocessing built host-only (hfd3_options.host_only, no GPU) against the 3D
    oracle on a 6^3 box: edges, stencils, ranks and two-level sets identical; frames and 3-node
    weights to rounding; 5-node weights within their systems' conditioning; divergence rows to
    1e-12 of each row's scale.  Device calls on a host-only mesh are refused."""
    import ctypes
    from paper_2109_01286_gb300 import hfd3d
    from oracle import hfd3d as O
    from synth import three_d as T
    m = T.periodic_tet_box(6, 6, 6, 10.0, 10.0, 10.0, seed=3)
    P = O.prepare(m)
    mesh = hfd3d.Mesh3(m, host_only=1)
    topo = P.topo
    V = topo["V"]
    assert np.array_equal(mesh.prep_get("edges").reshape(-1, 2), topo["edges"])
    assert np.array_equal(mesh.prep_get("sten").reshape(-1, 6), P.stencil)
    assert np.array_equal(mesh.prep_get("rank").reshape(-1, 2), P.rank)
    np.testing.assert_allclose(mesh.prep_get("frame").reshape(-1, 9),
                               np.concatenate([P.normal, P.t1, P.t2], 1), atol=1e-15)
    np.testing.assert_allclose(mesh.prep_get("w3").reshape(P.w3.shape), P.w3, rtol=1e-12, atol=1e-14)
    d5 = np.abs(mesh.prep_get("w5").reshape(P.w5.shape) - P.w5).max(axis=(1, 2))
    assert d5.max() < 1e-4 and np.median(d5) < 1e-9
    vptr, vidx = mesh.prep_get("vptr"), mesh.prep_get("vidx")
    eptr, eidx = mesh.prep_get("eptr"), mesh.prep_get("eidx")
    cv, ce = mesh.prep_get("cv").reshape(-1, 4, 3), mesh.prep_get("ce").reshape(-1, 4)
    for v in range(V):
        verts, edges = O.vertex_stencil(topo, v)
        assert np.array_equal(vidx[vptr[v]:vptr[v + 1]], verts)
        assert np.array_equal(eidx[eptr[v]:eptr[v + 1]], edges)
        if v % 5:
            continue
        for r in range(4):
            row = P.D[r].getrow(v).toarray()[0]
            ref = np.concatenate([row[(3 * verts[:, None] + np.arange(3)).ravel()], row[3 * V + edges]])
            lib = np.concatenate([cv[vptr[v]:vptr[v + 1], r, :].ravel(), ce[eptr[v]:eptr[v + 1], r]])
            assert np.abs(lib - ref).max() < 1e-12 * np.abs(ref).max()
    info = mesh.info()
    assert info["nv"] == V and info["nedges"] == len(topo["edges"])
    assert info["div_nv_total"] == len(vidx) and info["div_ne_total"] == len(eidx)
    # no device arrays: residual and steps are refused before any pointer is used
    lib = pkg.hfd._lib
    fake = ctypes.c_void_p(16)
    assert lib.hfd3_residual(mesh._h, fake, ctypes.c_void_p(32), None) == 9
    assert lib.hfd3_steps(mesh._h, fake, 0.1, 1, None) == 9
    assert lib.hfd3_check(mesh._h) == 0
    # coefficient arrays can still be replaced on the host
    mesh.prep_set("w5", P.w5)
    assert np.array_equal(mesh.prep_get("w5").reshape(P.w5.shape), P.w5)


def test_bounds_checked_build_exports_the_same_entry_points(pkg):
    """The bounds-checked library (kernels built with -DHFD_CHECK=1) is built beside the normal
    one and exports every entry point of include/hfd.h."""
    import ctypes
    path = os.path.join(os.path.dirname(pkg.hfd.__file__), "_lib", "libhfd_check.so")
    lib = ctypes.CDLL(path)
    for name in pkg.hfd.EXPORTED:
        assert hasattr(lib, name), name


def test_index_arrays_are_read_only_through_prep_set(pkg):
    """Only coefficient arrays may be overwritten: the index streams the kernels gather through
    stay those of the validated mesh."""
    m = synth.jittered_grid(8, 8, 1.0, 1.0, seed=0)
    prep = pkg.Prep(m)
    for name in ("stencil", "flux_edges", "div_vidx", "div_eidx", "div_vptr", "div_eptr", "active",
                 "edges"):
        with pytest.raises(pkg.HfdError):
            prep.set(name, prep.get(name))
    prep.set("w5", prep.get("w5"))


def test_default_options(pkg):
    o = pkg.options()
    assert (o.div_degree, o.visc_degree, o.precision, o.renumber) == (5, 4, 0, 1)
    assert (o.sens_lo, o.sens_hi, o.weno_eps, o.cfl) == (0.01, 0.79, 1e-2, 0.3)


@pytest.fixture(scope="module")
def c1(pkg):
    m = synth.jittered_grid(40, 40, 10.0, 10.0, seed=1)
    return m, oracle.prepare(m), pkg.Prep(m)


def test_host_prep_discrete_choices_match_oracle(c1):
    m, P, prep = c1
    np.testing.assert_array_equal(prep.get("edges").reshape(-1, 2), P.topo["edges"])
    np.testing.assert_array_equal(prep.get("flux_edges"), P.edges)
    np.testing.assert_array_equal(prep.get("stencil").reshape(-1, 6), P.stencil)
    np.testing.assert_array_equal(prep.get("rank").reshape(-1, 2), P.rank)
    np.testing.assert_array_equal(prep.get("active"), P.active)
    np.testing.assert_array_equal(prep.get("div_degree"), P.div_degree)


def test_host_prep_coefficients_match_oracle(c1):
    m, P, prep = c1
    from gpu_helpers import oracle_blocks
    # 3-node weights: both sides round the exact (rational) weights -> equal
    np.testing.assert_allclose(prep.get("w3").reshape(-1, 2, 3, 3), P.w3, rtol=0, atol=1e-15)
    np.testing.assert_array_equal(prep.get("normal").reshape(-1, 2), P.normal)
    # divergence rows: full-rank least squares, condition ~1e3
    ref = oracle_blocks(P, len(m["x"]))["div_coef"]
    got = prep.get("div_coef")
    assert np.abs(got - ref).max() < 1e-11 * np.abs(ref).max()
    # 5-node weights: truncated pseudo-inverses; most agree to ~1e-13, the ill-conditioned few
    # (small retained singular values) to ~1e-7
    d = np.abs(prep.get("w5").reshape(-1, 2, 15) - P.w5).max(axis=(1, 2))
    assert np.median(d) < 1e-12
    assert np.mean(d < 1e-10) > 0.95
    assert d.max() < 1e-6


def test_host_prep_five_node_gaps_follow_from_conditioning(c1):
    """The library's 5-node weights (one-sided Jacobi SVD) and the oracle's (LAPACK) are two
    backward-stable evaluations of a truncated pseudo-inverse (Sec. 2.2, R3).  Its first-order
    sensitivity to a relative perturbation eps of the 15x15 system is eps * sigma_max /
    sigma_kept (the dropped singular value is the structural zero of the squared conic), so on
    every edge side the two must agree to within a small multiple of that bound: the gaps of up
    to ~1e-7 are the stencils' conditioning, not an error of either side."""
    m, P, prep = c1
    from oracle import hfd_oracle as H
    wl = prep.get("w5").reshape(-1, 2, 15)
    worst = 0.0
    for i, e in enumerate(P.edges):
        ids, rel, ell, n = H.edge_geometry(m, P.topo, int(e))
        for side, five in enumerate([H.LEFT5, H.RIGHT5]):
            X = rel[five] / ell
            p, px, py = H.taylor_basis(X[:, 0], X[:, 1], 4)
            A = np.zeros((15, 15))
            A[0::3], A[1::3], A[2::3] = p.T, px.T, py.T
            S = np.linalg.svd(A, compute_uv=False)
            kappa = S[0] / S[P.rank[i, side] - 1]
            gap = np.abs(wl[i, side] - P.w5[i, side]).max()
            worst = max(worst, gap / (np.finfo(float).eps * kappa))
    assert worst < 4.0, worst


@pytest.mark.parametrize("n", [16, 24])
def test_host_prep_viscous_rows_match_oracle(pkg, n):
    m = synth.jittered_grid(n, n, 2 * np.pi, 2 * np.pi, seed=3)
    P = oracle.prepare(m, oracle.Options(viscous=True, mu=0.01))
    prep = pkg.Prep(m, viscous=True, mu=0.01)
    from gpu_helpers import oracle_blocks
    ref = oracle_blocks(P, len(m["x"]))["visc_coef"]
    got = prep.get("visc_coef")
    assert np.abs(got - ref).max() < 1e-10 * np.abs(ref).max()


def test_host_prep_viscous_degree_drop_matches_oracle(pkg):
    """R6b on both sides: the default bound on the 48 x 48 torus (a handful of drops) and a
    tight bound on 16 x 16 (a quarter of the vertices drop) give the same degrees and rows."""
    from gpu_helpers import oracle_blocks
    m = synth.jittered_grid(48, 48, 2 * np.pi, 2 * np.pi, seed=3)
    topo = oracle.build_topology(m)
    opts = oracle.Options(viscous=True, mu=0.01)
    want = np.array([oracle.visc_rows(m, topo, v, opts)[2] for v in range(len(m["x"]))])
    prep = pkg.Prep(m, viscous=True, mu=0.01)
    got = prep.get("visc_degree")
    np.testing.assert_array_equal(got, want)
    assert 0 < np.sum(got < 4) < 0.01 * len(got)
    m = synth.jittered_grid(16, 16, 2 * np.pi, 2 * np.pi, seed=3)
    kw = dict(viscous=True, mu=0.01, visc_coef_max=1.5)
    P = oracle.prepare(m, oracle.Options(**kw))
    prep = pkg.Prep(m, **kw)
    np.testing.assert_array_equal(prep.get("visc_degree"), P.visc_degree)
    assert len(set(P.visc_degree.tolist())) >= 2
    ref = oracle_blocks(P, len(m["x"]))["visc_coef"]
    assert np.abs(prep.get("visc_coef") - ref).max() < 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("kind", ["periodic", "ghosts"])
def test_host_prep_conservative_matches_oracle(pkg, kind):
    """Conservative variant: dual faces, cell areas and flux directions bit-identical to the
    oracle's; divergence rows (finite-volume value rows, least-squares derivative rows with
    dual-normal edge rows) to rounding."""
    from gpu_helpers import oracle_blocks
    if kind == "periodic":
        m = synth.jittered_grid(16, 16, 1.0, 1.0, seed=3)
    else:
        m = synth.jittered_box_with_ghosts(12, 10, (0.0, 1.0), (0.0, 1.0), 5, seed=2)
    P = oracle.prepare(m, oracle.Options(conservative=True))
    prep = pkg.Prep(m, conservative=True)
    S, A = oracle.hfd_oracle.dual_faces(m, P.topo)
    np.testing.assert_array_equal(prep.get("dual_S").reshape(-1, 2), S)
    np.testing.assert_array_equal(prep.get("dual_A"), A)
    np.testing.assert_array_equal(prep.get("normal").reshape(-1, 2), P.normal)
    ref = oracle_blocks(P, len(m["x"]))["div_coef"]
    assert np.abs(prep.get("div_coef") - ref).max() < 1e-12 * np.abs(ref).max()


def test_host_prep_with_ghosts_matches_oracle(pkg):
    m = synth.jittered_box_with_ghosts(20, 16, (0.0, 1.0), (0.0, 1.0), 5, seed=2)
    P = oracle.prepare(m)
    prep = pkg.Prep(m)
    np.testing.assert_array_equal(prep.get("flux_edges"), P.edges)
    np.testing.assert_array_equal(prep.get("stencil").reshape(-1, 6), P.stencil)
    np.testing.assert_array_equal(prep.get("active"), P.active)


def test_host_prep_on_embedded_circle_delaunay_mesh_matches_oracle(pkg):
    """A Delaunay mesh (Sec. 3.3 circular Sod, vertex valences 4-9, a ring of vertices on the
    circle) instead of a split grid: same discrete choices and coefficients."""
    m = synth.embedded_circle_box(16, seed=8)
    P = oracle.prepare(m)
    prep = pkg.Prep(m)
    from gpu_helpers import oracle_blocks
    np.testing.assert_array_equal(prep.get("edges").reshape(-1, 2), P.topo["edges"])
    np.testing.assert_array_equal(prep.get("flux_edges"), P.edges)
    np.testing.assert_array_equal(prep.get("stencil").reshape(-1, 6), P.stencil)
    np.testing.assert_array_equal(prep.get("rank").reshape(-1, 2), P.rank)
    np.testing.assert_array_equal(prep.get("active"), P.active)
    np.testing.assert_array_equal(prep.get("div_degree"), P.div_degree)
    deg = np.bincount(np.asarray(P.topo["edges"]).ravel(), minlength=len(m["x"]))
    assert deg[P.active].min() <= 4 and deg[P.active].max() >= 8
    ref = oracle_blocks(P, len(m["x"]))["div_coef"]
    assert np.abs(prep.get("div_coef") - ref).max() < 1e-11 * np.abs(ref).max()
    d = np.abs(prep.get("w5").reshape(-1, 2, 15) - P.w5).max(axis=(1, 2))
    assert np.median(d) < 1e-12 and d.max() < 1e-6


def test_allocator_and_flux_options_are_checked(pkg):
    with pytest.raises(ValueError):
        pkg.options(allocator="malloc")
    assert pkg.options(flux="rusanov").flux == 1 and pkg.options().flux == 0
    m = synth.jittered_grid(8, 8, 1.0, 1.0, seed=0)
    d, keep = pkg.hfd._desc(m)
    h = pkg.hfd._P()
    ct = pkg.hfd.ctypes
    bad = pkg.options(flux=2)
    assert pkg.hfd._lib.hfd_prep_create(ct.byref(d), ct.byref(bad), ct.byref(h)) == 1
    assert pkg.options(force_branch="weno").force_branch == 2 and pkg.options().force_branch == 0
    bad = pkg.options(force_branch=3)
    assert pkg.hfd._lib.hfd_prep_create(ct.byref(d), ct.byref(bad), ct.byref(h)) == 1
    o = pkg.options(allocator="torch")
    assert bool(o.dev_alloc) and bool(o.dev_free)
    o.dev_free = pkg.hfd._FREE_FN()          # only one of the two callbacks: rejected
    assert pkg.hfd._lib.hfd_prep_create(ct.byref(d), ct.byref(o), ct.byref(h)) == 1


def test_invalid_meshes_are_rejected(pkg):
    m = synth.jittered_grid(6, 6, 1.0, 1.0, seed=0)
    bad = dict(m)
    bad["tri"] = m["tri"].copy()
    bad["tri"][0, 0] = 10 ** 6
    with pytest.raises(pkg.HfdError) as e:
        pkg.Prep(bad)
    assert e.value.status == 2
    bad = dict(m)
    bad["tri"] = np.concatenate([m["tri"], m["tri"][:1]])      # edge in three triangles
    with pytest.raises(pkg.HfdError) as e:
        pkg.Prep(bad)
    assert e.value.status == 2
    with pytest.raises(pkg.HfdError) as e:
        pkg.Prep(m, div_degree=9)
    assert e.value.status == 1
    # two triangles: no edge has enough neighbours for a 6-node stencil
    tiny = {"x": np.array([0.0, 1.0, 1.0, 0.0]), "y": np.array([0.0, 0.0, 1.0, 1.0]),
            "tri": np.array([[0, 1, 2], [0, 2, 3]]), "periodic_x": False, "periodic_y": False}
    with pytest.raises(pkg.HfdError) as e:
        pkg.Prep(tiny)
    assert e.value.status == 3


def test_roofline_accounting_matches_the_per_vertex_stage_budget(pkg):
    """bench.py's algorithmic bytes per launch (the numerator of the roofline fractions), summed
    over the three kernels of a stage on a periodic mesh, per vertex: about 4.0 KB in FP64 and
    2.3 KB in FP32 bulk (the budget of divergence coefficients, edge weights, indices, state,
    fluxes and normals), and the divergence's share is the largest."""
    import bench
    m = synth.jittered_grid(40, 40, 10.0, 10.0, seed=1)
    prep = pkg.Prep(m)
    vptr, eptr = prep.get("div_vptr"), prep.get("div_eptr")
    stats = {"nv": len(m["x"]), "nactive": len(prep.get("active")),
             "nflux_edges": len(prep.get("flux_edges")),
             "div_nv_total": int(vptr[-1]), "div_ne_total": int(eptr[-1])}
    for T, lo, hi in ((8, 3500, 4600), (4, 1900, 2800)):
        c = bench.algorithmic_costs(stats, T)
        per_vertex = sum(c[k]["bytes"] for k in ("vertex", "edge", "div")) / stats["nv"]
        assert lo < per_vertex < hi, (T, per_vertex)
        assert c["div"]["bytes"] > c["edge"]["bytes"] > c["vertex"]["bytes"]
        assert c["ghost"]["bytes"] == 0                       # periodic: no ghost vertices
    # the flops: 48 per stencil vertex and 24 per stencil edge (12 rows x 2 or 1 multiply-adds)
    c = bench.algorithmic_costs(stats, 8)
    assert c["div"]["flops"] == 48 * vptr[-1] + 24 * eptr[-1] + 48 * stats["nactive"]
